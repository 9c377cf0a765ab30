// Host side of the batched scan: a plan lays out the tiles of many columns,
// keeps a device descriptor table, and records one CUDA graph per plan:
//   descriptors H2D -> reset results/counters -> the width groups' kernels
// (results are copied back to the host after the replay only when a caller
// asks for host results).
// Running the plan again with new predicates only rewrites the pinned
// descriptor table and replays the graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/gbscan.h"
#include "batch_kernels.cuh"

#include "internal.h"

namespace {

scan_status bfail(scan_status s, const char* msg)
{
    gb_set_last_error(msg);
    return s;
}

scan_status bcuda(cudaError_t e, const char* what)
{
    static thread_local char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    gb_set_last_error(buf);
    return e == cudaErrorMemoryAllocation ? SCAN_ENOMEM : SCAN_ECUDA;
}

#define BT_CUDA(call)                                 \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return bcuda(e_, #call); \
    } while (0)

int batch_grid() { return gb_device_sms(); }


// Control words after the results: one pop counter per width group (u32),
// then the status word at u32 index kMaxGroups.
constexpr size_t kMaxGroups = 64;
constexpr size_t kCtlWords = 40;  // u64 words: 64 + 1 u32 fit in 33
constexpr int kBranches = 8;      // concurrent chains of width-group kernels in the graph
constexpr int kPairChains = 2;    // chains 0 and 1: the large groups, narrow and wide widths
// A group's time on the whole GPU by the bandwidth law, with GB300 figures
// (copy bandwidth 6.7 TB/s, branch-free decode 4.3 Tvalues/s), in
// microseconds; its packed bytes and values count whole columns (zone skipping
// only shortens it).
double law_us(double bytes, int b) { return std::max(bytes / 6.7e6, bytes * 8.0 / b / 4.3e6); }
// Groups shorter than this run on the small-group chains (2..7).
constexpr double kSmallGroupUs = 16.0;
// A group of this law time or more gets two CTAs per SM; a shorter one a
// proportional share (fewer warps to start, to pop and to drain).
constexpr double kFullGridUs = 10.0;

}  // namespace

struct scan_batch {
    uint32_t ncols = 0;
    std::vector<const scan_column*> cols;
    std::vector<int> kernel_of;        // 0 branch-free, 1 branchy
    std::vector<uint32_t> zone;        // 1 if the column skips by zone map
    std::vector<uint32_t> slot_of;     // index of the column in the descriptor table
    uint32_t ncol_k[2] = {0, 0};
    uint32_t ntiles_k[2] = {0, 0};
    uint32_t chunk_k[2] = {1, 1};
    uint32_t tiles_per_pop = 0;
    struct Group {
        int kernel, b;
        uint32_t first, count, ntiles, chunk;
        int grid;
        uint32_t chunk_off;  // offset of this group's chunk -> column table
        gb::LaunchShape shape;  // warps, stages and tile blocks of this width group
        double bytes;           // packed bytes of its columns
    };
    std::vector<Group> groups;  // one width-specialised launch each
    uint32_t* d_chunk_col = nullptr;  // all groups' chunk -> first-column tables
    size_t chunk_cap = 0;
    gb::BatchCol* h_table = nullptr;   // pinned
    gb::BatchCol* d_table = nullptr;
    unsigned long long* d_results = nullptr;  // 4 words per column, then 2 pop counters + status
    scan_result* h_results = nullptr;  // pinned copy of the results
    cudaStream_t capture_stream = nullptr;
    cudaStream_t branch[kBranches] = {};  // capture-time branches (one graph node chain each)
    cudaEvent_t fork = nullptr, join[kBranches] = {};
    cudaGraphExec_t graph = nullptr;
};

namespace gb {
static cudaError_t launch_batch_kernel(bool branchy, int b, const BatchParams& p, int warps, int grid,
                                       cudaStream_t st)
{
    return gb_launch_batch(branchy, b, p, warps, grid, st);
}
}  // namespace gb

namespace {

// Lay out the tiles for the current strategies: branch-free columns first,
// and within each kernel by width, one width-specialised launch per group,
// so that an SM runs at most two widths' decode code at a time (one CTA of
// each graph chain; a kernel holding all 32 fully unrolled width variants
// thrashed the instruction cache).
scan_status layout(scan_batch* bt)
{
    std::vector<uint32_t> order;
    std::vector<uint32_t> width(bt->ncols);
    for (uint32_t i = 0; i < bt->ncols; ++i) {
        const uint2* zm = nullptr;
        const uint32_t* pk;
        uint64_t n;
        uint32_t b, base;
        gb_column_view(bt->cols[i], &pk, &n, &b, &base, &zm);
        width[i] = b;
    }
    for (int k = 0; k < 2; ++k)
        for (uint32_t b = 1; b <= 32; ++b)
            for (uint32_t i = 0; i < bt->ncols; ++i)
                if (bt->kernel_of[i] == k && width[i] == b) order.push_back(i);
    const size_t table_bytes = std::max<size_t>(1, bt->ncols) * sizeof(gb::BatchCol);
    std::memset(bt->h_table, 0, table_bytes);
    uint32_t tiles[2] = {0, 0};
    bt->ncol_k[0] = bt->ncol_k[1] = 0;
    bt->groups.clear();
    uint32_t group_tiles = 0;
    for (uint32_t j = 0; j < order.size(); ++j) {
        const uint32_t i = order[j];
        const int k = bt->kernel_of[i];
        if (bt->groups.empty() || bt->groups.back().kernel != k ||
            bt->groups.back().b != static_cast<int>(width[i])) {
            scan_batch::Group g{k, static_cast<int>(width[i]), j, 0, 0, 1, 1, 0, {}, 0.0};
            g.shape = gb_shape_for(g.b, k == 1 ? gb::kOpBatchBR : gb::kOpBatchBF);
            bt->groups.push_back(g);
            group_tiles = 0;
        }
        const uint2* zm = nullptr;
        const uint32_t* pk;
        uint64_t n;
        uint32_t b, base;
        gb_column_view(bt->cols[i], &pk, &n, &b, &base, &zm);
        gb::BatchCol& d = bt->h_table[j];
        d.packed = pk;
        d.zonemap = zm;
        d.n = n;
        d.b = b;
        d.base = base;
        d.tile_blocks = static_cast<uint32_t>(bt->groups.back().shape.tile_blocks);
        d.tile_begin = group_tiles;  // tile numbers restart in every width group
        d.out = i;
        const uint64_t nblocks = (n + 1023u) >> 10;
        const uint64_t t = (nblocks + d.tile_blocks - 1) / d.tile_blocks;
        if (group_tiles + t > 0xffffffffull) return bfail(SCAN_EINVAL, "too many tiles in one batch");
        group_tiles += static_cast<uint32_t>(t);
        tiles[k] += static_cast<uint32_t>(t);
        bt->groups.back().bytes += static_cast<double>(nblocks) * 128.0 * b;
        bt->groups.back().count += 1;
        bt->groups.back().ntiles = group_tiles;
        bt->slot_of[i] = j;
        bt->ncol_k[k] += 1;
    }
    for (int k = 0; k < 2; ++k) bt->ntiles_k[k] = tiles[k];
    if (bt->groups.size() > kMaxGroups) return bfail(SCAN_EINVAL, "too many width groups");
    // per group: two CTAs per SM for a group of kFullGridUs or more, a share
    // in proportion to its law time below that (and a tile per warp at
    // least), pops of about a quarter of a warp's share (at least 4 tiles),
    // and a host-built table of each pop's first column.  Two CTAs per SM let
    // the block scheduler give every SM one CTA of each concurrent chain; with
    // one per SM the chains split the SMs between them and the replay took
    // 22% longer.  Full grids for small groups cost 5-21% on batches of 64 and
    // 512 columns (thousands of warps popping a few tiles from one counter).
    std::vector<uint32_t> chunk_col;
    const uint64_t cap = 2ull * static_cast<uint64_t>(batch_grid());
    for (auto& g : bt->groups) {
        const uint64_t gw = static_cast<uint64_t>(g.shape.warps);
        const uint64_t by_tiles = (static_cast<uint64_t>(g.ntiles) + gw - 1) / gw;
        const uint64_t by_time =
            static_cast<uint64_t>(std::ceil(static_cast<double>(cap) * law_us(g.bytes, g.b) / kFullGridUs));
        g.grid = static_cast<int>(std::max<uint64_t>(1, std::min({by_tiles, by_time, cap})));
        const uint32_t warps = static_cast<uint32_t>(g.grid * gw);
        const uint32_t c = bt->tiles_per_pop ? bt->tiles_per_pop : std::max<uint32_t>(4, g.ntiles / (4 * warps));
        g.chunk = std::min<uint32_t>(c, 1024);
        g.chunk_off = static_cast<uint32_t>(chunk_col.size());
        uint32_t col = g.first;
        for (uint64_t t0 = 0; t0 < g.ntiles; t0 += g.chunk) {
            while (col + 1 < g.first + g.count && bt->h_table[col + 1].tile_begin <= t0) ++col;
            chunk_col.push_back(col - g.first);
        }
    }
    if (chunk_col.size() > bt->chunk_cap) {
        if (bt->d_chunk_col) cudaFree(bt->d_chunk_col);
        bt->d_chunk_col = nullptr;
        bt->chunk_cap = 0;
        if (cudaMalloc(reinterpret_cast<void**>(&bt->d_chunk_col), chunk_col.size() * sizeof(uint32_t)) != cudaSuccess)
            return bfail(SCAN_ENOMEM, "chunk table allocation");
        bt->chunk_cap = chunk_col.size();
    }
    if (!chunk_col.empty() &&
        cudaMemcpy(bt->d_chunk_col, chunk_col.data(), chunk_col.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) !=
            cudaSuccess)
        return bfail(SCAN_ECUDA, "chunk table upload");
    if (bt->graph) {
        cudaGraphExecDestroy(bt->graph);
        bt->graph = nullptr;
    }
    return SCAN_OK;
}

scan_status set_strategy(scan_batch* bt, uint32_t i, scan_strategy st)
{
    const uint2* zm = nullptr;
    const uint32_t* pk;
    uint64_t n;
    uint32_t b, base;
    gb_column_view(bt->cols[i], &pk, &n, &b, &base, &zm);
    bt->kernel_of[i] = 0;
    bt->zone[i] = 0;
    switch (st) {
    case SCAN_AUTO:
    case SCAN_BRANCHFREE: break;
    case SCAN_BRANCHY: bt->kernel_of[i] = 1; break;
    case SCAN_ZONE_SKIP_BF: bt->zone[i] = 1; break;
    case SCAN_ZONE_SKIP_BR:
        bt->zone[i] = 1;
        bt->kernel_of[i] = 1;
        break;
    default: return bfail(SCAN_EINVAL, "unknown strategy");
    }
    if (bt->zone[i] && !zm) return bfail(SCAN_EINVAL, "a zone-skip column has no zone map (scan_zonemap_build first)");
    return SCAN_OK;
}

// Write the predicate fields of the pinned descriptor table.
void fill_predicates(scan_batch* bt, const scan_pred* preds)
{
    for (uint32_t i = 0; i < bt->ncols; ++i) {
        gb::BatchCol& d = bt->h_table[bt->slot_of[i]];
        const int64_t lo_v = static_cast<int64_t>(d.base);
        const int64_t hi_v = lo_v + (1ll << d.b);
        const int64_t lo = std::max(preds[i].lo, lo_v);
        const int64_t hi = std::min(preds[i].hi, hi_v);
        d.flags = bt->zone[i] ? gb::kColZone : 0u;
        if (lo >= hi || d.n == 0) {
            d.flags |= gb::kColEmpty;
            d.lo = 0;
            d.wm1 = 0;
            d.zlo = d.zhi = 0;
        } else {
            d.lo = static_cast<uint32_t>(lo - lo_v);
            d.wm1 = static_cast<uint32_t>(hi - lo - 1);
            d.zlo = static_cast<uint64_t>(lo);
            d.zhi = static_cast<uint64_t>(hi);
        }
    }
}

// Planner features, one CTA per column:
//   f0 = b / 32, f1 = log2(max(N, 1)) / 31,
//   f2 = (log10(max(sigma_hat, 1e-5)) + 5) / 5, sigma_hat = matches / values over up to
//        32 evenly spaced blocks (exact integer sample of the true predicate),
//   f3 = clustering c = 1 - mean_k (max_k - min_k + 1) / (colmax - colmin + 1) from the
//        zone map (0 without one): about 0 for shuffled data, about 1 for sorted data.
__global__ void __launch_bounds__(256) k_batch_features(const gb::BatchCol* __restrict__ cols, float* feats)
{
    __shared__ unsigned long long red_a[8], red_b[8];
    __shared__ double red_d[8];
    const gb::BatchCol c = cols[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t nblocks = (c.n + 1023u) >> 10;
    const uint32_t S = static_cast<uint32_t>(nblocks < 32 ? nblocks : 32);
    const uint64_t mask = (c.b == 32) ? 0xffffffffull : ((1ull << c.b) - 1ull);
    unsigned long long match = 0, seen = 0;
    for (uint32_t idx = threadIdx.x; idx < S * 1024u; idx += blockDim.x) {
        const uint32_t j = idx >> 10, pos = idx & 1023u;
        const uint64_t k = static_cast<uint64_t>(j) * nblocks / S;
        if ((k << 10) + pos >= c.n) continue;
        ++seen;
        if (c.flags & gb::kColEmpty) continue;
        const uint32_t l = pos & 31u, row = pos >> 5;
        const uint32_t bit = row * c.b, w = bit >> 5, sh = bit & 31u;
        const uint32_t* blk = c.packed + k * 32u * c.b;
        uint64_t win = __ldg(&blk[32u * w + l]);
        if (sh + c.b > 32u) win |= static_cast<uint64_t>(__ldg(&blk[32u * (w + 1u) + l])) << 32;
        const uint32_t u = static_cast<uint32_t>((win >> sh) & mask);
        if (u - c.lo <= c.wm1) ++match;
    }
    for (int o = 16; o; o >>= 1) {
        match += __shfl_xor_sync(0xffffffffu, match, o);
        seen += __shfl_xor_sync(0xffffffffu, seen, o);
    }
    if (lane == 0) {
        red_a[warp] = match;
        red_b[warp] = seen;
    }
    __syncthreads();
    unsigned long long tm = 0, ts = 0;
    for (int w = 0; w < 8; ++w) {
        tm += red_a[w];
        ts += red_b[w];
    }
    __syncthreads();
    // clustering from the zone map: column range, then the mean relative block range
    double mean_rel = 1.0;
    if (c.zonemap && nblocks) {
        unsigned long long mn = ~0ull, mx = 0;
        for (uint64_t k = threadIdx.x; k < nblocks; k += blockDim.x) {
            const uint2 z = __ldg(&c.zonemap[k]);
            mn = min(mn, static_cast<unsigned long long>(z.x));
            mx = max(mx, static_cast<unsigned long long>(z.y));
        }
        for (int o = 16; o; o >>= 1) {
            mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            red_a[warp] = mn;
            red_b[warp] = mx;
        }
        __syncthreads();
        unsigned long long cmn = ~0ull, cmx = 0;
        for (int w = 0; w < 8; ++w) {
            cmn = min(cmn, red_a[w]);
            cmx = max(cmx, red_b[w]);
        }
        const double span = static_cast<double>(cmx - cmn + 1ull);
        double acc = 0.0;
        for (uint64_t k = threadIdx.x; k < nblocks; k += blockDim.x) {
            const uint2 z = __ldg(&c.zonemap[k]);
            acc += static_cast<double>(static_cast<unsigned long long>(z.y) - z.x + 1ull) / span;
        }
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) red_d[warp] = acc;
        __syncthreads();
        double tot = 0.0;
        for (int w = 0; w < 8; ++w) tot += red_d[w];
        mean_rel = tot / static_cast<double>(nblocks);
    }
    if (threadIdx.x == 0) {
        const double sigma = ts ? static_cast<double>(tm) / static_cast<double>(ts) : 0.0;
        float* f = feats + 4ull * c.out;
        f[0] = static_cast<float>(c.b) / 32.f;
        f[1] = static_cast<float>(log2(c.n > 0 ? static_cast<double>(c.n) : 1.0) / 31.0);
        f[2] = static_cast<float>((log10(sigma > 1e-5 ? sigma : 1e-5) + 5.0) / 5.0);
        f[3] = static_cast<float>(c.zonemap ? 1.0 - mean_rel : 0.0);
    }
}

// Law fallback (Eq. 2 per strategy): the predicted time of strategy s is
//   max(bytes_s / beta, values_s / T_dec[s]); a zone skip reads the zone map
//   plus a fraction phi = min(1, sigma_hat + (1 - c) + 2 / blocks) of the blocks.
//   Strategies: 0 branch-free, 1 branchy, 2 zone-skip branch-free, 3 zone-skip branchy.
//   A zone strategy of a column without a zone map gets a negative time (unavailable).
__device__ void law_seconds(const float* f, const gb::BatchCol& c, float beta, const double (&tdec)[4],
                            double (&t)[4])
{
    const double n = static_cast<double>(c.n), nb = static_cast<double>((c.n + 1023u) >> 10);
    const double bytes = nb * 128.0 * c.b;
    const double sigma = pow(10.0, 5.0 * f[2] - 5.0);
    double phi = sigma + (1.0 - f[3]) + (nb > 0 ? 2.0 / nb : 1.0);
    phi = phi > 1.0 ? 1.0 : phi;
    const bool has_zone = c.zonemap != nullptr;
    for (int s = 0; s < 4; ++s) {
        const bool zone = s >= 2;
        const double rd = zone ? phi * bytes + 8.0 * nb : bytes;
        const double vals = zone ? phi * n : n;
        t[s] = (zone && !has_zone) ? -1.0 : fmax(rd / beta, vals / tdec[s]);
    }
}

__global__ void k_law_choose(const float* __restrict__ feats, const gb::BatchCol* __restrict__ cols,
                             uint32_t ncols, float beta, float t0, float t1, float t2, float t3,
                             int32_t* __restrict__ out)
{
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ncols) return;
    const gb::BatchCol c = cols[j];
    const double tdec[4] = {t0, t1, t2, t3};
    double t[4];
    law_seconds(feats + 4ull * c.out, c, beta, tdec, t);
    int best = 0;
    double bt = 1e300;
    for (int s = 0; s < 4; ++s) {
        if (t[s] < 0.0) continue;
        if (t[s] < bt) {
            bt = t[s];
            best = s;
        }
    }
    out[c.out] = best;
}

// The same law times as natural-log milliseconds, ncols x 4 (row = the
// column's position in the batch); an unavailable strategy gets kLawNoLogMs.
constexpr float kLawNoLogMs = 30.0f;
__global__ void k_law_times(const float* __restrict__ feats, const gb::BatchCol* __restrict__ cols,
                            uint32_t ncols, float beta, float t0, float t1, float t2, float t3,
                            float* __restrict__ out)
{
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ncols) return;
    const gb::BatchCol c = cols[j];
    const double tdec[4] = {t0, t1, t2, t3};
    double t[4];
    law_seconds(feats + 4ull * c.out, c, beta, tdec, t);
    for (int s = 0; s < 4; ++s)
        out[4ull * c.out + s] = t[s] < 0.0 ? kLawNoLogMs : static_cast<float>(log(t[s] * 1e3 + 1e-9));
}

}  // namespace

extern "C" {

scan_status scan_batch_create(scan_column* const* cols, uint32_t ncols, const scan_strategy* strategies,
                              uint32_t tiles_per_pop, void* stream, scan_batch** out)
{
    (void)stream;
    gb_set_last_error("");
    if (!out || (ncols && !cols)) return bfail(SCAN_EINVAL, "null pointer");
    *out = nullptr;
    for (uint32_t i = 0; i < ncols; ++i) {
        if (!cols[i]) return bfail(SCAN_EINVAL, "a column pointer is NULL");
        const uint32_t* pk;
        const uint2* zm;
        uint64_t n;
        uint32_t b, base;
        if (!gb_column_view(cols[i], &pk, &n, &b, &base, &zm))
            return bfail(SCAN_EINVAL, "batched scans take lane-interleaved columns");
    }
    auto* bt = new (std::nothrow) scan_batch();
    if (!bt) return bfail(SCAN_ENOMEM, "host allocation failed");
    bt->ncols = ncols;
    bt->tiles_per_pop = tiles_per_pop;
    bt->cols.assign(cols, cols + ncols);
    bt->kernel_of.assign(ncols, 0);
    bt->zone.assign(ncols, 0);
    bt->slot_of.assign(ncols, 0);
    for (uint32_t i = 0; i < ncols; ++i) {
        const scan_status s = set_strategy(bt, i, strategies ? strategies[i] : SCAN_BRANCHFREE);
        if (s != SCAN_OK) {
            delete bt;
            return s;
        }
    }
    const size_t table_bytes = std::max<size_t>(1, ncols) * sizeof(gb::BatchCol);
    const size_t res_bytes = (4ull * std::max<uint32_t>(1, ncols) + kCtlWords) * sizeof(unsigned long long);
    cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&bt->h_table), table_bytes);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&bt->d_table), table_bytes);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&bt->d_results), res_bytes);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&bt->h_results), res_bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bt->capture_stream, cudaStreamNonBlocking);
    for (int k = 0; k < kBranches && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&bt->branch[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->join[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->fork, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        scan_batch_destroy(bt);
        return bcuda(e, "batch allocation");
    }
    const scan_status s = layout(bt);
    if (s != SCAN_OK) {
        scan_batch_destroy(bt);
        return s;
    }
    *out = bt;
    return SCAN_OK;
}

scan_status scan_batch_destroy(scan_batch* bt)
{
    if (!bt) return SCAN_OK;
    cudaDeviceSynchronize();
    if (bt->graph) cudaGraphExecDestroy(bt->graph);
    if (bt->capture_stream) cudaStreamDestroy(bt->capture_stream);
    for (int k = 0; k < kBranches; ++k) {
        if (bt->branch[k]) cudaStreamDestroy(bt->branch[k]);
        if (bt->join[k]) cudaEventDestroy(bt->join[k]);
    }
    if (bt->fork) cudaEventDestroy(bt->fork);
    if (bt->h_table) cudaFreeHost(bt->h_table);
    if (bt->h_results) cudaFreeHost(bt->h_results);
    if (bt->d_table) cudaFree(bt->d_table);
    if (bt->d_results) cudaFree(bt->d_results);
    if (bt->d_chunk_col) cudaFree(bt->d_chunk_col);
    delete bt;
    return SCAN_OK;
}

scan_status scan_batch_set_strategies(scan_batch* bt, const scan_strategy* strategies)
{
    gb_set_last_error("");
    if (!bt || (bt->ncols && !strategies)) return bfail(SCAN_EINVAL, "null pointer");
    cudaDeviceSynchronize();  // a replay in flight may still read the table
    for (uint32_t i = 0; i < bt->ncols; ++i) {
        const scan_status s = set_strategy(bt, i, strategies[i]);
        if (s != SCAN_OK) return s;
    }
    return layout(bt);
}

scan_status scan_batch_features(scan_batch* bt, const scan_pred* preds, void* stream, float* dev_features)
{
    gb_set_last_error("");
    if (!bt || !dev_features || (bt->ncols && !preds)) return bfail(SCAN_EINVAL, "null pointer");
    if (!bt->ncols) return SCAN_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    BT_CUDA(cudaStreamSynchronize(st));
    fill_predicates(bt, preds);
    BT_CUDA(cudaMemcpyAsync(bt->d_table, bt->h_table, bt->ncols * sizeof(gb::BatchCol), cudaMemcpyHostToDevice, st));
    k_batch_features<<<bt->ncols, 256, 0, st>>>(bt->d_table, dev_features);
    BT_CUDA(cudaGetLastError());
    return SCAN_OK;
}

scan_status scan_batch_law_choose(scan_batch* bt, const float* dev_features, float beta_bytes_per_s,
                                  const float* t_dec_values_per_s, void* stream, int32_t* dev_choice)
{
    gb_set_last_error("");
    if (!bt || !dev_features || !dev_choice || !t_dec_values_per_s) return bfail(SCAN_EINVAL, "null pointer");
    if (!bt->ncols) return SCAN_OK;
    if (!(beta_bytes_per_s > 0.f)) return bfail(SCAN_EINVAL, "beta must be positive");
    for (int s = 0; s < 4; ++s)
        if (!(t_dec_values_per_s[s] > 0.f)) return bfail(SCAN_EINVAL, "every T_dec must be positive");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_law_choose<<<(bt->ncols + 255) / 256, 256, 0, st>>>(dev_features, bt->d_table, bt->ncols, beta_bytes_per_s,
                                                          t_dec_values_per_s[0], t_dec_values_per_s[1],
                                                          t_dec_values_per_s[2], t_dec_values_per_s[3], dev_choice);
    BT_CUDA(cudaGetLastError());
    return SCAN_OK;
}

scan_status scan_batch_law_times(scan_batch* bt, const float* dev_features, float beta_bytes_per_s,
                                 const float* t_dec_values_per_s, void* stream, float* dev_log_ms)
{
    gb_set_last_error("");
    if (!bt || !dev_features || !dev_log_ms || !t_dec_values_per_s) return bfail(SCAN_EINVAL, "null pointer");
    if (!bt->ncols) return SCAN_OK;
    if (!(beta_bytes_per_s > 0.f)) return bfail(SCAN_EINVAL, "beta must be positive");
    for (int s = 0; s < 4; ++s)
        if (!(t_dec_values_per_s[s] > 0.f)) return bfail(SCAN_EINVAL, "every T_dec must be positive");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_law_times<<<(bt->ncols + 255) / 256, 256, 0, st>>>(dev_features, bt->d_table, bt->ncols, beta_bytes_per_s,
                                                         t_dec_values_per_s[0], t_dec_values_per_s[1],
                                                         t_dec_values_per_s[2], t_dec_values_per_s[3], dev_log_ms);
    BT_CUDA(cudaGetLastError());
    return SCAN_OK;
}

scan_status scan_batch_exec(scan_batch* bt, const scan_pred* preds, void* stream, scan_result* host_out,
                            scan_result* dev_out)
{
    gb_set_last_error("");
    if (!bt || (bt->ncols && !preds)) return bfail(SCAN_EINVAL, "null pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the previous replay may still read the pinned table: wait for it
    BT_CUDA(cudaStreamSynchronize(st));
    fill_predicates(bt, preds);
    const size_t table_bytes = std::max<size_t>(1, bt->ncols) * sizeof(gb::BatchCol);
    const size_t res_words = 4ull * std::max<uint32_t>(1, bt->ncols) + kCtlWords;
    unsigned long long* ctl = bt->d_results + 4ull * std::max<uint32_t>(1, bt->ncols);
    if (!bt->graph) {
        // copy descriptors -> reset -> {one kernel per width group, as parallel
        // branches} -> copy results.  Branches let small groups run side by side
        // and fill each other's tails; a group's grid is sized to its work.
        cudaStream_t cs = bt->capture_stream;
        BT_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        cudaMemcpyAsync(bt->d_table, bt->h_table, table_bytes, cudaMemcpyHostToDevice, cs);
        cudaMemsetAsync(bt->d_results, 0, res_words * sizeof(unsigned long long), cs);
        cudaEventRecord(bt->fork, cs);
        // Large groups (law time kSmallGroupUs or more) on two chains: the
        // narrow half in ascending width, the wide half in descending width,
        // captured alternately.  At any moment a decode-bound kernel (small b)
        // runs beside a bandwidth-bound one (large b), one CTA of each per SM,
        // and both chains end on the middle widths.  (Eight chains in width
        // order, one CTA per SM: 0.97 ms on the 4096-column workload; these two
        // chains: 0.86-0.87 ms.  Halves cut by equal law time instead of equal
        // group counts: 0.93 ms.)  Small groups, whose time is mostly launch
        // and ramp, go round-robin on six more chains so that few of them queue
        // behind one another: 512 columns of 2^28 values in all took 0.38 ms
        // on the two chains and 0.23 ms this way.
        std::vector<size_t> live, small;
        for (size_t gi = 0; gi < bt->groups.size(); ++gi) {
            const auto& g = bt->groups[gi];
            if (!g.ntiles) continue;
            (law_us(g.bytes, g.b) < kSmallGroupUs ? small : live).push_back(gi);
        }
        const auto by_width = [&](size_t x, size_t y) { return bt->groups[x].b < bt->groups[y].b; };
        std::stable_sort(live.begin(), live.end(), by_width);
        std::stable_sort(small.begin(), small.end(), by_width);
        const size_t half = (live.size() + 1) / 2;
        std::vector<std::pair<size_t, int>> seq;  // (group, chain) in capture order
        for (size_t i = 0; i < small.size(); ++i)
            seq.push_back({small[i], kPairChains + static_cast<int>(i % (kBranches - kPairChains))});
        for (size_t i = 0; i < half; ++i) {
            seq.push_back({live[i], 0});
            if (half + i < live.size()) seq.push_back({live[live.size() - 1 - i], 1});
        }
        bool used[kBranches] = {};
        for (const auto& [gi, k] : seq) {
            const auto& g = bt->groups[gi];
            cudaStream_t bs = bt->branch[k];
            if (!used[k]) cudaStreamWaitEvent(bs, bt->fork, 0);  // joins the capture
            used[k] = true;
            gb::BatchParams p{};
            p.cols = bt->d_table + g.first;
            p.chunk_col = bt->d_chunk_col + g.chunk_off;
            p.ncols = g.count;
            p.ntiles = g.ntiles;
            p.chunk = g.chunk;
            p.head = reinterpret_cast<unsigned int*>(ctl) + gi;
            p.results = bt->d_results;
            p.status = reinterpret_cast<unsigned int*>(ctl) + kMaxGroups;
            p.stages = static_cast<uint32_t>(g.shape.stages);
            p.slot_bytes = static_cast<uint32_t>(g.shape.tile_blocks) * 128u * static_cast<uint32_t>(g.b);
            gb::launch_batch_kernel(g.kernel == 1, g.b, p, g.shape.warps, g.grid, bs);
        }
        for (int k = 0; k < kBranches; ++k) {
            if (!used[k]) continue;
            cudaEventRecord(bt->join[k], bt->branch[k]);
            cudaStreamWaitEvent(cs, bt->join[k], 0);
        }
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(cs, &g);
        if (ec != cudaSuccess || !g) return bcuda(ec != cudaSuccess ? ec : cudaErrorUnknown, "graph capture");
        const cudaError_t ei = cudaGraphInstantiate(&bt->graph, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) return bcuda(ei, "cudaGraphInstantiate");
    }
    BT_CUDA(cudaGraphLaunch(bt->graph, st));
    if (dev_out)
        BT_CUDA(cudaMemcpyAsync(dev_out, bt->d_results, 4ull * bt->ncols * sizeof(unsigned long long),
                                cudaMemcpyDeviceToDevice, st));
    if (host_out) {  // results and control words back to the host only when asked for
        BT_CUDA(cudaMemcpyAsync(bt->h_results, bt->d_results, res_words * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, st));
        BT_CUDA(cudaStreamSynchronize(st));
        const unsigned int status = reinterpret_cast<const unsigned int*>(
            reinterpret_cast<const unsigned long long*>(bt->h_results) + 4ull * std::max<uint32_t>(1, bt->ncols))[kMaxGroups];
        if (status) return bfail(SCAN_ETIMEOUT, "a device-side wait timed out in the batch kernel");
        std::memcpy(host_out, bt->h_results, sizeof(scan_result) * bt->ncols);
    }
    return SCAN_OK;
}

scan_status scan_batch_status(scan_batch* bt, void* stream)
{
    gb_set_last_error("");
    if (!bt) return bfail(SCAN_EINVAL, "batch is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned long long* ctl = bt->d_results + 4ull * std::max<uint32_t>(1, bt->ncols);
    unsigned long long* h_ctl = reinterpret_cast<unsigned long long*>(bt->h_results) + 4ull * std::max<uint32_t>(1, bt->ncols);
    BT_CUDA(cudaMemcpyAsync(h_ctl, ctl, kCtlWords * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    BT_CUDA(cudaStreamSynchronize(st));
    if (reinterpret_cast<const unsigned int*>(h_ctl)[kMaxGroups])
        return bfail(SCAN_ETIMEOUT, "a device-side wait timed out in the batch kernel");
    return SCAN_OK;
}

scan_status scan_batch_autotune(scan_batch* bt, const scan_pred* preds, uint32_t reps, void* stream,
                                uint32_t* groups_tuned, float* rule_us, float* tuned_us)
{
    gb_set_last_error("");
    if (!bt || (bt->ncols && !preds)) return bfail(SCAN_EINVAL, "null pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    reps = std::max<uint32_t>(1, std::min<uint32_t>(reps, 100));
    BT_CUDA(cudaStreamSynchronize(st));
    unsigned long long* ctl = bt->d_results + 4ull * std::max<uint32_t>(1, bt->ncols);
    const size_t table_bytes = std::max<size_t>(1, bt->ncols) * sizeof(gb::BatchCol);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BT_CUDA(cudaEventCreate(&e0));
    BT_CUDA(cudaEventCreate(&e1));
    auto op_of = [](const scan_batch::Group& g) { return g.kernel == 1 ? gb::kOpBatchBR : gb::kOpBatchBF; };
    // Mean time of `reps` launches of group gi alone, with the shapes installed now.
    auto time_group = [&](size_t gi, float* us) -> scan_status {
        scan_status s = layout(bt);
        if (s != SCAN_OK) return s;
        fill_predicates(bt, preds);
        const auto& g = bt->groups[gi];
        BT_CUDA(cudaMemcpyAsync(bt->d_table, bt->h_table, table_bytes, cudaMemcpyHostToDevice, st));
        gb::BatchParams p{};
        p.cols = bt->d_table + g.first;
        p.chunk_col = bt->d_chunk_col + g.chunk_off;
        p.ncols = g.count;
        p.ntiles = g.ntiles;
        p.chunk = g.chunk;
        p.head = reinterpret_cast<unsigned int*>(ctl) + gi;
        p.results = bt->d_results;
        p.status = reinterpret_cast<unsigned int*>(ctl) + kMaxGroups;
        p.stages = static_cast<uint32_t>(g.shape.stages);
        p.slot_bytes = static_cast<uint32_t>(g.shape.tile_blocks) * 128u * static_cast<uint32_t>(g.b);
        float total = 0.f;
        for (uint32_t r = 0; r <= reps; ++r) {  // the first launch warms up
            BT_CUDA(cudaMemsetAsync(p.head, 0, sizeof(unsigned int), st));
            BT_CUDA(cudaEventRecord(e0, st));
            BT_CUDA(gb::launch_batch_kernel(g.kernel == 1, g.b, p, g.shape.warps, g.grid, st));
            BT_CUDA(cudaEventRecord(e1, st));
            BT_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r) total += ms;
        }
        *us = total * 1000.f / static_cast<float>(reps);
        return SCAN_OK;
    };
    // Median time of the whole graph (descriptor copy, reset, every group, result
    // copy) over 2 * reps + 1 replays, with the shapes installed now.
    auto time_graph = [&](float* us) -> scan_status {
        scan_status s = layout(bt);
        if (s != SCAN_OK) return s;
        if ((s = scan_batch_exec(bt, preds, stream, nullptr, nullptr)) != SCAN_OK) return s;  // records the graph
        std::vector<float> ts;
        for (uint32_t r = 0; r < 2 * reps + 1; ++r) {
            BT_CUDA(cudaEventRecord(e0, st));
            BT_CUDA(cudaGraphLaunch(bt->graph, st));
            BT_CUDA(cudaEventRecord(e1, st));
            BT_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ts.push_back(ms * 1000.f);
        }
        std::nth_element(ts.begin(), ts.begin() + ts.size() / 2, ts.end());
        *us = ts[ts.size() / 2];
        return SCAN_OK;
    };
    const std::vector<scan_batch::Group> groups = bt->groups;
    for (const auto& g : groups) gb_shape_install(g.b, op_of(g), nullptr, 0.f, 0.f);
    scan_status status = SCAN_OK;
    // 1. screen: each group alone, the rule and every candidate; keep the three fastest
    std::vector<std::vector<gb::LaunchShape>> finalists(groups.size());
    for (size_t gi = 0; gi < groups.size() && status == SCAN_OK; ++gi) {
        const auto& g = groups[gi];
        if (!g.ntiles) continue;
        float rule = 0.f;
        if ((status = time_group(gi, &rule)) != SCAN_OK) break;
        std::vector<std::pair<float, gb::LaunchShape>> timed;
        for (const gb::LaunchShape& c : gb_shape_candidates(g.b, op_of(g))) {
            gb_shape_install(g.b, op_of(g), &c, 0.f, 0.f);
            float us = 0.f;
            if ((status = time_group(gi, &us)) != SCAN_OK) break;
            if (us < rule) timed.push_back({us, c});
        }
        gb_shape_install(g.b, op_of(g), nullptr, 0.f, 0.f);
        std::sort(timed.begin(), timed.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
        for (size_t k = 0; k < timed.size() && k < 3; ++k) finalists[gi].push_back(timed[k].second);
    }
    // 2. the whole replay: the largest groups first, try each group's finalists
    //    with the others fixed and keep one only if the replay gets faster by
    //    more than 0.3% (the replay's run-to-run spread)
    float rule_graph = 0.f, best_graph = 0.f;
    uint32_t tuned = 0;
    if (status == SCAN_OK) status = time_graph(&rule_graph);
    best_graph = rule_graph;
    std::vector<size_t> order(groups.size());
    for (size_t gi = 0; gi < order.size(); ++gi) order[gi] = gi;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return groups[x].bytes > groups[y].bytes; });
    for (const size_t gi : order) {
        if (status != SCAN_OK) break;
        const auto& g = groups[gi];
        const gb::LaunchShape* keep = nullptr;
        for (const gb::LaunchShape& c : finalists[gi]) {
            gb_shape_install(g.b, op_of(g), &c, 0.f, 0.f);
            float us = 0.f;
            if ((status = time_graph(&us)) != SCAN_OK) break;
            if (us < best_graph * 0.997f) {
                best_graph = us;
                keep = &c;
            }
        }
        gb_shape_install(g.b, op_of(g), keep, keep ? best_graph : 0.f, keep ? rule_graph : 0.f);
        if (keep) ++tuned;
    }
    if (status == SCAN_OK && tuned) {  // the whole result must beat the rule, measured again
        float again = 0.f, rule_again = 0.f;
        status = time_graph(&again);
        std::vector<gb::LaunchShape> chosen(groups.size());
        for (size_t gi = 0; gi < groups.size(); ++gi) chosen[gi] = gb_shape_for(groups[gi].b, op_of(groups[gi]));
        for (const auto& g : groups) gb_shape_install(g.b, op_of(g), nullptr, 0.f, 0.f);
        if (status == SCAN_OK) status = time_graph(&rule_again);
        if (status == SCAN_OK && again < rule_again) {
            for (size_t gi = 0; gi < groups.size(); ++gi)
                if (chosen[gi].warps != gb_shape_for(groups[gi].b, op_of(groups[gi])).warps ||
                    chosen[gi].stages != gb_shape_for(groups[gi].b, op_of(groups[gi])).stages ||
                    chosen[gi].tile_blocks != gb_shape_for(groups[gi].b, op_of(groups[gi])).tile_blocks)
                    gb_shape_install(groups[gi].b, op_of(groups[gi]), &chosen[gi], again, rule_again);
            best_graph = again;
            rule_graph = rule_again;
        } else {
            tuned = 0;
            best_graph = rule_again;
            rule_graph = rule_again;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != SCAN_OK) {
        for (const auto& g : groups) gb_shape_install(g.b, op_of(g), nullptr, 0.f, 0.f);
        layout(bt);
        return status;
    }
    const scan_status ls = layout(bt);  // the installed shapes; the graph is recorded again
    if (ls != SCAN_OK) return ls;
    if (groups_tuned) *groups_tuned = tuned;
    if (rule_us) *rule_us = rule_graph;
    if (tuned_us) *tuned_us = best_graph;
    return SCAN_OK;
}

scan_status scan_batch_run(const scan_column* const* cols, const scan_pred* preds, uint32_t ncols,
                           const scan_strategy* strategies, void* stream, scan_result* host_out)
{
    scan_batch* bt = nullptr;
    scan_status s = scan_batch_create(const_cast<scan_column* const*>(cols), ncols, strategies, 0, stream, &bt);
    if (s != SCAN_OK) return s;
    s = scan_batch_exec(bt, preds, stream, host_out, nullptr);
    if (s == SCAN_OK) cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    scan_batch_destroy(bt);
    return s;
}

}  // extern "C"
