// Batched scan: thousands of columns in one CUDA-graph launch.
//
// The host cuts every column's 1024-value blocks into tiles (per width, the
// most blocks that fill a 6 KB slot in whole warp steps), groups the
// columns by width and numbers each group's tiles consecutively.  One
// persistent kernel serves a group: warps pop chunks of consecutive tile
// numbers from the group's atomic counter (a host-built table gives each
// chunk's first column), so a warp usually stays on one column for many
// tiles; each tile is fetched into the warp's slot ring by bulk TMA copies and
// decoded by the width-specialised code of the single-column scan, compiled
// for that group's width only (BFIX), which keeps the instruction cache warm.
// Columns marked for zone skipping test their blocks' (min, max) before the
// copy and fetch only the surviving runs.  A warp keeps running (count, sum)
// totals while the column does not change and adds them to the column's
// result with three atomics when it does.  The frame of reference is applied
// per flush (SUM_v = SUM_u + base*COUNT is linear).
#pragma once
#include "scan_kernels.cuh"

namespace gb {

enum : uint32_t { kColZone = 1u, kColEmpty = 2u };

struct BatchCol {
    const uint32_t* packed;  // lane-interleaved words
    const uint2* zonemap;    // per-block (min, max) of decoded values, or null
    uint64_t n;              // values
    uint32_t b, base;
    uint32_t tile_blocks;    // blocks per tile
    uint32_t tile_begin;     // first tile number of this column in the launch
    uint32_t lo, wm1;        // predicate in code space (width >= 1)
    uint64_t zlo, zhi;       // predicate on decoded values, for zone tests
    uint32_t flags;          // kColZone, kColEmpty
    uint32_t out;            // result slot
};

struct BatchParams {
    const BatchCol* cols;
    const uint32_t* chunk_col;     // first column of every pop-sized chunk, or null (binary search)
    uint32_t ncols;
    uint32_t ntiles;
    uint32_t chunk;                // tiles per atomic pop
    unsigned int* head;            // pop counter, zero before the launch
    unsigned long long* results;   // per output slot: count, sum, blocks, 0
    unsigned int* status;
    uint32_t stages;               // slots per warp (warps per CTA = blockDim.x / 32)
    uint32_t slot_bytes;           // bytes per slot: the group's largest tile
};

// Default batch shape: 8 warps, each with 2 slots of 6 KB, and at most
// kBatchPairSmem of slots per CTA so that two CTAs share an SM (the kernel
// is compiled for 128 registers a thread).  The graph runs the narrow widths
// (decode-bound) and the wide ones (bandwidth-bound) as two concurrent chains,
// so an SM holds one CTA of each kind and its ALUs and the HBM are busy at
// once.  On the 4096-column workload this took the replay from 0.97 to
// 0.86 ms; 3 or 4 stages of smaller slots, 4- or 6-warp CTAs and three CTAs
// per SM were all slower.  The shape is a run-time choice per width group;
// the autotuner may replace it.
constexpr int kBatchWarps = 8;
constexpr int kBatchStages = 2;
constexpr int kBatchSlot = 6 * 1024;
constexpr uint32_t kBatchSlotExtra = 8 + 16;   // a slot's barrier and metadata
// Slot bytes of a CTA that leave room for a second one on the SM (228 KB of
// shared memory per SM, 1 KB of it reserved per CTA).
constexpr uint32_t kBatchPairSmem = 112 * 1024;

__host__ __device__ constexpr uint32_t batch_smem_bytes(uint32_t warps, uint32_t stages, uint32_t slot_bytes)
{
    return warps * stages * (slot_bytes + kBatchSlotExtra);
}

// Default blocks per batch tile at width b: as many as fill a 6 KB slot, a
// multiple of the warp step (4 blocks for b <= 16, else 2), at most 64 (the
// keep mask).
__host__ __device__ constexpr uint32_t batch_tile_blocks(uint32_t b)
{
    const uint32_t step = b <= 16 ? 4u : 2u;
    const uint32_t tb = (static_cast<uint32_t>(kBatchSlot) / (128u * b)) / step * step;
    return tb < step ? step : (tb > 64u ? 64u : tb);
}

// Default warps per CTA at width b: 8, fewer where the one-step tiles of the
// widest columns (b = 14..16, 28..32: 7-8 KB) would overflow kBatchPairSmem.
__host__ __device__ constexpr int batch_default_warps(uint32_t b)
{
    const uint32_t per_warp = static_cast<uint32_t>(kBatchStages) * (batch_tile_blocks(b) * 128u * b + kBatchSlotExtra);
    const uint32_t w = kBatchPairSmem / per_warp;
    return w >= static_cast<uint32_t>(kBatchWarps) ? kBatchWarps : static_cast<int>(w);
}
static_assert(batch_default_warps(32) == 6 && batch_default_warps(1) == 8, "default batch CTAs fit two per SM");

struct SlotMeta {
    uint32_t col;   // column index
    uint32_t nk;    // blocks in the slot
    uint32_t tail;  // 1 if the last block in the slot is the column's partial tail
    uint32_t pad;
};

struct CountSum {
    uint64_t cnt, sum;
};

// The consumer's copy of its column's descriptor (what decoding a slot needs).
struct ConsCol {
    uint32_t lo, wm1;  // predicate in code space
    uint32_t tail;     // values in the column's last block (0: whole)
    uint32_t b;
};

template <int B, bool BRANCHY>
__device__ __forceinline__ CountSum batch_consume_body(const unsigned char* slot, const SlotMeta m,
                                                       const ConsCol& c, int lane)
{
    uint64_t cnt = 0, sum = 0;
    const Lanes L = make_lanes<B>(c.lo, c.wm1);
    const uint32_t nfull = m.tail ? m.nk - 1u : m.nk;
    scan_tile<B, BRANCHY>(slot, nfull, lane, L, c.lo, c.wm1, cnt, sum);
    if (m.tail) {
        const int q = lane % Geo<B>::kTpb;
        agg_block_masked<B>(block_rows<B>(slot + nfull * (128u * B), q), c.lo, c.wm1, cnt, sum,
                            lane < Geo<B>::kTpb, c.tail, q);
    }
    return CountSum{cnt, sum};
}

// Every column of the launch has width BFIX and its decode is inlined: one
// width's code per kernel keeps the instruction cache warm (a kernel holding
// all 32 unrolled decoders stalled on instruction fetch), so a batch runs one
// such kernel per width group.  Compiled for CTAs of up to 16 warps, which
// caps it at 128 registers a thread: two 8-warp CTAs then fit one SM.
template <bool BRANCHY, int BFIX>
__global__ void __launch_bounds__(512, 1) k_scan_batch(const BatchParams P)
{
    static_assert(BFIX >= 1 && BFIX <= 32, "batch kernels are width-specialised");
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t nwarps = blockDim.x >> 5;
    const int kStages = static_cast<int>(P.stages);
    const uint32_t kSlot = P.slot_bytes;
    unsigned char* slots = smem + static_cast<size_t>(warp) * kStages * kSlot;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + static_cast<size_t>(nwarps) * kStages * kSlot) +
                     warp * kStages;
    SlotMeta* meta =
        reinterpret_cast<SlotMeta*>(smem + static_cast<size_t>(nwarps) * kStages * (kSlot + 8)) + warp * kStages;
    if (lane == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncwarp();

    // producer cursor (warp-uniform) and the descriptor of its column, kept in
    // registers: a warp's tiles come in runs of one column, so the descriptor
    // and the next column's first tile are loaded once per run, not per tile
    uint32_t t_next = 0, t_end = 0, col = 0;
    bool exhausted = false;
    uint32_t phase = 0;  // bit s: parity of slot s's next completion
    uint32_t pc_id = ~0u, next_begin = 0;
    // zone skipping: blocks [zs_begin, zs_end) of column zs_col are known to hold no
    // survivor (found by a look-ahead read of zone entries), so tiles inside
    // that run are skipped without loading their entries again
    uint32_t zs_col = ~0u;
    uint64_t zs_begin = 0, zs_end = 0;
    const uint32_t* pc_packed = nullptr;
    const uint2* pc_zm = nullptr;
    uint64_t pc_n = 0, pc_zlo = 0, pc_zhi = 0;
    uint32_t pc_b = 0, pc_begin = 0, pc_tb = 0, pc_flags = 0;
    auto load_col = [&](uint32_t c) {
        const BatchCol* d = P.cols + c;
        pc_packed = d->packed;
        pc_zm = d->zonemap;
        pc_n = d->n;
        pc_b = static_cast<uint32_t>(BFIX);
        pc_begin = d->tile_begin;
        pc_tb = d->tile_blocks;
        pc_flags = d->flags;
        pc_zlo = d->zlo;
        pc_zhi = d->zhi;
        next_begin = c + 1 < P.ncols ? __ldg(&P.cols[c + 1].tile_begin) : 0xffffffffu;
        pc_id = c;
    };

    // Next tile number, or false when the launch has no more work.
    auto next_tile = [&](uint32_t& t) -> bool {
        if (t_next >= t_end) {
            if (exhausted) return false;
            unsigned int start = 0;
            if (lane == 0) start = atomicAdd(P.head, P.chunk);
            start = __shfl_sync(kFull, start, 0);
            if (start >= P.ntiles) {
                exhausted = true;
                return false;
            }
            t_next = start;
            t_end = min(start + P.chunk, P.ntiles);
            if (P.chunk_col) {  // host-built table: one load per pop
                col = __ldg(&P.chunk_col[start / P.chunk]);
            } else {            // binary search over tile_begin
                uint32_t lo = 0, hi = P.ncols - 1;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi + 1) >> 1;
                    if (__ldg(&P.cols[mid].tile_begin) <= start) lo = mid;
                    else hi = mid - 1;
                }
                col = lo;
            }
            if (col != pc_id) load_col(col);
        }
        t = t_next++;
        while (next_begin <= t) load_col(++col);  // the last column's next_begin is past every tile
        return true;
    };

    // Fetch the next tile into slot s; false when there is none.
    auto produce = [&](int s) -> bool {
        uint32_t t;
        if (!next_tile(t)) return false;
        const uint32_t bb = 128u * pc_b;
        const uint64_t nblocks = (pc_n + 1023u) >> 10;
        const uint64_t k0 = static_cast<uint64_t>(t - pc_begin) * pc_tb;
        const uint64_t left = nblocks - k0;
        const uint32_t nb = left < pc_tb ? static_cast<uint32_t>(left) : pc_tb;
        const bool has_tail = (pc_n & 1023u) && (k0 + nb == nblocks);
        uint64_t keep = (nb >= 64) ? ~0ull : ((1ull << nb) - 1ull);
        if (pc_flags & kColEmpty) {
            keep = 0;
        } else if (pc_flags & kColZone) {
            if (zs_col == pc_id && k0 >= zs_begin && k0 + nb <= zs_end) {
                keep = 0;  // inside a run already known to hold no survivor
            } else if (nb < 32u) {
                // one load covers this tile and the blocks after it, up to 32
                const uint64_t span = nblocks - k0 < 32u ? nblocks - k0 : 32u;
                bool k = false;
                if (lane < span) {
                    const uint2 z = __ldg(&pc_zm[k0 + lane]);
                    k = static_cast<uint64_t>(z.y) >= pc_zlo && static_cast<uint64_t>(z.x) < pc_zhi;
                }
                const uint32_t m32 = __ballot_sync(kFull, k);
                keep = m32 & ((1u << nb) - 1u);
                if (!keep) {  // no survivor up to the first one found (or the whole span)
                    zs_col = pc_id;
                    zs_begin = k0;
                    zs_end = k0 + (m32 ? static_cast<uint64_t>(__ffs(static_cast<int>(m32)) - 1) : span);
                }
            } else {
                uint64_t km = 0;
                for (uint32_t base_i = 0; base_i < nb; base_i += 32u) {
                    const uint32_t i = base_i + lane;
                    bool k = false;
                    if (i < nb) {
                        const uint2 z = __ldg(&pc_zm[k0 + i]);
                        k = static_cast<uint64_t>(z.y) >= pc_zlo && static_cast<uint64_t>(z.x) < pc_zhi;
                    }
                    km |= static_cast<uint64_t>(__ballot_sync(kFull, k)) << base_i;
                }
                keep = km;
            }
        }
        const uint32_t nk = static_cast<uint32_t>(__popcll(keep));
        if (lane == 0) {
            SlotMeta m;
            m.col = col;
            m.nk = nk;
            m.tail = (has_tail && ((keep >> (nb - 1)) & 1ull)) ? 1u : 0u;
            m.pad = 0;
            meta[s] = m;
            if (nk) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bars[s], nk * bb);
                unsigned char* dst = slots + s * kSlot;
                uint64_t rem = keep;
                uint32_t placed = 0;
                while (rem) {
                    const uint32_t first = static_cast<uint32_t>(__ffsll(static_cast<long long>(rem)) - 1);
                    const uint64_t from = rem >> first;
                    const uint32_t len = (~from == 0ull) ? (64u - first)
                                                          : static_cast<uint32_t>(__ffsll(static_cast<long long>(~from)) - 1);
                    bulk_g2s(dst + placed * bb, pc_packed + (k0 + first) * 32u * pc_b, len * bb, &bars[s]);
                    placed += len;
                    rem &= (len + first >= 64u) ? 0ull : (~0ull << (first + len));
                }
            }
        }
        __syncwarp();
        return true;
    };

    int produced = 0;
    for (int s = 0; s < kStages; ++s) {
        if (!produce(s)) break;
        ++produced;
    }

    uint64_t cnt = 0, sum = 0, blocks = 0;
    int cur = -1;
    ConsCol cc{0u, 0u, 0u, 0u};   // the consumer's column (loaded when it changes)
    uint32_t cur_out = 0, cur_base = 0;
    auto flush = [&]() {
        uint64_t c2 = cnt, s2 = sum;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            c2 += __shfl_xor_sync(kFull, c2, o);
            s2 += __shfl_xor_sync(kFull, s2, o);
        }
        if (lane == 0 && cur >= 0) {
            unsigned long long* r = P.results + 4u * cur_out;
            if (c2) atomicAdd(&r[0], static_cast<unsigned long long>(c2));
            if (c2) atomicAdd(&r[1], static_cast<unsigned long long>(s2 + static_cast<uint64_t>(cur_base) * c2));
            if (blocks) atomicAdd(&r[2], static_cast<unsigned long long>(blocks));
        }
        cnt = 0;
        sum = 0;
        blocks = 0;
    };

    bool failed = false;
    int it = 0, s = 0;  // s = it mod stages, kept without a division per tile
#pragma unroll 1
    for (; it < produced; ++it, s = (s + 1 == kStages) ? 0 : s + 1) {
        const SlotMeta m = meta[s];
        if (static_cast<int>(m.col) != cur) {
            flush();
            cur = static_cast<int>(m.col);
            const BatchCol* d = P.cols + m.col;
            cc.lo = d->lo;
            cc.wm1 = d->wm1;
            cc.tail = static_cast<uint32_t>(d->n & 1023u);
            cc.b = static_cast<uint32_t>(BFIX);
            cur_out = d->out;
            cur_base = d->base;
        }
        if (m.nk) {
            const bool ok = mbar_wait(&bars[s], (phase >> s) & 1u, kWaitLimitNs);
            if (!__all_sync(kFull, ok)) {
                failed = true;
                break;
            }
            phase ^= 1u << s;
            const CountSum r = batch_consume_body<BFIX, BRANCHY>(slots + s * kSlot, m, cc, lane);
            cnt += r.cnt;
            sum += r.sum;
            blocks += m.nk;
        }
        __syncwarp();
        if (produce(s)) ++produced;
    }
    if (failed) {
        if (lane == 0) atomicOr(P.status, kErrTimeout);
        // let this warp's copies in flight land before shared memory is released
        for (int j = it; j < produced && j < it + kStages; ++j) {
            const int s = j % kStages;
            if (meta[s].nk) {
                mbar_wait(&bars[s], (phase >> s) & 1u, kDrainLimitNs);
                phase ^= 1u << s;
            }
        }
    }
    flush();
}

}  // namespace gb

// One launcher per flavour and range of four widths (separate objects).
#define GB_DECLARE_BATCH(lo, hi)                                                                                \
    cudaError_t gb_launch_batch_bf_##lo##_##hi##_w(int b, const gb::BatchParams& p, int warps, int grid,        \
                                                   cudaStream_t st);                                             \
    cudaError_t gb_launch_batch_br_##lo##_##hi##_w(int b, const gb::BatchParams& p, int warps, int grid,        \
                                                   cudaStream_t st);
GB_DECLARE_BATCH(1, 4)
GB_DECLARE_BATCH(5, 8)
GB_DECLARE_BATCH(9, 12)
GB_DECLARE_BATCH(13, 16)
GB_DECLARE_BATCH(17, 20)
GB_DECLARE_BATCH(21, 24)
GB_DECLARE_BATCH(25, 28)
GB_DECLARE_BATCH(29, 32)
#undef GB_DECLARE_BATCH

// The batch kernel of one width group: flavour, width b, CTAs of `warps` warps.
inline cudaError_t gb_launch_batch(bool branchy, int b, const gb::BatchParams& p, int warps, int grid,
                                   cudaStream_t st)
{
#define GB_RANGE(k, lo, hi)                                                                                       \
    case k:                                                                                                      \
        return branchy ? gb_launch_batch_br_##lo##_##hi##_w(b, p, warps, grid, st)                                 \
                       : gb_launch_batch_bf_##lo##_##hi##_w(b, p, warps, grid, st);
    switch ((b - 1) / 4) {
        GB_RANGE(0, 1, 4)
        GB_RANGE(1, 5, 8)
        GB_RANGE(2, 9, 12)
        GB_RANGE(3, 13, 16)
        GB_RANGE(4, 17, 20)
        GB_RANGE(5, 21, 24)
        GB_RANGE(6, 25, 28)
        GB_RANGE(7, 29, 32)
    default: return cudaErrorInvalidValue;
    }
#undef GB_RANGE
}


