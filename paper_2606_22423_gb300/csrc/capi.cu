// C-ABI of the scan library: argument checking, column lifetime, the host and
// device encoders, predicate translation and kernel dispatch.  No compute
// happens on the host except the host encoder; every scan step runs in the
// kernels of scan_kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/gbscan.h"
#include "internal.h"
#include "scan_kernels.cuh"

namespace {

thread_local std::string g_err;

scan_status fail(scan_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
scan_status fail(scan_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

scan_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(e == cudaErrorMemoryAllocation ? SCAN_ENOMEM : SCAN_ECUDA, "%s: %s (%s)", what,
                cudaGetErrorName(e), cudaGetErrorString(e));
}

#define GB_CUDA(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

constexpr uint64_t kMaxValues = 1ull << 31;  // keeps SUM < 2^63
constexpr int kMaxGrid = 1024;                // partial slots in the workspace

inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

bool width_ok(uint32_t b, uint32_t base)
{
    return b >= 1 && b <= 32 && static_cast<uint64_t>(base) + ((1ull << b) - 1ull) <= 0xffffffffull;
}

uint64_t n_blocks(uint64_t n) { return (n + 1023u) >> 10; }

// Device workspace of one column, one allocation:
//   result[4] (32 B) | status (4 B) | done (4 B) | pad | qctl[8] (64 B) | partials[2*kMaxGrid]
struct Workspace {
    long long* result;
    unsigned int* status;
    unsigned int* done;
    unsigned long long* qctl;
    unsigned long long* partials;
    static constexpr size_t kBytes = 128 + 16 * kMaxGrid;
};

struct DeviceInfo {
    int sms = 0;
};

DeviceInfo device_info()
{
    DeviceInfo d;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    return d;
}

// Launches kernel `op` at width b with its current shape (tuned or the rule).
cudaError_t launch(int b, int op, const gb::ScanParams& p, int grid, cudaStream_t st)
{
    return gb_launch(b, op, p, gb_shape_for(b, op), grid, st);
}

}  // namespace

// Lets other units of the library set the message scan_last_error() returns.
void gb_set_last_error(const char* msg) { g_err = msg ? msg : ""; }

// SM count and cooperative-launch support of the current device, read once
// per device.
namespace {
constexpr int kMaxDevices = 64;
std::atomic<int> g_dev_sms[kMaxDevices];
std::atomic<int> g_dev_coop[kMaxDevices];
int current_device()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = 0;
    return dev;
}
}  // namespace

int gb_device_sms()
{
    const int dev = current_device();
    int n = g_dev_sms[dev].load(std::memory_order_relaxed);
    if (n <= 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
        g_dev_sms[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

bool gb_device_coop()
{
    const int dev = current_device();
    int v = g_dev_coop[dev].load(std::memory_order_relaxed);
    if (v == 0) {
        int c = 0;
        if (cudaDeviceGetAttribute(&c, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) c = 0;
        v = c ? 1 : -1;
        g_dev_coop[dev].store(v, std::memory_order_relaxed);
    }
    return v > 0;
}

namespace gb {
// ----------------------------------------------------- zone-map filtering
// Keeps block k iff max_k >= lo and min_k < hi (a block whose [min, max]
// misses [lo, hi) holds no match).  Each CTA compacts 2048 consecutive
// blocks in order in shared memory and reserves its output range with one
// atomic, so runs of consecutive candidates survive for merged copies.
// With kFlagAgg a block whose [min, max] lies inside [lo, hi) matches
// entirely: it is not kept, and its count and code sum (the metadata sum
// minus base * 1024) go to qctl[3], qctl[4] with one atomic pair per CTA.
__global__ void __launch_bounds__(kFilterThreads) k_zone_filter(const ScanParams p)
{
    __shared__ uint32_t list[kFilterPerCta];
    __shared__ uint32_t wcnt[kFilterThreads / 32];
    __shared__ uint32_t total;
    __shared__ unsigned long long out_base;
    __shared__ unsigned long long in_cnt, in_sum;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t full_blocks = p.n >> 10;
    const uint64_t first = static_cast<uint64_t>(blockIdx.x) * kFilterPerCta;
    const bool agg = (p.flags & kFlagAgg) != 0u;
    unsigned long long my_cnt = 0, my_sum = 0;
    if (threadIdx.x == 0) {
        total = 0u;
        in_cnt = 0ull;
        in_sum = 0ull;
    }
    __syncthreads();
    for (int pass = 0; pass < kFilterPerCta / kFilterThreads; ++pass) {
        const uint64_t k = first + pass * kFilterThreads + threadIdx.x;
        bool keep = false;
        if (k < full_blocks) {
            const uint2 z = p.zonemap[k];
            keep = static_cast<uint64_t>(z.y) >= p.zlo && static_cast<uint64_t>(z.x) < p.zhi;
            if (agg && keep && static_cast<uint64_t>(z.x) >= p.zlo && static_cast<uint64_t>(z.y) < p.zhi) {
                keep = false;
                my_cnt += 1024ull;
                my_sum += p.blocksum[k] - 1024ull * p.base;
            }
        }
        const uint32_t bal = __ballot_sync(kFull, keep);
        if (lane == 0) wcnt[warp] = __popc(bal);
        __syncthreads();
        uint32_t off = total;
        for (int w = 0; w < warp; ++w) off += wcnt[w];
        if (keep) list[off + __popc(bal & lanemask_lt())] = static_cast<uint32_t>(k);
        __syncthreads();
        if (threadIdx.x == 0)
            for (int w = 0; w < kFilterThreads / 32; ++w) total += wcnt[w];
        __syncthreads();
    }
    if (agg) {
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            my_cnt += __shfl_xor_sync(kFull, my_cnt, o);
            my_sum += __shfl_xor_sync(kFull, my_sum, o);
        }
        if (lane == 0 && my_cnt) {
            atomicAdd(&in_cnt, my_cnt);
            atomicAdd(&in_sum, my_sum);
        }
    }
    if (threadIdx.x == 0 && total) out_base = atomicAdd(&p.qctl[0], static_cast<unsigned long long>(total));
    __syncthreads();
    if (threadIdx.x == 0 && in_cnt) {
        atomicAdd(&p.qctl[3], in_cnt);
        atomicAdd(&p.qctl[4], in_sum);
    }
    for (uint32_t i = threadIdx.x; i < total; i += kFilterThreads) p.cand[out_base + i] = list[i];
}

}  // namespace gb

struct scan_column {
    uint64_t n = 0;
    uint32_t b = 0;
    uint32_t base = 0;
    int device = 0;
    uint32_t* packed = nullptr;
    bool owns_packed = false;
    uint2* zonemap = nullptr;
    unsigned long long* blocksum = nullptr;  // per-block sums, built with the zone map
    bool zonemap_valid = false;
    // SCAN_AUTO: the zone map's block minima and maxima, each sorted, on the
    // host (taken on the first SCAN_AUTO call after the zone map is built)
    std::vector<uint32_t> zmin_sorted, zmax_sorted;
    bool zsorted_valid = false;
    unsigned int* cand = nullptr;
    void* ws_raw = nullptr;
    Workspace ws{};
    scan_result* host_result = nullptr;  // pinned staging, 48 bytes (result + status)
    int layout = SCAN_LAYOUT_LANES;         // order of the codes inside each block
    uint32_t* conj_mask = nullptr;          // conjunctive scans: selection vector (grown on demand)
    uint64_t conj_words = 0;
    unsigned long long* sel_agg = nullptr;  // materializing select: tagged CTA totals
    uint64_t sel_words = 0;
    uint32_t sel_epoch = 0;
};

// Read-only view of a column for the batch planner (not part of the C ABI).
bool gb_column_view(const scan_column* c, const uint32_t** packed, uint64_t* n, uint32_t* b,
                    uint32_t* base, const uint2** zonemap)
{
    if (!c || c->layout != SCAN_LAYOUT_LANES) return false;
    *packed = c->packed;
    *n = c->n;
    *b = c->b;
    *base = c->base;
    *zonemap = c->zonemap_valid ? c->zonemap : nullptr;
    return true;
}

// Scan parameters of a column (its data and workspace), for other units of the library.
gb::ScanParams gb_column_params(const scan_column* c);

cudaError_t gb_column_conj_mask(scan_column* c, uint64_t words, uint32_t** out)
{
    if (words > c->conj_words) {
        if (c->conj_mask) cudaFree(c->conj_mask);  // synchronises: no earlier scan still uses it
        c->conj_mask = nullptr;
        c->conj_words = 0;
        const cudaError_t e = cudaMalloc(&c->conj_mask, words * sizeof(uint32_t));
        if (e != cudaSuccess) return e;
        c->conj_words = words;
    }
    *out = c->conj_mask;
    return cudaSuccess;
}

cudaError_t gb_column_select_ws(scan_column* c, uint64_t words, cudaStream_t st, GbSelectWs* out)
{
    cudaError_t e = cudaSuccess;
    if (words > c->sel_words) {
        if (c->sel_agg) cudaFree(c->sel_agg);
        c->sel_agg = nullptr;
        c->sel_words = 0;
        if ((e = cudaMalloc(&c->sel_agg, words * sizeof(unsigned long long))) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(c->sel_agg, 0, words * sizeof(unsigned long long), st)) != cudaSuccess) return e;
        c->sel_words = words;
        c->sel_epoch = 0;
    }
    if (++c->sel_epoch == 0) {  // the tag wrapped: words from 2^32 launches ago would match again
        if ((e = cudaMemsetAsync(c->sel_agg, 0, c->sel_words * sizeof(unsigned long long), st)) != cudaSuccess)
            return e;
        c->sel_epoch = 1;
    }
    out->agg = c->sel_agg;
    out->epoch = c->sel_epoch;
    out->status = c->ws.status;
    out->result = c->ws.result;
    out->host_result = c->host_result;
    return cudaSuccess;
}

// ---------------------------------------------------------------- encoders
namespace {

__global__ void k_encode(const uint32_t* __restrict__ v, uint64_t n, uint32_t b, uint32_t base,
                         uint32_t* __restrict__ out, uint64_t words, unsigned int* status)
{
    // one thread per output word (block k, lane word w, lane l); the 32 lanes
    // of a warp read 32 consecutive values per row and write 32 consecutive words
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    const uint64_t span = 32ull * b;
    const uint64_t mask = (b == 32) ? 0xffffffffull : ((1ull << b) - 1ull);
    for (uint64_t t = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < words; t += stride) {
        const uint64_t k = t / span;
        const uint32_t rem = static_cast<uint32_t>(t - k * span);
        const uint32_t w = rem >> 5, l = rem & 31u;
        const uint32_t bit0 = 32u * w;                     // first stream bit of this word
        const uint32_t r_first = bit0 / b;
        const uint32_t r_last = min(31u, (bit0 + 31u) / b);
        uint64_t acc = 0;
        bool bad = false;
        for (uint32_t r = r_first; r <= r_last; ++r) {
            const uint64_t j = (k << 10) + 32ull * r + l;
            uint64_t u = 0;
            if (j < n) {
                const uint32_t x = v[j];
                u = static_cast<uint64_t>(x) - base;
                // the thread holding the value's first bit checks its range
                if (r * b >= bit0 && (x < base || (u & ~mask))) bad = true;
                u &= mask;
            }
            const int64_t sh = static_cast<int64_t>(r) * b - bit0;
            acc |= sh >= 0 ? (u << sh) : (u >> (-sh));
        }
        out[t] = static_cast<uint32_t>(acc);
        if (bad) atomicOr(status, gb::kErrRange);
    }
}

// Row-major stream (§3 strategy i; at b = 8/16/32 also the byte-aligned
// array): one thread per output word; word t holds stream bits
// [32t, 32t + 32), i.e. parts of values floor(32t/b) .. floor((32t+31)/b).
__global__ void k_encode_rowmajor(const uint32_t* __restrict__ v, uint64_t n, uint32_t b, uint32_t base,
                                  uint32_t* __restrict__ out, uint64_t words, unsigned int* status)
{
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    const uint64_t mask = (b == 32) ? 0xffffffffull : ((1ull << b) - 1ull);
    for (uint64_t t = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < words; t += stride) {
        const uint64_t bit0 = 32ull * t;
        const uint64_t first = bit0 / b, last = (bit0 + 31u) / b;
        uint64_t acc = 0;
        bool bad = false;
        for (uint64_t j = first; j <= last; ++j) {
            uint64_t u = 0;
            if (j < n) {
                const uint32_t x = v[j];
                u = static_cast<uint64_t>(x) - base;
                // the thread holding the value's first bit checks its range
                if (j * b >= bit0 && (x < base || (u & ~mask))) bad = true;
                u &= mask;
            }
            const int64_t sh = static_cast<int64_t>(j * b) - static_cast<int64_t>(bit0);
            acc |= sh >= 0 ? (u << sh) : (u >> (-sh));
        }
        out[t] = static_cast<uint32_t>(acc);
        if (bad) atomicOr(status, gb::kErrRange);
    }
}

// Waits, with the library's bounded wait, on a transaction barrier that
// nothing ever completes; the wait gives up after limit_ns and records the
// timeout in the status word exactly as a lost copy would.
__global__ void k_selftest_wait(unsigned long long limit_ns, unsigned int* status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        gb::mbar_init(&bar, 1);
        gb::fence_mbar_init();
    }
    __syncwarp();
    const bool ok = gb::mbar_wait(&bar, 0u, limit_ns);
    if (!__all_sync(gb::kFull, ok) && threadIdx.x == 0) atomicOr(status, gb::kErrTimeout);
}

// STREAM triad a = b + s*c over float4 vectors (streaming loads and stores,
// four vectors per thread in flight).
__global__ void k_triad_probe(float4* __restrict__ a, const float4* __restrict__ b, const float4* __restrict__ c,
                              float s, uint64_t n4)
{
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n4; i += 4 * stride) {
        float4 x[4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            x[u] = __ldcs(b + i + u * stride);
            y[u] = __ldcs(c + i + u * stride);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            __stcs(a + i + u * stride, make_float4(fmaf(s, y[u].x, x[u].x), fmaf(s, y[u].y, x[u].y),
                                                   fmaf(s, y[u].z, x[u].z), fmaf(s, y[u].w, x[u].w)));
    }
    for (; i < n4; i += stride) {
        const float4 x = __ldcs(b + i), y = __ldcs(c + i);
        __stcs(a + i, make_float4(fmaf(s, y.x, x.x), fmaf(s, y.y, x.y), fmaf(s, y.z, x.z), fmaf(s, y.w, x.w)));
    }
}

__global__ void k_read_probe(const uint4* __restrict__ p, uint64_t n16, unsigned long long* out)
{
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    uint32_t x = 0;
    for (; i + 7 * stride < n16; i += 8 * stride) {
        uint4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcs(p + i + u * stride);
#pragma unroll
        for (int u = 0; u < 8; ++u) x += v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    }
    for (; i < n16; i += stride) {
        const uint4 v = __ldcs(p + i);
        x += v.x ^ v.y ^ v.z ^ v.w;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(gb::kFull, x, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, static_cast<unsigned long long>(x));
}

void encode_blocks(const uint32_t* v, uint64_t n, uint32_t b, uint32_t base, uint32_t* out,
                   uint64_t k0, uint64_t k1)
{
    // lane by lane: append each row's code to a 64-bit bit buffer, spill whole words
    for (uint64_t k = k0; k < k1; ++k) {
        uint32_t* blk = out + k * 32ull * b;
        for (uint32_t l = 0; l < 32; ++l) {
            uint64_t bits = 0;
            uint32_t fill = 0, w = 0;
            for (uint32_t r = 0; r < 32; ++r) {
                const uint64_t j = (k << 10) + 32ull * r + l;
                const uint64_t u = j < n ? static_cast<uint64_t>(v[j] - base) : 0ull;
                bits |= u << fill;
                fill += b;
                if (fill >= 32) {
                    blk[32u * w + l] = static_cast<uint32_t>(bits);
                    ++w;
                    bits >>= 32;
                    fill -= 32;
                }
            }
        }
    }
}

void encode_rowmajor_blocks(const uint32_t* v, uint64_t n, uint32_t b, uint32_t base, uint32_t* out,
                            uint64_t k0, uint64_t k1)
{
    // value by value: append each code to a 64-bit bit buffer, spill whole words
    for (uint64_t k = k0; k < k1; ++k) {
        uint32_t* blk = out + k * 32ull * b;
        uint64_t bits = 0;
        uint32_t fill = 0, w = 0;
        for (uint32_t j = 0; j < 1024; ++j) {
            const uint64_t i = (k << 10) + j;
            const uint64_t u = i < n ? static_cast<uint64_t>(v[i] - base) : 0ull;
            bits |= u << fill;
            fill += b;
            if (fill >= 32) {
                blk[w++] = static_cast<uint32_t>(bits);
                bits >>= 32;
                fill -= 32;
            }
        }
    }
}

bool layout_ok(uint32_t b, scan_layout layout)
{
    if (layout == SCAN_LAYOUT_LANES || layout == SCAN_LAYOUT_ROWMAJOR) return true;
    return layout == SCAN_LAYOUT_BYTES && (b == 8 || b == 16 || b == 32);
}

scan_status check_values_host(const uint32_t* v, uint64_t n, uint32_t b, uint32_t base)
{
    const uint64_t lim = 1ull << b;
    for (uint64_t i = 0; i < n; ++i) {
        if (v[i] < base || static_cast<uint64_t>(v[i] - base) >= lim)
            return fail(SCAN_EINVAL, "value %u at index %llu is outside [%u, %llu)", v[i],
                        static_cast<unsigned long long>(i), base,
                        static_cast<unsigned long long>(base + lim));
    }
    return SCAN_OK;
}

scan_status new_column(uint64_t n, uint32_t b, uint32_t base, scan_column** out)
{
    auto* c = new (std::nothrow) scan_column();
    if (!c) return fail(SCAN_ENOMEM, "host allocation failed");
    c->n = n;
    c->b = b;
    c->base = base;
    cudaGetDevice(&c->device);
    cudaError_t e = cudaMalloc(&c->ws_raw, Workspace::kBytes);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaMalloc(workspace)");
    }
    e = cudaMemset(c->ws_raw, 0, Workspace::kBytes);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&c->host_result), 64);
    if (e != cudaSuccess) {
        cudaFree(c->ws_raw);
        delete c;
        return cuda_fail(e, "workspace setup");
    }
    auto* base_ptr = static_cast<unsigned char*>(c->ws_raw);
    c->ws.result = reinterpret_cast<long long*>(base_ptr);
    c->ws.status = reinterpret_cast<unsigned int*>(base_ptr + 32);
    c->ws.done = reinterpret_cast<unsigned int*>(base_ptr + 36);
    c->ws.qctl = reinterpret_cast<unsigned long long*>(base_ptr + 64);
    c->ws.partials = reinterpret_cast<unsigned long long*>(base_ptr + 128);
    *out = c;
    return SCAN_OK;
}

gb::ScanParams base_params(const scan_column* c)
{
    gb::ScanParams p{};
    p.packed = c->packed;
    p.n = c->n;
    p.base = c->base;
    p.zonemap = c->zonemap;
    p.blocksum = c->blocksum;
    p.partials = c->ws.partials;
    p.done = c->ws.done;
    p.status = c->ws.status;
    p.cand = c->cand;
    p.qctl = c->ws.qctl;
    p.result = c->ws.result;
    return p;
}

}  // namespace

gb::ScanParams gb_column_params(const scan_column* c) { return base_params(c); }

namespace {

int persistent_grid() { return std::max(1, std::min(gb_device_sms(), kMaxGrid)); }

// Translate [lo, hi) on decoded values into code space; false if empty.
bool translate(const scan_column* c, scan_pred pr, gb::ScanParams& p)
{
    const int64_t lo_v = static_cast<int64_t>(c->base);
    const int64_t hi_v = static_cast<int64_t>(c->base) + (1ll << c->b);  // exclusive domain end
    const int64_t lo = std::max(pr.lo, lo_v);
    const int64_t hi = std::min(pr.hi, hi_v);
    if (lo >= hi) return false;
    p.lo = static_cast<uint32_t>(lo - lo_v);
    p.wm1 = static_cast<uint32_t>(hi - lo - 1);
    p.zlo = static_cast<uint64_t>(lo);
    p.zhi = static_cast<uint64_t>(hi);
    return true;
}

// SCAN_AUTO reads every block once the zone test would keep at least this
// many of the column's blocks: the law's break-even, where the 8 bytes of zone
// map and candidate id per block cost as much as the 128*b data bytes the
// skipped blocks save, f = (128b - 8) / (128b + 8), capped at 0.9.
uint64_t auto_dense_min(uint32_t b, uint64_t nblocks)
{
    const double db = static_cast<double>(b);
    const double f = std::min(0.9, (128.0 * db - 8.0) / (128.0 * db + 8.0));
    return static_cast<uint64_t>(std::ceil(f * static_cast<double>(nblocks)));
}

// Exact number of blocks the zone test keeps for [zlo, zhi): a block is
// skipped iff max < zlo or min >= zhi, two disjoint cases since min <= max,
// so survivors = blocks - #(max < zlo) - #(min >= zhi): two binary searches
// over sorted copies of the bounds (copied and sorted on first use).
scan_status auto_survivors(scan_column* c, uint64_t zlo, uint64_t zhi, cudaStream_t st, uint64_t* out)
{
    const uint64_t nb = n_blocks(c->n);
    if (!c->zsorted_valid) {
        std::vector<uint2> z(nb);
        GB_CUDA(cudaMemcpyAsync(z.data(), c->zonemap, nb * sizeof(uint2), cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaStreamSynchronize(st));
        c->zmin_sorted.resize(nb);
        c->zmax_sorted.resize(nb);
        for (uint64_t i = 0; i < nb; ++i) {
            c->zmin_sorted[i] = z[i].x;
            c->zmax_sorted[i] = z[i].y;
        }
        std::sort(c->zmin_sorted.begin(), c->zmin_sorted.end());
        std::sort(c->zmax_sorted.begin(), c->zmax_sorted.end());
        c->zsorted_valid = true;
    }
    // #(max < zlo): maxima below zlo; #(min >= zhi): minima at or above zhi
    const uint64_t below = zlo > 0xffffffffull
                               ? nb
                               : static_cast<uint64_t>(std::lower_bound(c->zmax_sorted.begin(), c->zmax_sorted.end(),
                                                                        static_cast<uint32_t>(zlo)) -
                                                       c->zmax_sorted.begin());
    const uint64_t above = zhi > 0xffffffffull
                               ? 0
                               : static_cast<uint64_t>(c->zmin_sorted.end() -
                                                       std::lower_bound(c->zmin_sorted.begin(), c->zmin_sorted.end(),
                                                                        static_cast<uint32_t>(zhi)));
    *out = nb - below - above;
    return SCAN_OK;
}

scan_status enqueue_scan(scan_column* c, scan_pred pred, scan_strategy strategy, cudaStream_t st,
                         long long* dev_result, bool* empty)
{
    gb::ScanParams p = base_params(c);
    *empty = false;
    if (c->n == 0 || !translate(c, pred, p)) {
        *empty = true;
        return SCAN_OK;
    }
    if (dev_result) p.result = dev_result;
    if (strategy == SCAN_AUTO) {
        strategy = SCAN_BRANCHFREE;
        if (c->zonemap_valid && c->layout == SCAN_LAYOUT_LANES) {
            uint64_t survivors = 0;
            const scan_status s = auto_survivors(c, p.zlo, p.zhi, st, &survivors);
            if (s != SCAN_OK) return s;
            if (survivors < auto_dense_min(c->b, n_blocks(c->n))) strategy = SCAN_ZONE_SKIP_BF;
        }
    }
    const int grid = persistent_grid();
    int op;
    switch (strategy) {
    case SCAN_BRANCHFREE: op = gb::kOpFullBF; break;
    case SCAN_BRANCHY: op = gb::kOpFullBR; break;
    case SCAN_ZONE_SKIP_BF: op = gb::kOpQueueBF; break;
    case SCAN_ZONE_SKIP_BR: op = gb::kOpQueueBR; break;
    case SCAN_ZONE_AGG_BF:
        op = gb::kOpQueueBF;
        p.flags |= gb::kFlagAgg;
        break;
    case SCAN_ZONE_AGG_BR:
        op = gb::kOpQueueBR;
        p.flags |= gb::kFlagAgg;
        break;
    default: return fail(SCAN_EINVAL, "unknown strategy %d", static_cast<int>(strategy));
    }
    // at b = 32 every layout is the plain array, which the lane kernels read
    if (c->layout != SCAN_LAYOUT_LANES && c->b != 32) {
        const bool branchy = op == gb::kOpFullBR;
        if (op != gb::kOpFullBF && op != gb::kOpFullBR)
            return fail(SCAN_EINVAL, "zone-skip strategies need a lane-interleaved column");
        if (c->layout == SCAN_LAYOUT_ROWMAJOR) op = branchy ? gb::kOpRowBR : gb::kOpRowBF;
        else op = branchy ? gb::kOpBytesBR : gb::kOpBytesBF;
    } else if (c->layout != SCAN_LAYOUT_LANES && op != gb::kOpFullBF && op != gb::kOpFullBR) {
        return fail(SCAN_EINVAL, "zone-skip strategies need a lane-interleaved column");
    }
    if (op == gb::kOpQueueBF || op == gb::kOpQueueBR) {
        if (!c->zonemap_valid) return fail(SCAN_EINVAL, "zone-skip strategy needs scan_zonemap_build first");
        const uint64_t full = c->n >> 10;
        if (full) {
            const unsigned fgrid = static_cast<unsigned>((full + gb::kFilterPerCta - 1) / gb::kFilterPerCta);
            gb::k_zone_filter<<<fgrid, gb::kFilterThreads, 0, st>>>(p);
            GB_CUDA(cudaGetLastError());
        }
    }
    const cudaError_t e = launch(static_cast<int>(c->b), op, p, grid, st);
    if (e != cudaSuccess) return cuda_fail(e, "scan kernel launch");
    return SCAN_OK;
}

}  // namespace

scan_status gb_enqueue_scan(scan_column* c, scan_pred pred, scan_strategy strategy, cudaStream_t st,
                            long long* dev_result, bool* empty)
{
    return enqueue_scan(c, pred, strategy, st, dev_result, empty);
}

// =================================================================== ABI
extern "C" {

const char* scan_last_error(void) { return g_err.c_str(); }

const char* scan_status_string(scan_status s)
{
    switch (s) {
    case SCAN_OK: return "SCAN_OK";
    case SCAN_EINVAL: return "SCAN_EINVAL";
    case SCAN_ENOMEM: return "SCAN_ENOMEM";
    case SCAN_ECUDA: return "SCAN_ECUDA";
    case SCAN_ETIMEOUT: return "SCAN_ETIMEOUT";
    case SCAN_EBUSY: return "SCAN_EBUSY";
    case SCAN_ENOTSUP: return "SCAN_ENOTSUP";
    }
    return "SCAN_UNKNOWN";
}

uint64_t scan_packed_words(uint64_t n, uint32_t b)
{
    if (b < 1 || b > 32) return 0;
    return n_blocks(n) * 32ull * b;
}

scan_status scan_encode_host(const uint32_t* host_values, uint64_t n, uint32_t b, uint32_t base,
                             uint32_t* host_out)
{
    return scan_encode_host_layout(host_values, n, b, base, SCAN_LAYOUT_LANES, host_out);
}

scan_status scan_encode_host_layout(const uint32_t* host_values, uint64_t n, uint32_t b, uint32_t base,
                                    scan_layout layout, uint32_t* host_out)
{
    g_err.clear();
    if (!width_ok(b, base)) return fail(SCAN_EINVAL, "bad width b=%u / base=%u", b, base);
    if (!layout_ok(b, layout)) return fail(SCAN_EINVAL, "layout %d does not take b=%u", static_cast<int>(layout), b);
    if (n > kMaxValues) return fail(SCAN_EINVAL, "n=%llu exceeds 2^31", static_cast<unsigned long long>(n));
    if (n == 0) return SCAN_OK;
    if (!host_values || !host_out) return fail(SCAN_EINVAL, "null pointer");
    scan_status s = check_values_host(host_values, n, b, base);
    if (s != SCAN_OK) return s;
    const uint64_t nb = n_blocks(n);
    // the lane layout at b = 32 and the byte layouts are the row-major stream
    auto* enc = layout == SCAN_LAYOUT_LANES ? encode_blocks : encode_rowmajor_blocks;
    unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const unsigned threads = static_cast<unsigned>(std::min<uint64_t>(std::min(hw, 64u), (nb + 63) / 64));
    if (threads <= 1) {
        enc(host_values, n, b, base, host_out, 0, nb);
        return SCAN_OK;
    }
    std::vector<std::thread> pool;
    const uint64_t per = (nb + threads - 1) / threads;
    for (unsigned t = 0; t < threads; ++t) {
        const uint64_t k0 = std::min(nb, t * per), k1 = std::min(nb, k0 + per);
        pool.emplace_back(enc, host_values, n, b, base, host_out, k0, k1);
    }
    for (auto& th : pool) th.join();
    return SCAN_OK;
}

scan_status scan_encode_device(const uint32_t* dev_values, uint64_t n, uint32_t b, uint32_t base,
                               uint32_t* dev_out, void* stream)
{
    return scan_encode_device_layout(dev_values, n, b, base, SCAN_LAYOUT_LANES, dev_out, stream);
}

scan_status scan_encode_device_layout(const uint32_t* dev_values, uint64_t n, uint32_t b, uint32_t base,
                                      scan_layout layout, uint32_t* dev_out, void* stream)
{
    g_err.clear();
    if (!width_ok(b, base)) return fail(SCAN_EINVAL, "bad width b=%u / base=%u", b, base);
    if (!layout_ok(b, layout)) return fail(SCAN_EINVAL, "layout %d does not take b=%u", static_cast<int>(layout), b);
    if (n > kMaxValues) return fail(SCAN_EINVAL, "n exceeds 2^31");
    if (n == 0) return SCAN_OK;
    if (!dev_values || !dev_out) return fail(SCAN_EINVAL, "null pointer");
    if (reinterpret_cast<uintptr_t>(dev_out) & 15u) return fail(SCAN_EINVAL, "dev_out must be 16-byte aligned");
    cudaStream_t st = as_stream(stream);
    unsigned int* flag = nullptr;
    GB_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&flag), sizeof(unsigned int), st));
    GB_CUDA(cudaMemsetAsync(flag, 0, sizeof(unsigned int), st));
    const uint64_t words = scan_packed_words(n, b);
    const int grid = persistent_grid() * 8;
    if (layout == SCAN_LAYOUT_LANES)
        k_encode<<<grid, 256, 0, st>>>(dev_values, n, b, base, dev_out, words, flag);
    else
        k_encode_rowmajor<<<grid, 256, 0, st>>>(dev_values, n, b, base, dev_out, words, flag);
    GB_CUDA(cudaGetLastError());
    unsigned int hflag = 0;
    GB_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof hflag, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaFreeAsync(flag, st));
    GB_CUDA(cudaStreamSynchronize(st));
    if (hflag & gb::kErrRange) return fail(SCAN_EINVAL, "a value lies outside [base, base + 2^b)");
    return SCAN_OK;
}

scan_status scan_column_create(const uint32_t* host_values, uint64_t n, uint32_t b, uint32_t base,
                               void* stream, scan_column** out)
{
    return scan_column_create_layout(host_values, n, b, base, SCAN_LAYOUT_LANES, stream, out);
}

scan_status scan_column_create_layout(const uint32_t* host_values, uint64_t n, uint32_t b, uint32_t base,
                                      scan_layout layout, void* stream, scan_column** out)
{
    g_err.clear();
    if (!out) return fail(SCAN_EINVAL, "out is NULL");
    *out = nullptr;
    if (!width_ok(b, base)) return fail(SCAN_EINVAL, "bad width b=%u / base=%u", b, base);
    if (!layout_ok(b, layout)) return fail(SCAN_EINVAL, "layout %d does not take b=%u", static_cast<int>(layout), b);
    if (n > kMaxValues) return fail(SCAN_EINVAL, "n exceeds 2^31");
    if (n && !host_values) return fail(SCAN_EINVAL, "host_values is NULL");
    const uint64_t words = scan_packed_words(n, b);
    std::vector<uint32_t> packed;
    try {
        packed.resize(words);
    } catch (...) {
        return fail(SCAN_ENOMEM, "host staging allocation failed");
    }
    scan_status s = scan_encode_host_layout(host_values, n, b, base, layout, packed.data());
    if (s != SCAN_OK) return s;
    scan_column* c = nullptr;
    s = new_column(n, b, base, &c);
    if (s != SCAN_OK) return s;
    c->layout = layout;
    cudaError_t e = cudaMalloc(&c->packed, std::max<uint64_t>(words, 4) * 4);
    if (e != cudaSuccess) {
        scan_column_destroy(c);
        return cuda_fail(e, "cudaMalloc(packed)");
    }
    c->owns_packed = true;
    if (words) {
        e = cudaMemcpyAsync(c->packed, packed.data(), words * 4, cudaMemcpyHostToDevice, as_stream(stream));
        if (e == cudaSuccess) e = cudaStreamSynchronize(as_stream(stream));
        if (e != cudaSuccess) {
            scan_column_destroy(c);
            return cuda_fail(e, "upload");
        }
    }
    *out = c;
    return SCAN_OK;
}

scan_status scan_column_create_device(const uint32_t* dev_values, uint64_t n, uint32_t b,
                                      uint32_t base, void* stream, scan_column** out)
{
    return scan_column_create_device_layout(dev_values, n, b, base, SCAN_LAYOUT_LANES, stream, out);
}

scan_status scan_column_create_device_layout(const uint32_t* dev_values, uint64_t n, uint32_t b, uint32_t base,
                                             scan_layout layout, void* stream, scan_column** out)
{
    g_err.clear();
    if (!out) return fail(SCAN_EINVAL, "out is NULL");
    *out = nullptr;
    if (!width_ok(b, base)) return fail(SCAN_EINVAL, "bad width b=%u / base=%u", b, base);
    if (!layout_ok(b, layout)) return fail(SCAN_EINVAL, "layout %d does not take b=%u", static_cast<int>(layout), b);
    if (n > kMaxValues) return fail(SCAN_EINVAL, "n exceeds 2^31");
    if (n && !dev_values) return fail(SCAN_EINVAL, "dev_values is NULL");
    scan_column* c = nullptr;
    scan_status s = new_column(n, b, base, &c);
    if (s != SCAN_OK) return s;
    const uint64_t words = scan_packed_words(n, b);
    cudaError_t e = cudaMalloc(&c->packed, std::max<uint64_t>(words, 4) * 4);
    if (e != cudaSuccess) {
        scan_column_destroy(c);
        return cuda_fail(e, "cudaMalloc(packed)");
    }
    c->owns_packed = true;
    c->layout = layout;
    s = scan_encode_device_layout(dev_values, n, b, base, layout, c->packed, stream);
    if (s != SCAN_OK) {
        std::string msg = g_err;
        scan_column_destroy(c);
        g_err = msg;
        return s;
    }
    *out = c;
    return SCAN_OK;
}

scan_status scan_column_create_packed(const uint32_t* dev_packed, uint64_t n, uint32_t b,
                                      uint32_t base, void* stream, scan_column** out)
{
    return scan_column_create_packed_layout(dev_packed, n, b, base, SCAN_LAYOUT_LANES, stream, out);
}

scan_status scan_column_create_packed_layout(const uint32_t* dev_packed, uint64_t n, uint32_t b, uint32_t base,
                                             scan_layout layout, void* stream, scan_column** out)
{
    (void)stream;
    g_err.clear();
    if (!out) return fail(SCAN_EINVAL, "out is NULL");
    *out = nullptr;
    if (!width_ok(b, base)) return fail(SCAN_EINVAL, "bad width b=%u / base=%u", b, base);
    if (!layout_ok(b, layout)) return fail(SCAN_EINVAL, "layout %d does not take b=%u", static_cast<int>(layout), b);
    if (n > kMaxValues) return fail(SCAN_EINVAL, "n exceeds 2^31");
    if (n && !dev_packed) return fail(SCAN_EINVAL, "dev_packed is NULL");
    if (reinterpret_cast<uintptr_t>(dev_packed) & 15u)
        return fail(SCAN_EINVAL, "dev_packed must be 16-byte aligned for bulk copies");
    scan_column* c = nullptr;
    scan_status s = new_column(n, b, base, &c);
    if (s != SCAN_OK) return s;
    c->packed = const_cast<uint32_t*>(dev_packed);
    c->owns_packed = false;
    c->layout = layout;
    *out = c;
    return SCAN_OK;
}

scan_status scan_column_blocksums(const scan_column* col, const uint64_t** dev_blocksums)
{
    g_err.clear();
    if (!col || !dev_blocksums) return fail(SCAN_EINVAL, "null pointer");
    *dev_blocksums = col->zonemap_valid ? reinterpret_cast<const uint64_t*>(col->blocksum) : nullptr;
    return SCAN_OK;
}

scan_status scan_column_get_layout(const scan_column* col, scan_layout* layout)
{
    g_err.clear();
    if (!col || !layout) return fail(SCAN_EINVAL, "null pointer");
    *layout = static_cast<scan_layout>(col->layout);
    return SCAN_OK;
}

scan_status scan_column_upload_packed(scan_column* col, const uint32_t* host_packed, void* stream)
{
    g_err.clear();
    if (!col || (!host_packed && col->n)) return fail(SCAN_EINVAL, "null pointer");
    const uint64_t words = scan_packed_words(col->n, col->b);
    if (words)
        GB_CUDA(cudaMemcpyAsync(col->packed, host_packed, words * 4, cudaMemcpyHostToDevice,
                                as_stream(stream)));
    col->zonemap_valid = false;
    col->zsorted_valid = false;
    return SCAN_OK;
}

scan_status scan_column_destroy(scan_column* col)
{
    g_err.clear();
    if (!col) return SCAN_OK;
    cudaDeviceSynchronize();
    if (col->owns_packed && col->packed) cudaFree(col->packed);
    if (col->zonemap) cudaFree(col->zonemap);
    if (col->blocksum) cudaFree(col->blocksum);
    if (col->cand) cudaFree(col->cand);
    if (col->ws_raw) cudaFree(col->ws_raw);
    if (col->host_result) cudaFreeHost(col->host_result);
    if (col->sel_agg) cudaFree(col->sel_agg);
    if (col->conj_mask) cudaFree(col->conj_mask);
    delete col;
    return SCAN_OK;
}

scan_status scan_column_info(const scan_column* col, uint64_t* n, uint32_t* b, uint32_t* base,
                             const uint32_t** dev_packed, const uint32_t** dev_zonemap)
{
    g_err.clear();
    if (!col) return fail(SCAN_EINVAL, "col is NULL");
    if (n) *n = col->n;
    if (b) *b = col->b;
    if (base) *base = col->base;
    if (dev_packed) *dev_packed = col->packed;
    if (dev_zonemap)
        *dev_zonemap = col->zonemap_valid ? reinterpret_cast<const uint32_t*>(col->zonemap) : nullptr;
    return SCAN_OK;
}

scan_status scan_zonemap_build(scan_column* col, void* stream)
{
    g_err.clear();
    if (!col) return fail(SCAN_EINVAL, "col is NULL");
    if (col->layout != SCAN_LAYOUT_LANES) return fail(SCAN_EINVAL, "zone maps are built on lane-interleaved columns");
    if (col->zonemap_valid) return SCAN_OK;
    const uint64_t nb = n_blocks(col->n);
    if (!col->zonemap) {
        GB_CUDA(cudaMalloc(&col->zonemap, std::max<uint64_t>(nb, 1) * sizeof(uint2)));
        GB_CUDA(cudaMalloc(&col->blocksum, std::max<uint64_t>(nb, 1) * sizeof(unsigned long long)));
        GB_CUDA(cudaMalloc(&col->cand, std::max<uint64_t>(nb, 1) * sizeof(unsigned int)));
    }
    if (nb) {
        gb::ScanParams p = base_params(col);
        p.zonemap_out = col->zonemap;
        p.blocksum = col->blocksum;
        const cudaError_t e = launch(static_cast<int>(col->b), gb::kOpZoneBuild, p, persistent_grid(),
                                     as_stream(stream));
        if (e != cudaSuccess) return cuda_fail(e, "zone-map build launch");
    }
    col->zonemap_valid = true;
    col->zsorted_valid = false;
    return SCAN_OK;
}

scan_status scan_run_async(scan_column* col, scan_pred pred, scan_strategy strategy, void* stream,
                           scan_result* dev_out)
{
    g_err.clear();
    if (!col || !dev_out) return fail(SCAN_EINVAL, "null pointer");
    if (reinterpret_cast<uintptr_t>(dev_out) & 7u) return fail(SCAN_EINVAL, "dev_out must be 8-byte aligned");
    bool empty = false;
    scan_status s = enqueue_scan(col, pred, strategy, as_stream(stream),
                                 reinterpret_cast<long long*>(dev_out), &empty);
    if (s != SCAN_OK) return s;
    if (empty) GB_CUDA(cudaMemsetAsync(dev_out, 0, sizeof(scan_result), as_stream(stream)));
    return SCAN_OK;
}

scan_status scan_column_status(scan_column* col, void* stream)
{
    g_err.clear();
    if (!col) return fail(SCAN_EINVAL, "col is NULL");
    unsigned int st = 0;
    GB_CUDA(cudaMemcpyAsync(&st, col->ws.status, sizeof st, cudaMemcpyDeviceToHost, as_stream(stream)));
    GB_CUDA(cudaStreamSynchronize(as_stream(stream)));
    if (st) {
        GB_CUDA(cudaMemset(col->ws_raw, 0, Workspace::kBytes));
        if (st & gb::kErrTimeout) return fail(SCAN_ETIMEOUT, "a device-side wait timed out");
        return fail(SCAN_ECUDA, "device status 0x%x", st);
    }
    return SCAN_OK;
}

scan_status scan_run(scan_column* col, scan_pred pred, scan_strategy strategy, void* stream,
                     scan_result* host_out)
{
    g_err.clear();
    if (!col || !host_out) return fail(SCAN_EINVAL, "null pointer");
    cudaStream_t st = as_stream(stream);
    bool empty = false;
    scan_status s = enqueue_scan(col, pred, strategy, st, nullptr, &empty);
    if (s != SCAN_OK) return s;
    if (empty) {
        std::memset(host_out, 0, sizeof *host_out);
        return SCAN_OK;
    }
    // result (32 B) and status word (4 B) are adjacent: one small copy
    GB_CUDA(cudaMemcpyAsync(col->host_result, col->ws.result, 36, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    unsigned int dev_status = 0;
    std::memcpy(&dev_status, reinterpret_cast<unsigned char*>(col->host_result) + 32, 4);
    if (dev_status) {
        GB_CUDA(cudaMemset(col->ws_raw, 0, Workspace::kBytes));
        return fail(SCAN_ETIMEOUT, "a device-side wait timed out (status 0x%x)", dev_status);
    }
    *host_out = *col->host_result;
    return SCAN_OK;
}

scan_status scan_probe_read(const void* dev_buf, uint64_t bytes, void* stream, uint64_t* dev_out)
{
    g_err.clear();
    if (!dev_buf || !dev_out) return fail(SCAN_EINVAL, "null pointer");
    if ((reinterpret_cast<uintptr_t>(dev_buf) & 15u) || (bytes & 15u))
        return fail(SCAN_EINVAL, "buffer must be 16-byte aligned and a multiple of 16 bytes");
    cudaStream_t st = as_stream(stream);
    GB_CUDA(cudaMemsetAsync(dev_out, 0, 8, st));
    const int grid = persistent_grid() * 4;
    k_read_probe<<<grid, 512, 0, st>>>(static_cast<const uint4*>(dev_buf), bytes / 16,
                                       reinterpret_cast<unsigned long long*>(dev_out));
    GB_CUDA(cudaGetLastError());
    return SCAN_OK;
}

scan_status scan_probe_triad(float* dev_a, const float* dev_b, const float* dev_c, float s, uint64_t n,
                             void* stream)
{
    g_err.clear();
    if (n == 0) return SCAN_OK;  // nothing to touch (empty arrays may be NULL)
    if (!dev_a || !dev_b || !dev_c) return fail(SCAN_EINVAL, "null pointer");
    if (((reinterpret_cast<uintptr_t>(dev_a) | reinterpret_cast<uintptr_t>(dev_b) |
          reinterpret_cast<uintptr_t>(dev_c)) & 15u) || (n & 3u))
        return fail(SCAN_EINVAL, "arrays must be 16-byte aligned and n a multiple of 4");
    cudaStream_t st = as_stream(stream);
    const int grid = persistent_grid() * 4;
    k_triad_probe<<<grid, 512, 0, st>>>(reinterpret_cast<float4*>(dev_a), reinterpret_cast<const float4*>(dev_b),
                                        reinterpret_cast<const float4*>(dev_c), s, n / 4);
    GB_CUDA(cudaGetLastError());
    return SCAN_OK;
}

scan_status scan_selftest_wait_timeout(uint64_t limit_ns, void* stream)
{
    g_err.clear();
    if (limit_ns == 0 || limit_ns > 1000000000ull) return fail(SCAN_EINVAL, "limit_ns must be in (0, 1e9]");
    cudaStream_t st = as_stream(stream);
    unsigned int* flag = nullptr;
    GB_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&flag), sizeof(unsigned int), st));
    GB_CUDA(cudaMemsetAsync(flag, 0, sizeof(unsigned int), st));
    k_selftest_wait<<<1, 32, 0, st>>>(limit_ns, flag);
    GB_CUDA(cudaGetLastError());
    unsigned int h = 0;
    GB_CUDA(cudaMemcpyAsync(&h, flag, sizeof h, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaFreeAsync(flag, st));
    GB_CUDA(cudaStreamSynchronize(st));
    if (h & gb::kErrTimeout) return fail(SCAN_ETIMEOUT, "the bounded wait gave up as designed");
    return fail(SCAN_ECUDA, "the bounded wait did not report its timeout");
}

scan_status scan_launch_shape(uint32_t b, uint32_t* sms, uint32_t* ctas, uint32_t* warps_per_cta,
                              uint32_t* blocks_per_tile, uint32_t* stages)
{
    g_err.clear();
    if (b < 1 || b > 32) return fail(SCAN_EINVAL, "b must be in 1..32");
    const gb::LaunchShape si = gb_shape_for(static_cast<int>(b), gb::kOpFullBF);
    if (sms) *sms = static_cast<uint32_t>(device_info().sms);
    if (ctas) *ctas = static_cast<uint32_t>(persistent_grid());
    if (warps_per_cta) *warps_per_cta = static_cast<uint32_t>(si.warps);
    if (blocks_per_tile) *blocks_per_tile = static_cast<uint32_t>(si.tile_blocks);
    if (stages) *stages = static_cast<uint32_t>(si.stages);
    return SCAN_OK;
}

}  // extern "C"
