// Host side of the materializing select: argument checks, predicate
// translation to code space, the per-column workspace of tagged CTA totals,
// and a cooperative launch of the width-specialised k_select kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <atomic>
#include <cstdio>
#include <cstring>

#include "internal.h"
#include "select_kernels.cuh"

namespace {

scan_status sfail(scan_status s, const char* msg)
{
    gb_set_last_error(msg);
    return s;
}

scan_status scuda(cudaError_t e, const char* what)
{
    static thread_local char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    gb_set_last_error(buf);
    return e == cudaErrorMemoryAllocation ? SCAN_ENOMEM : SCAN_ECUDA;
}

#define SL_CUDA(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return scuda(e_, #call); \
    } while (0)

template <int B, bool BRANCHY>
cudaError_t launch_one(const gb::SelectParams& p, int grid, cudaStream_t st)
{
    using S = gb::SelShape<B>;
    auto kernel = gb::k_select<B, BRANCHY>;
    static std::atomic<unsigned long long> configured{0ull};  // one bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured.load(std::memory_order_acquire) & bit)) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kSmemBytes);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit, std::memory_order_acq_rel);
    }
    gb::SelectParams q = p;
    void* args[] = {&q};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kernel), dim3(grid),
                                       dim3(gb::kSelWarps * 32), args, S::kSmemBytes, st);
}

template <bool BRANCHY, int LO, int HI>
cudaError_t launch_range(int b, const gb::SelectParams& p, int grid, cudaStream_t st)
{
    if constexpr (LO > HI) {
        return cudaErrorInvalidValue;
    } else {
        if (b == LO) return launch_one<LO, BRANCHY>(p, grid, st);
        return launch_range<BRANCHY, LO + 1, HI>(b, p, grid, st);
    }
}

// Blocks a warp covers per iteration (tiles per iteration x blocks per tile).
template <int LO, int HI>
int iter_blocks_range(int b)
{
    if constexpr (LO > HI) {
        return 1;
    } else {
        if (b == LO) return gb::SelShape<LO>::kIB;
        return iter_blocks_range<LO + 1, HI>(b);
    }
}

// Enqueue the select; *empty = true when no value can match (nothing launched).
scan_status enqueue_select(scan_column* col, scan_pred pred, scan_strategy strategy, uint32_t* dev_positions,
                           uint64_t capacity, cudaStream_t st, unsigned long long* dev_count, bool* empty,
                           GbSelectWs* ws_out, uint64_t wait_limit_ns = gb::kWaitLimitNs, int32_t silent_cta = -1)
{
    *empty = false;
    if (!col) return sfail(SCAN_EINVAL, "col is NULL");
    if (capacity && !dev_positions) return sfail(SCAN_EINVAL, "dev_positions is NULL with capacity > 0");
    bool branchy;
    switch (strategy) {
    case SCAN_AUTO:
    case SCAN_BRANCHFREE: branchy = false; break;
    case SCAN_BRANCHY: branchy = true; break;
    default: return sfail(SCAN_EINVAL, "select takes SCAN_BRANCHFREE, SCAN_BRANCHY or SCAN_AUTO");
    }
    const uint32_t* packed = nullptr;
    const uint2* zm = nullptr;
    uint64_t n = 0;
    uint32_t b = 0, base = 0;
    if (!gb_column_view(col, &packed, &n, &b, &base, &zm))
        return sfail(SCAN_EINVAL, "the select takes lane-interleaved columns");
    // [lo, hi) on decoded values -> code space, clipped to the column's domain
    const int64_t lo_v = static_cast<int64_t>(base);
    const int64_t hi_v = static_cast<int64_t>(base) + (1ll << b);
    const int64_t lo = std::max(pred.lo, lo_v);
    const int64_t hi = std::min(pred.hi, hi_v);
    if (n == 0 || lo >= hi) {
        *empty = true;
        return SCAN_OK;
    }
    if (!gb_device_coop()) return sfail(SCAN_ENOTSUP, "the device cannot launch cooperative kernels");
    const int grid = std::min(gb_device_sms(), 256);  // the kernel polls up to 256 CTA totals per iteration
    const uint64_t nblocks = (n + 1023u) >> 10;
    // iteration i covers blocks [i*warps*ib, (i+1)*warps*ib): ib per warp, tiles
    // never straddling two warps (ib is a whole number of tiles)
    const uint64_t ib = static_cast<uint64_t>(iter_blocks_range<1, 32>(static_cast<int>(b)));
    const uint64_t warps = static_cast<uint64_t>(grid) * gb::kSelWarps;
    const uint64_t niter = (nblocks + warps * ib - 1) / (warps * ib);
    GbSelectWs ws{};
    SL_CUDA(gb_column_select_ws(col, niter * static_cast<uint64_t>(grid), st, &ws));
    gb::SelectParams p{};
    p.packed = packed;
    p.n = n;
    p.lo = static_cast<uint32_t>(lo - lo_v);
    p.wm1 = static_cast<uint32_t>(hi - lo - 1);
    p.pos = dev_positions;
    p.capacity = capacity;
    p.agg = ws.agg;
    p.epoch = ws.epoch;
    p.niter = static_cast<uint32_t>(niter);
    p.count = dev_count ? dev_count : reinterpret_cast<unsigned long long*>(ws.result);
    p.status = ws.status;
    p.wait_limit_ns = wait_limit_ns;
    p.silent_cta = silent_cta;
    const cudaError_t e = branchy ? launch_range<true, 1, 32>(static_cast<int>(b), p, grid, st)
                                  : launch_range<false, 1, 32>(static_cast<int>(b), p, grid, st);
    if (e != cudaSuccess) return scuda(e, "select kernel launch");
    if (ws_out) *ws_out = ws;
    return SCAN_OK;
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

}  // namespace

extern "C" {

scan_status scan_select_async(scan_column* col, scan_pred pred, scan_strategy strategy, uint32_t* dev_positions,
                              uint64_t capacity, void* stream, uint64_t* dev_count)
{
    gb_set_last_error("");
    if (!dev_count) return sfail(SCAN_EINVAL, "dev_count is NULL");
    bool empty = false;
    const scan_status s = enqueue_select(col, pred, strategy, dev_positions, capacity, as_stream(stream),
                                         reinterpret_cast<unsigned long long*>(dev_count), &empty, nullptr);
    if (s != SCAN_OK) return s;
    if (empty) SL_CUDA(cudaMemsetAsync(dev_count, 0, sizeof(uint64_t), as_stream(stream)));
    return SCAN_OK;
}

scan_status scan_select(scan_column* col, scan_pred pred, scan_strategy strategy, uint32_t* dev_positions,
                        uint64_t capacity, void* stream, uint64_t* host_count)
{
    gb_set_last_error("");
    if (!host_count) return sfail(SCAN_EINVAL, "host_count is NULL");
    cudaStream_t st = as_stream(stream);
    bool empty = false;
    GbSelectWs ws{};
    const scan_status s = enqueue_select(col, pred, strategy, dev_positions, capacity, st, nullptr, &empty, &ws);
    if (s != SCAN_OK) return s;
    if (empty) {
        *host_count = 0;
        return SCAN_OK;
    }
    // result slot (32 B) and status word (4 B) are adjacent: one small copy
    SL_CUDA(cudaMemcpyAsync(ws.host_result, ws.result, 36, cudaMemcpyDeviceToHost, st));
    SL_CUDA(cudaStreamSynchronize(st));
    unsigned int dev_status = 0;
    std::memcpy(&dev_status, reinterpret_cast<unsigned char*>(ws.host_result) + 32, 4);
    if (dev_status) {
        SL_CUDA(cudaMemset(ws.status, 0, sizeof(unsigned int)));
        return sfail(SCAN_ETIMEOUT, "a device-side wait timed out in the select kernel");
    }
    *host_count = static_cast<uint64_t>(ws.host_result->count);
    return SCAN_OK;
}

scan_status scan_selftest_select_timeout(scan_column* col, uint64_t limit_ns, void* stream)
{
    gb_set_last_error("");
    if (!col) return sfail(SCAN_EINVAL, "col is NULL");
    if (limit_ns == 0 || limit_ns > 1000000000ull) return sfail(SCAN_EINVAL, "limit_ns must be in (0, 1e9]");
    cudaStream_t st = as_stream(stream);
    bool empty = false;
    GbSelectWs ws{};
    // every value matches, nothing is written (capacity 0), and CTA 0 never publishes
    const scan_status s = enqueue_select(col, scan_pred{INT64_MIN / 2, INT64_MAX / 2}, SCAN_BRANCHFREE, nullptr, 0,
                                         st, nullptr, &empty, &ws, limit_ns, 0);
    if (s != SCAN_OK) return s;
    if (empty) return sfail(SCAN_EINVAL, "the column is empty");
    unsigned int dev_status = 0;
    SL_CUDA(cudaMemcpyAsync(&dev_status, ws.status, sizeof dev_status, cudaMemcpyDeviceToHost, st));
    SL_CUDA(cudaStreamSynchronize(st));
    if (dev_status & gb::kSelSelectErr) {
        SL_CUDA(cudaMemset(ws.status, 0, sizeof(unsigned int)));
        return sfail(SCAN_ETIMEOUT, "the waits on the silent CTA gave up as designed");
    }
    return sfail(SCAN_ECUDA, "the select finished although one CTA never published");
}

}  // extern "C"
