// Host side of the conjunctive scan: argument checks, predicate translation,
// the selection-vector buffer, and the per-width mask and aggregate launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <vector>

#include "conj_kernels.cuh"
#include "internal.h"

namespace {

scan_status cfail(scan_status s, const char* msg)
{
    gb_set_last_error(msg);
    return s;
}

scan_status ccuda(cudaError_t e, const char* what)
{
    static thread_local char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    gb_set_last_error(buf);
    return e == cudaErrorMemoryAllocation ? SCAN_ENOMEM : SCAN_ECUDA;
}

#define CJ_CUDA(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return ccuda(e_, #call); \
    } while (0)

int sm_count() { return gb_device_sms(); }

// cudaFuncSetAttribute once per (kernel, device).
bool set_smem(const void* fn, int bytes, std::atomic<unsigned long long>& done)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return true;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) return false;
    done.fetch_or(bit, std::memory_order_acq_rel);
    return true;
}

template <int B, int MODE>
cudaError_t launch_pass(const gb::ConjParams& c, const gb::ScanParams& p, int grid, cudaStream_t st)
{
    static std::atomic<unsigned long long> done{0ull};
    using S = gb::ConjShape<B>;
    auto k = gb::k_conj_pass<B, MODE>;
    if (!set_smem(reinterpret_cast<const void*>(k), S::kSmemBytes, done)) return cudaErrorInvalidValue;
    k<<<grid, S::kWarps * 32, S::kSmemBytes, st>>>(c, p);
    return cudaGetLastError();
}

template <int LO, int HI>
cudaError_t pass_range(int b, int mode, const gb::ConjParams& c, const gb::ScanParams& p, int grid,
                       cudaStream_t st)
{
    if constexpr (LO > HI) {
        return cudaErrorInvalidValue;
    } else {
        if (b == LO) {
            if (mode == gb::kConjFirst) return launch_pass<LO, gb::kConjFirst>(c, p, grid, st);
            if (mode == gb::kConjAnd) return launch_pass<LO, gb::kConjAnd>(c, p, grid, st);
            return launch_pass<LO, gb::kConjAgg>(c, p, grid, st);
        }
        return pass_range<LO + 1, HI>(b, mode, c, p, grid, st);
    }
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

// Enqueue the conjunctive scan; the result (count, sum, blocks decoded, 0)
// goes to dev_result (device), or to the result column's workspace when NULL.
// *empty: no launch was needed (the result is all zero).
scan_status enqueue_conj(scan_column* const* cols, const scan_pred* preds, uint32_t k, scan_column* agg,
                         scan_strategy strategy, cudaStream_t st, long long* dev_result, bool* empty_out,
                         gb::ScanParams* rp_out)
{
    *empty_out = false;
    if (!cols || !preds || k == 0) return cfail(SCAN_EINVAL, "cols and preds are required, k >= 1");
    if (strategy != SCAN_AUTO && strategy != SCAN_BRANCHFREE)
        return cfail(SCAN_EINVAL, "the conjunctive scan takes SCAN_AUTO or SCAN_BRANCHFREE");
    struct Col {
        const uint32_t* packed;
        uint64_t n;
        uint32_t b, base, lo, wm1;
    };
    std::vector<Col> cs(k);
    bool empty = false;
    for (uint32_t c = 0; c < k; ++c) {
        const uint2* zm;
        if (!cols[c] || !gb_column_view(cols[c], &cs[c].packed, &cs[c].n, &cs[c].b, &cs[c].base, &zm))
            return cfail(SCAN_EINVAL, "a column is NULL or not lane-interleaved");
        if (cs[c].n != cs[0].n) return cfail(SCAN_EINVAL, "the columns differ in length");
        const int64_t lo_v = cs[c].base, hi_v = static_cast<int64_t>(cs[c].base) + (1ll << cs[c].b);
        const int64_t lo = std::max(preds[c].lo, lo_v), hi = std::min(preds[c].hi, hi_v);
        if (lo >= hi) {
            empty = true;
        } else {
            cs[c].lo = static_cast<uint32_t>(lo - lo_v);
            cs[c].wm1 = static_cast<uint32_t>(hi - lo - 1);
        }
    }
    Col ag{};
    if (agg) {
        const uint2* zm;
        if (!gb_column_view(agg, &ag.packed, &ag.n, &ag.b, &ag.base, &zm))
            return cfail(SCAN_EINVAL, "the aggregate column is not lane-interleaved");
        if (ag.n != cs[0].n) return cfail(SCAN_EINVAL, "the aggregate column differs in length");
    }
    gb::ScanParams rp = gb_column_params(agg ? agg : cols[0]);
    if (dev_result) rp.result = dev_result;
    if (rp_out) *rp_out = rp;
    const uint64_t n = cs[0].n;
    if (n == 0 || empty) {
        *empty_out = true;
        return SCAN_OK;
    }
    const uint64_t nblocks = (n + 1023u) >> 10;
    uint32_t* mask = nullptr;  // the result column's selection vector, reused across calls
    CJ_CUDA(gb_column_conj_mask(agg ? agg : cols[0], nblocks * 32u, &mask));
    const int grid = sm_count();
    cudaError_t e = cudaSuccess;
    for (uint32_t c = 0; c < k && e == cudaSuccess; ++c) {
        gb::ConjParams p{cs[c].packed, n, cs[c].lo, cs[c].wm1, mask, rp.status};
        e = pass_range<1, 32>(static_cast<int>(cs[c].b), c == 0 ? gb::kConjFirst : gb::kConjAnd, p, rp, grid, st);
    }
    if (e == cudaSuccess) {
        if (agg) {
            gb::ConjParams p{ag.packed, n, 0u, 0u, mask, rp.status};
            e = pass_range<1, 32>(static_cast<int>(ag.b), gb::kConjAgg, p, rp, grid, st);
        } else {
            gb::ScanParams cp = rp;
            cp.base = 0;
            gb::k_conj_count<<<grid, 256, 0, st>>>(cp, mask, nblocks * 32u);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) return ccuda(e, "conjunctive scan launch");
    return SCAN_OK;
}

}  // namespace

extern "C" scan_status scan_conj(scan_column* const* cols, const scan_pred* preds, uint32_t k, scan_column* agg,
                                 scan_strategy strategy, void* stream, scan_result* host_out)
{
    gb_set_last_error("");
    if (!host_out) return cfail(SCAN_EINVAL, "host_out is NULL");
    std::memset(host_out, 0, sizeof *host_out);
    cudaStream_t st = as_stream(stream);
    bool empty = false;
    gb::ScanParams rp{};
    const scan_status s = enqueue_conj(cols, preds, k, agg, strategy, st, nullptr, &empty, &rp);
    if (s != SCAN_OK || empty) return s;
    long long res[4];
    unsigned int dev_status = 0;
    CJ_CUDA(cudaMemcpyAsync(res, rp.result, sizeof res, cudaMemcpyDeviceToHost, st));
    CJ_CUDA(cudaMemcpyAsync(&dev_status, rp.status, sizeof dev_status, cudaMemcpyDeviceToHost, st));
    CJ_CUDA(cudaStreamSynchronize(st));
    if (dev_status) {
        CJ_CUDA(cudaMemset(rp.status, 0, sizeof(unsigned int)));
        return cfail(SCAN_ETIMEOUT, "a device-side wait timed out in the conjunctive scan");
    }
    host_out->count = res[0];
    host_out->sum = res[1];
    host_out->blocks_scanned = res[2];
    return SCAN_OK;
}

extern "C" scan_status scan_conj_async(scan_column* const* cols, const scan_pred* preds, uint32_t k,
                                       scan_column* agg, scan_strategy strategy, void* stream, scan_result* dev_out)
{
    gb_set_last_error("");
    if (!dev_out) return cfail(SCAN_EINVAL, "dev_out is NULL");
    cudaStream_t st = as_stream(stream);
    bool empty = false;
    const scan_status s =
        enqueue_conj(cols, preds, k, agg, strategy, st, reinterpret_cast<long long*>(dev_out), &empty, nullptr);
    if (s != SCAN_OK) return s;
    if (empty) CJ_CUDA(cudaMemsetAsync(dev_out, 0, sizeof(scan_result), st));
    return SCAN_OK;
}
