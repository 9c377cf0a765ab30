// Instantiates the scan kernels for widths GB_BLO..GB_BHI (set by the build,
// one object per range so the ranges compile in parallel) and exposes one
// launcher per range.
#include <atomic>

#include "scan_kernels.cuh"

#ifndef GB_BLO
#error "GB_BLO / GB_BHI must be defined by the build"
#endif

namespace gb {
namespace {

// cudaFuncSetAttribute once per (kernel, device).
template <int B, int OP>
bool smem_configured(const void* fn, int smem)
{
    static std::atomic<unsigned long long> done_mask{0ull};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done_mask.load(std::memory_order_acquire) & bit) return true;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return false;
    done_mask.fetch_or(bit, std::memory_order_acq_rel);
    return true;
}

template <int B, int OP, class K>
cudaError_t launch_one(K kernel, const ScanParams& p, int grid, cudaStream_t st)
{
    using S = Shape<B>;
    if (!smem_configured<B, OP>(reinterpret_cast<const void*>(kernel), S::kSmemBytes))
        return cudaGetLastError() != cudaSuccess ? cudaGetLastError() : cudaErrorInvalidValue;
    kernel<<<grid, S::kWarps * 32, S::kSmemBytes, st>>>(p);
    return cudaGetLastError();
}

template <int B>
cudaError_t launch_b(int op, const ScanParams& p, int grid, cudaStream_t st)
{
    switch (op) {
    case kOpFullBF: return launch_one<B, kOpFullBF>(k_scan_full<B, false>, p, grid, st);
    case kOpFullBR: return launch_one<B, kOpFullBR>(k_scan_full<B, true>, p, grid, st);
    case kOpQueueBF: return launch_one<B, kOpQueueBF>(k_scan_queue<B, false>, p, grid, st);
    case kOpQueueBR: return launch_one<B, kOpQueueBR>(k_scan_queue<B, true>, p, grid, st);
    case kOpZoneBuild: return launch_one<B, kOpZoneBuild>(k_zonemap_build<B>, p, grid, st);
    case kOpRowBF: return launch_one<B, kOpRowBF>(k_scan_full<B, false, kLayRow>, p, grid, st);
    case kOpRowBR: return launch_one<B, kOpRowBR>(k_scan_full<B, true, kLayRow>, p, grid, st);
    case kOpBytesBF:
    case kOpBytesBR:
        if constexpr (B == 8 || B == 16) {
            if (op == kOpBytesBF) return launch_one<B, kOpBytesBF>(k_scan_full<B, false, kLayBytes>, p, grid, st);
            return launch_one<B, kOpBytesBR>(k_scan_full<B, true, kLayBytes>, p, grid, st);
        }
        return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

template <int LO, int HI>
cudaError_t dispatch_range(int b, int op, const ScanParams& p, int grid, cudaStream_t st)
{
    if constexpr (LO > HI) {
        return cudaErrorInvalidValue;
    } else {
        if (b == LO) return launch_b<LO>(op, p, grid, st);
        return dispatch_range<LO + 1, HI>(b, op, p, grid, st);
    }
}

}  // namespace
}  // namespace gb

#define GB_CAT2(a, b, c) a##b##_##c
#define GB_CAT(a, b, c) GB_CAT2(a, b, c)

cudaError_t GB_CAT(gb_launch_range_, GB_BLO, GB_BHI)(int b, int op, const gb::ScanParams& p, int grid,
                                                     cudaStream_t st)
{
    return gb::dispatch_range<GB_BLO, GB_BHI>(b, op, p, grid, st);
}
