// Instantiates the batched scan kernel for one predicate flavour
// (GB_BATCH_BRANCHY = 0 or 1, set by the build) and exposes its launcher.
#include <atomic>

#include "batch_kernels.cuh"

#ifndef GB_BATCH_BRANCHY
#error "GB_BATCH_BRANCHY must be defined by the build"
#endif

#if GB_BATCH_BRANCHY
#define GB_BATCH_LAUNCH gb_launch_batch_branchy
#else
#define GB_BATCH_LAUNCH gb_launch_batch_branchfree
#endif

namespace {

constexpr bool kBr = GB_BATCH_BRANCHY != 0;

template <int BFIX>
cudaError_t launch_fixed(const gb::BatchParams& p, int grid, cudaStream_t st)
{
    static std::atomic<unsigned long long> configured{0ull};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    const void* fn = reinterpret_cast<const void*>(gb::k_scan_batch<kBr, BFIX>);
    if (!(configured.load() & bit)) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, gb::kBatchSmem);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    gb::k_scan_batch<kBr, BFIX><<<grid, gb::kBatchWarps * 32, gb::kBatchSmem, st>>>(p);
    return cudaGetLastError();
}

template <int LO, int HI>
cudaError_t launch_width(int b, const gb::BatchParams& p, int grid, cudaStream_t st)
{
    if constexpr (LO > HI) {
        return cudaErrorInvalidValue;
    } else {
        if (b == LO) return launch_fixed<LO>(p, grid, st);
        return launch_width<LO + 1, HI>(b, p, grid, st);
    }
}

}  // namespace

// Columns of any width (b = 0) or all of width b (1..32).
cudaError_t GB_BATCH_LAUNCH(int b, const gb::BatchParams& p, int grid, cudaStream_t st)
{
    if (b == 0) return launch_fixed<0>(p, grid, st);
    return launch_width<1, 32>(b, p, grid, st);
}
