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

cudaError_t GB_BATCH_LAUNCH(const gb::BatchParams& p, int grid, cudaStream_t st)
{
    static std::atomic<unsigned long long> configured{0ull};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    const void* fn = reinterpret_cast<const void*>(gb::k_scan_batch<GB_BATCH_BRANCHY != 0>);
    if (!(configured.load() & bit)) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, gb::kBatchSmem);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    gb::k_scan_batch<GB_BATCH_BRANCHY != 0><<<grid, gb::kBatchWarps * 32, gb::kBatchSmem, st>>>(p);
    return cudaGetLastError();
}
