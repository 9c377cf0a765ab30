// Instantiates the batched scan kernel for one predicate flavour and a range
// of widths (GB_BATCH_BRANCHY = 0 or 1, GB_BLO..GB_BHI, set by the build, one
// object per range so the ranges compile in parallel) and exposes its launcher.
#include <atomic>

#include "batch_kernels.cuh"

#if !defined(GB_BATCH_BRANCHY) || !defined(GB_BLO) || !defined(GB_BHI)
#error "GB_BATCH_BRANCHY, GB_BLO and GB_BHI must be defined by the build"
#endif

#define GB_CAT3(a, b, c, d) a##b##_##c##_##d
#define GB_NAME(a, b, c, d) GB_CAT3(a, b, c, d)
#if GB_BATCH_BRANCHY
#define GB_BATCH_LAUNCH GB_NAME(gb_launch_batch_br_, GB_BLO, GB_BHI, w)
#else
#define GB_BATCH_LAUNCH GB_NAME(gb_launch_batch_bf_, GB_BLO, GB_BHI, w)
#endif

namespace {

constexpr bool kBr = GB_BATCH_BRANCHY != 0;

template <int BFIX>
cudaError_t launch_fixed(const gb::BatchParams& p, int warps, int grid, cudaStream_t st)
{
    if (warps < 1 || warps > 16) return cudaErrorInvalidValue;
    static std::atomic<unsigned long long> configured{0ull};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    const void* fn = reinterpret_cast<const void*>(gb::k_scan_batch<kBr, BFIX>);
    if (!(configured.load() & bit)) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, gb::kSmemMax);
        if (e != cudaSuccess) return e;
        // all of the SM's unified memory as shared memory: two CTAs of up to
        // 112 KB of slots each must fit side by side
        e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 static_cast<int>(cudaSharedmemCarveoutMaxShared));
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    const uint32_t smem = gb::batch_smem_bytes(static_cast<uint32_t>(warps), p.stages, p.slot_bytes);
    gb::k_scan_batch<kBr, BFIX><<<grid, warps * 32, smem, st>>>(p);
    return cudaGetLastError();
}

template <int LO, int HI>
cudaError_t launch_width(int b, const gb::BatchParams& p, int warps, int grid, cudaStream_t st)
{
    if constexpr (LO > HI) {
        return cudaErrorInvalidValue;
    } else {
        if (b == LO) return launch_fixed<LO>(p, warps, grid, st);
        return launch_width<LO + 1, HI>(b, p, warps, grid, st);
    }
}

}  // namespace

// Columns all of width b (GB_BLO..GB_BHI), CTAs of `warps` warps.
cudaError_t GB_BATCH_LAUNCH(int b, const gb::BatchParams& p, int warps, int grid, cudaStream_t st)
{
    return launch_width<GB_BLO, GB_BHI>(b, p, warps, grid, st);
}
