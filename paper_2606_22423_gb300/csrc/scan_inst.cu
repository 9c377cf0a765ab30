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

// cudaFuncSetAttribute once per (kernel, device): every instantiation may use
// up to the whole shared-memory budget; each launch passes its own size.
template <auto KERNEL>
bool smem_configured()
{
    static std::atomic<unsigned long long> done_mask{0ull};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done_mask.load(std::memory_order_acquire) & bit) return true;
    if (cudaFuncSetAttribute(reinterpret_cast<const void*>(KERNEL), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmemMax) != cudaSuccess)
        return false;
    done_mask.fetch_or(bit, std::memory_order_acq_rel);
    return true;
}

template <int B, auto KERNEL>
cudaError_t launch_one(const ScanParams& p, const LaunchShape& sh, int grid, cudaStream_t st)
{
    if (!smem_configured<KERNEL>())
        return cudaGetLastError() != cudaSuccess ? cudaGetLastError() : cudaErrorInvalidValue;
    ScanParams q = p;
    q.tile_blocks = static_cast<uint32_t>(sh.tile_blocks);
    q.stages = static_cast<uint32_t>(sh.stages);
    const uint32_t smem = pipe_smem_bytes(B, sh.warps, sh.stages, sh.tile_blocks);
    KERNEL<<<grid, sh.warps * 32, smem, st>>>(q);
    return cudaGetLastError();
}

// Full scans: the 16-warp-bound instantiation for CTAs above 8 warps; the
// branchy vote group per row where the shape asks for it (b <= 21).
template <int B, bool BRANCHY>
cudaError_t launch_full(const ScanParams& p, const LaunchShape& sh, int grid, cudaStream_t st)
{
    if constexpr (B >= 9 && B <= 16) {  // the 2-lane geometry: 16-warp bound only
        if (sh.vec_lanes == 2) {
            if constexpr (BRANCHY) {
                if (sh.vote_rows == 3) return launch_one<B, k_scan_full<B, true, kLayLanes, 16, 3, 2>>(p, sh, grid, st);
                if (sh.vote_rows == 2) return launch_one<B, k_scan_full<B, true, kLayLanes, 16, 2, 2>>(p, sh, grid, st);
                if (sh.vote_rows) return launch_one<B, k_scan_full<B, true, kLayLanes, 16, 1, 2>>(p, sh, grid, st);
            }
            return launch_one<B, k_scan_full<B, BRANCHY, kLayLanes, 16, 0, 2>>(p, sh, grid, st);
        }
    }
    if (sh.vec_lanes != 0 && sh.vec_lanes != default_lpt(B)) return cudaErrorInvalidValue;
    const bool w16 = sh.warps > 8;
    if constexpr (BRANCHY && B <= 21) {
        // the PTX row vote: the 16-warp bound only (any CTA up to 16 warps)
        if (sh.vote_rows == 3) return launch_one<B, k_scan_full<B, true, kLayLanes, 16, 3>>(p, sh, grid, st);
        if (sh.vote_rows == 2) return launch_one<B, k_scan_full<B, true, kLayLanes, 16, 2>>(p, sh, grid, st);
        if (sh.vote_rows)
            return w16 ? launch_one<B, k_scan_full<B, true, kLayLanes, 16, 1>>(p, sh, grid, st)
                       : launch_one<B, k_scan_full<B, true, kLayLanes, 8, 1>>(p, sh, grid, st);
    }
    return w16 ? launch_one<B, k_scan_full<B, BRANCHY, kLayLanes, 16, 0>>(p, sh, grid, st)
               : launch_one<B, k_scan_full<B, BRANCHY, kLayLanes, 8, 0>>(p, sh, grid, st);
}

template <int B>
cudaError_t launch_b(int op, const ScanParams& p, const LaunchShape& sh, int grid, cudaStream_t st)
{
    if (sh.warps > 8 && op != kOpFullBF && op != kOpFullBR) return cudaErrorInvalidValue;
    switch (op) {
    case kOpFullBF: return launch_full<B, false>(p, sh, grid, st);
    case kOpFullBR: return launch_full<B, true>(p, sh, grid, st);
    case kOpQueueBF: return launch_one<B, k_scan_queue<B, false>>(p, sh, grid, st);
    case kOpQueueBR: return launch_one<B, k_scan_queue<B, true>>(p, sh, grid, st);
    case kOpZoneBuild: return launch_one<B, k_zonemap_build<B>>(p, sh, grid, st);
    case kOpRowBF: return launch_one<B, k_scan_full<B, false, kLayRow>>(p, sh, grid, st);
    case kOpRowBR: return launch_one<B, k_scan_full<B, true, kLayRow>>(p, sh, grid, st);
    case kOpBytesBF:
    case kOpBytesBR:
        if constexpr (B == 8 || B == 16) {
            if (op == kOpBytesBF) return launch_one<B, k_scan_full<B, false, kLayBytes>>(p, sh, grid, st);
            return launch_one<B, k_scan_full<B, true, kLayBytes>>(p, sh, grid, st);
        }
        return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

template <int LO, int HI>
cudaError_t dispatch_range(int b, int op, const ScanParams& p, const LaunchShape& sh, int grid, cudaStream_t st)
{
    if constexpr (LO > HI) {
        return cudaErrorInvalidValue;
    } else {
        if (b == LO) return launch_b<LO>(op, p, sh, grid, st);
        return dispatch_range<LO + 1, HI>(b, op, p, sh, grid, st);
    }
}

}  // namespace
}  // namespace gb

#define GB_CAT2(a, b, c) a##b##_##c
#define GB_CAT(a, b, c) GB_CAT2(a, b, c)

cudaError_t GB_CAT(gb_launch_range_, GB_BLO, GB_BHI)(int b, int op, const gb::ScanParams& p,
                                                     const gb::LaunchShape& sh, int grid, cudaStream_t st)
{
    return gb::dispatch_range<GB_BLO, GB_BHI>(b, op, p, sh, grid, st);
}
