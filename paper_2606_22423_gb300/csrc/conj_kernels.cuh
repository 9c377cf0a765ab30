// Conjunctive predicates over several columns of one table (the problem of
// paper §2 over rows shared by k columns): COUNT of the rows that satisfy
// every column's range, and SUM of an aggregate column over them.
//
// Selection vector: one 32-bit mask per (1024-row block, lane), bit r = row
// 32r + lane -- the per-lane mask of the materializing select.  One pass per
// predicate column streams the column through a persistent TMA pipeline and
// writes (first column) or ANDs (later columns) its masks -- the incoming
// masks of a tile arrive by bulk copy with its data, so no load waits in the
// loop -- and a block whose incoming selection is already empty is not
// decoded.  A last pass aggregates the aggregate column over the final masks
// (or, with no aggregate column, only counts the selected rows) and folds the
// grid's partial sums with the scans' last-CTA finish, FOR base included.
#pragma once
#include <cstdint>

#include "scan_kernels.cuh"
#include "select_kernels.cuh"

namespace gb {

struct ConjParams {
    const uint32_t* packed;  // the column of this pass (lane layout, padded to whole blocks)
    uint64_t n;              // rows
    uint32_t lo, wm1;        // predicate in code space (mask passes)
    uint32_t* mask;          // nblocks * 32 selection words
    unsigned int* status;
};

enum ConjMode : int { kConjFirst = 0, kConjAnd = 1, kConjAgg = 2 };

// Staging shape: a tile is kTB blocks of data (128*B bytes each) followed by
// their selection words (128 bytes each), both brought in by bulk copies on
// one transaction barrier, at most ~4 KB per slot; 16 warps per CTA, so that
// four warps per scheduler hide the latency of the decode's dependent steps.
template <int B>
struct ConjShape {
    static constexpr int kWarps = 16;
    static constexpr int kStages = 3;
    static constexpr int kBlockBytes = 128 * B;
    static constexpr int kRaw = 4096 / (kBlockBytes + 128);
    static constexpr int kTB = kRaw < 1 ? 1 : (kRaw > 64 ? 64 : kRaw);
    static constexpr int kDataBytes = kTB * kBlockBytes;
    static constexpr int kTileBytes = kDataBytes + kTB * 128;
    static constexpr int kSlotBytes = kWarps * kStages * kTileBytes;
    static constexpr int kSmemBytes = kSlotBytes + kWarps * kStages * 8;
    static_assert(kSmemBytes <= 227 * 1024, "shared-memory budget");
    static_assert(kDataBytes % 16 == 0 && kTileBytes % 16 == 0, "bulk copies move multiples of 16 bytes");
};

// One persistent pass over a column, per mode:
//   kConjFirst: mask := the column's predicate mask;
//   kConjAnd  : mask &= the column's predicate mask (blocks already empty are not decoded);
//   kConjAgg  : COUNT and code SUM of the column over the mask (blocks with no selected
//               row are not decoded); the last CTA finishes (count, sum + base*count,
//               blocks decoded) into p.result.
template <int B, int MODE>
__global__ void __launch_bounds__(ConjShape<B>::kWarps * 32, 1)
k_conj_pass(const ConjParams c, const ScanParams p)
{
    using S = ConjShape<B>;
    constexpr bool kMaskIn = MODE != kConjFirst;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned int decoded;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* slots = smem + static_cast<size_t>(warp) * S::kStages * S::kTileBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S::kSlotBytes) + warp * S::kStages;

    const uint64_t nblocks = (c.n + 1023u) >> 10;
    const uint64_t ntiles = (nblocks + S::kTB - 1) / S::kTB;
    const uint32_t tail = static_cast<uint32_t>(c.n & 1023u);
    // warp-major numbering, as the full scan: a partial last round is spread over all SMs
    const uint64_t gw = static_cast<uint64_t>(warp) * gridDim.x + blockIdx.x;
    const uint64_t GW = static_cast<uint64_t>(gridDim.x) * S::kWarps;

    if (threadIdx.x == 0) decoded = 0u;
    if (lane == 0) {
        for (int s = 0; s < S::kStages; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto tile_blocks = [&](uint64_t t) -> uint32_t {
        const uint64_t left = nblocks - t * S::kTB;
        return left < S::kTB ? static_cast<uint32_t>(left) : static_cast<uint32_t>(S::kTB);
    };
    auto issue = [&](uint64_t t, int s) {
        const uint32_t nb = tile_blocks(t);
        unsigned char* dst = slots + s * S::kTileBytes;
        mbar_arrive_expect_tx(&bars[s], nb * S::kBlockBytes + (kMaskIn ? nb * 128u : 0u));
        bulk_g2s(dst, c.packed + t * S::kTB * 32u * B, nb * S::kBlockBytes, &bars[s]);
        if constexpr (kMaskIn) bulk_g2s(dst + S::kDataBytes, c.mask + t * S::kTB * 32u, nb * 128u, &bars[s]);
    };
    if (lane == 0) {
        for (int s = 0; s < S::kStages; ++s) {
            const uint64_t t = gw + s * GW;
            if (t < ntiles) issue(t, s);
        }
    }
    uint64_t cnt = 0, sum = 0;
    uint32_t it = 0, mine = 0;
    bool failed = false;
#pragma unroll 1
    for (uint64_t t = gw; t < ntiles; t += GW, ++it) {
        const int s = static_cast<int>(it % S::kStages);
        const bool ok = mbar_wait(&bars[s], (it / S::kStages) & 1u, kWaitLimitNs);
        if (!__all_sync(kFull, ok)) {
            failed = true;
            break;
        }
        const uint32_t nb = tile_blocks(t);
        const uint32_t* tw = reinterpret_cast<const uint32_t*>(slots + s * S::kTileBytes);
        const uint32_t* tm = reinterpret_cast<const uint32_t*>(slots + s * S::kTileBytes + S::kDataBytes);
#pragma unroll 1
        for (uint32_t k = 0; k < nb; ++k) {
            const uint64_t blk = t * S::kTB + k;
            const uint32_t in = kMaskIn ? tm[k * 32u + lane] : 0xffffffffu;
            if constexpr (kMaskIn) {
                if (!__any_sync(kFull, in != 0u)) continue;  // no selected row in the block
            }
            if constexpr (MODE == kConjAgg) {
                ++mine;
                uint32_t W[B];
#pragma unroll
                for (int w = 0; w < B; ++w) W[w] = tw[k * 32u * B + w * 32 + lane];
                uint64_t bs = 0;
#pragma unroll
                for (int r = 0; r < 32; ++r)
                    if ((in >> r) & 1u) bs += sel_code<B>(W, r);
                cnt += static_cast<uint32_t>(__popc(in));
                sum += bs;
            } else {
                const uint32_t limit = (tail && blk == nblocks - 1) ? tail : 1024u;
                c.mask[blk * 32u + lane] = in & sel_block_mask<B>(tw + k * 32u * B, lane, c.lo, c.wm1, limit);
            }
        }
        __syncwarp();
        const uint64_t tn = t + static_cast<uint64_t>(S::kStages) * GW;
        if (lane == 0 && tn < ntiles) {
            fence_proxy_async_smem();
            issue(tn, s);
        }
    }
    if (failed) {
        if (lane == 0) atomicOr(c.status, kErrTimeout);
        for (uint32_t j = 0; j < static_cast<uint32_t>(S::kStages); ++j) {
            const uint64_t t = gw + static_cast<uint64_t>(it + j) * GW;
            if (t >= ntiles) break;
            const uint32_t jt = it + j;
            mbar_wait(&bars[jt % S::kStages], (jt / S::kStages) & 1u, kDrainLimitNs);
        }
    }
    if constexpr (MODE == kConjAgg) {
        if (lane == 0 && mine) atomicAdd(&decoded, mine);
        __syncthreads();
        // blocks decoded by the grid, folded in by the last CTA as the queue's candidate count
        if (threadIdx.x == 0 && decoded) atomicAdd(&p.qctl[0], static_cast<unsigned long long>(decoded));
        grid_finish<S::kWarps>(p, cnt, sum, true, 0);
    }
}

// Count-only pass (no aggregate column): popc of the masks.
__global__ void __launch_bounds__(256) k_conj_count(const ScanParams p, const uint32_t* mask, uint64_t words)
{
    uint64_t cnt = 0;
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < words;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        cnt += static_cast<uint32_t>(__popc(mask[i]));
    grid_finish<8>(p, cnt, 0, false, 0);
}

}  // namespace gb
