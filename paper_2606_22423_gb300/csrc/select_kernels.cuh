// Materializing select over a lane-interleaved bit-packed column: the
// positions i of the values with lo <= v_i < hi, written in increasing order
// (paper §3 lists "a materializing select" beside the count aggregates; §4
// "Branch" is where its branchy and predicated forms part ways).
//
// One persistent, co-resident grid (one CTA of 16 warps per SM).  Each warp
// streams its own tiles through a ring of two or three bulk copies.  The output
// order needs every tile's offset, i.e. the number of matches in all earlier
// tiles, so the work runs in iterations: in iteration i warp gw owns the M
// consecutive tiles starting at tile (i*GW + gw)*M (GW = warps in the grid;
// M tiles make about 8 blocks), which makes each iteration one contiguous
// range of tiles.
//   count pass : decode the tile from shared memory once and keep, per lane
//                and block, a 32-bit column mask (bit r = value 32r + lane
//                matches).  The data slot is refilled right away; only the
//                masks (128 B per block) stay.
//   publish    : the last warp of the CTA to count iteration i publishes the
//                CTA's total for i as (epoch << 32 | count) in global memory.
//   write pass : kSelLag iterations later (the other CTAs have published by
//                then), the warp reads the grid's totals for that iteration
//                and adds the totals of the CTAs and warps before it.  Per
//                block a 32 x 32 bit transpose across the warp turns column
//                masks into row masks (lane r holds row r: values 32r..32r+31
//                in index order), a warp scan of the row counts gives where
//                each row's matches start, lane r writes its row's positions
//                to the warp's shared-memory stage (padded against bank conflicts), and the warp copies the
//                stage out with consecutive lanes on consecutive positions.
// Branch-free visits all 32 bits of every row with a predicated store, a
// fixed cost; branchy loops over each row's set bits only, so its cost grows
// with the selectivity and its lanes diverge when their rows hold different
// numbers of matches (the SIMT counterpart of a data-dependent branch).
//
// Every wait (bulk copy, another CTA's total) is bounded by the global timer;
// on expiry the kernel sets kErrTimeout, lets its copies in flight land and
// returns.  The launch is cooperative, so all CTAs are resident together.
#pragma once
#include <cstdint>

#include "gb_ptx.cuh"

namespace gb {

struct SelectParams {
    const uint32_t* packed;       // lane-interleaved words, ceil(n/1024)*32*b of them
    uint64_t n;
    uint32_t lo;                  // predicate in code space: (u - lo) <= wm1
    uint32_t wm1;
    uint32_t* pos;                // output positions (capacity of them)
    uint64_t capacity;
    unsigned long long* agg;      // niter * gridDim.x words: (epoch << 32) | CTA count
    uint32_t epoch;               // this launch's tag; older words carry older tags
    uint32_t niter;               // ceil(tiles / warps in the grid)
    unsigned long long* count;    // total number of matches
    unsigned int* status;         // kErrTimeout on an expired wait
    uint64_t wait_limit_ns;       // bound of every wait (kWaitLimitNs in normal use)
    int32_t silent_cta;           // -1; a self-test names a CTA that never publishes
};

// 16 warps per CTA (four per scheduler): the count and write passes are
// chains of dependent ALU and shuffle steps, and more resident warps hide
// their latency.  That leaves ~14 KB of shared memory per warp.
constexpr int kSelWarps = 16;
constexpr int kSelTileBytes = 4096;  // data of one bulk copy, at most
constexpr int kSelLag = 3;      // a tile is written kSelLag iterations after it was counted
constexpr int kSelRing = 8;     // CTA count ring; must be >= 2 * kSelLag + 2
constexpr uint32_t kSelSelectErr = 1u;  // same bit as kErrTimeout
static_assert(kSelRing >= 2 * kSelLag + 2, "a CTA count slot is reused before every warp has read it");
// Per-warp stage of one block's in-block indices (u16): two padding entries
// after every 32, so that the 32 rows' writes at 32r + j fall in distinct banks.
constexpr int kSelStageHalfs = 1024 + 64;

// Shared memory of one warp: a ring of `st` tiles of tb blocks, the column
// masks of kSelLag + 1 iterations of m tiles, the index stage, the barriers.
__host__ __device__ constexpr int sel_warp_bytes(int b, int st, int tb, int m)
{
    return st * tb * 128 * b + (kSelLag + 1) * tb * m * 32 * 4 + kSelStageHalfs * 2 + st * 8;
}

__host__ __device__ constexpr bool sel_fits(int b, int st, int tb, int m)
{
    return kSelWarps * sel_warp_bytes(b, st, tb, m) + 1024 <= 227 * 1024;
}

// Blocks per tile for a ring of `st` slots: at most kSelTileBytes of data and
// 8 blocks, shrunk until the CTA's rings, masks and stages fit 227 KB.
__host__ __device__ constexpr int sel_tile_blocks_for(int b, int st)
{
    int tb = kSelTileBytes / (128 * b);
    tb = tb < 1 ? 1 : (tb > 8 ? 8 : tb);
    while (tb > 1 && !sel_fits(b, st, tb, 1)) --tb;
    return tb;
}

// Ring depth per warp: three slots where they fit without shrinking the tile
// (a slot is refilled right after its count pass), else two -- larger copies
// measured faster than a deeper ring of smaller ones.
__host__ __device__ constexpr int sel_stages(int b)
{
    return sel_fits(b, 3, 1, 1) && sel_tile_blocks_for(b, 3) >= sel_tile_blocks_for(b, 2) ? 3 : 2;
}

__host__ __device__ constexpr int sel_tile_blocks(int b) { return sel_tile_blocks_for(b, sel_stages(b)); }

// Tiles per warp and iteration: up to 8 blocks in all, as many as the masks'
// shared memory allows (wide widths have small tiles; taking several per
// iteration divides the iterations, and their synchronisation, by as much).
__host__ __device__ constexpr int sel_iter_tiles(int b)
{
    const int st = sel_stages(b);
    const int tb = sel_tile_blocks(b);
    int m = 8 / tb;
    m = m < 1 ? 1 : m;
    while (m > 1 && !sel_fits(b, st, tb, m)) --m;
    return m;
}

template <int B>
struct SelShape {
    static constexpr int kBlockBytes = 128 * B;
    static constexpr int kStages = sel_stages(B);
    static constexpr int kTB = sel_tile_blocks(B);
    static constexpr int kM = sel_iter_tiles(B);
    static constexpr int kIB = kM * kTB;  // blocks per warp and iteration
    static constexpr int kTileBytes = kTB * kBlockBytes;
    static constexpr int kDataBytes = kSelWarps * kStages * kTileBytes;
    static constexpr int kMaskBytes = kSelWarps * (kSelLag + 1) * kIB * 32 * 4;
    static constexpr int kStageBytes = kSelWarps * kSelStageHalfs * 2;
    static constexpr int kSmemBytes = kDataBytes + kMaskBytes + kStageBytes + kSelWarps * kStages * 8;
    static_assert(kSmemBytes + 1024 <= 227 * 1024, "shared-memory budget");
    static_assert(kTileBytes % 16 == 0, "bulk copies move multiples of 16 bytes");
};

// The tagged totals are self-contained (no other data is read on their
// account), so publishing and polling them needs no release/acquire order.
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Code of row r in this lane's b words (row r = stream bits [r*b, r*b + b)).
template <int B>
__device__ __forceinline__ uint32_t sel_code(const uint32_t (&W)[B], int r)
{
    if constexpr (B == 32) {
        return W[r];
    } else {
        const int bit = r * B;
        const int w0 = bit >> 5;
        const int s = bit & 31;
        uint32_t x;
        if (s + B <= 32) {
            x = W[w0] >> s;
        } else {
            const int w1 = (w0 + 1 < B) ? w0 + 1 : w0;
            x = __funnelshift_r(W[w0], W[w1], s);
        }
        return x & ((1u << B) - 1u);
    }
}

// Count pass over one staged block: this lane's column mask (bit r set when
// value 32r + lane matches and lies below `limit`).
template <int B>
__device__ __forceinline__ uint32_t sel_block_mask(const uint32_t* words, int lane, uint32_t lo,
                                                   uint32_t wm1, uint32_t limit)
{
    uint32_t W[B];
#pragma unroll
    for (int w = 0; w < B; ++w) W[w] = words[w * 32 + lane];
    // four interleaved OR chains (rows r = c mod 4), merged at the end, so
    // that no chain of 32 dependent ORs sets the pace
    uint32_t acc[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const uint32_t u = sel_code<B>(W, r);
        asm("{\n\t.reg .pred p;\n\t"
            "setp.le.u32 p, %1, %2;\n\t"
            "@p or.b32 %0, %0, %3;\n\t}"
            : "+r"(acc[r & 3])
            : "r"(u - lo), "r"(wm1), "r"(1u << r));
    }
    uint32_t pm = (acc[0] | acc[1]) | (acc[2] | acc[3]);
    if (limit < 1024u) {  // zero-padded tail block: rows at or past `limit` do not exist
        const uint32_t l = static_cast<uint32_t>(lane);
        const uint32_t rows = limit > l ? (limit - l + 31u) >> 5 : 0u;
        pm &= rows >= 32u ? 0xffffffffu : ((1u << rows) - 1u);
    }
    return pm;
}

// Per-lane constants of the 32 x 32 bit transpose across the warp: stage j
// (16, 8, 4, 2, 1) swaps the off-diagonal j x j sub-blocks.  A lane keeps the
// bits of its own half (`keep`) and takes the partner's other half, rotated
// by j towards it (`rot`).
struct Transpose {
    uint32_t keep[5];
    uint32_t rot[5];
    __device__ __forceinline__ explicit Transpose(int lane)
    {
        const uint32_t low[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            const int j = 16 >> s;
            const bool upper = (lane & j) != 0;
            keep[s] = upper ? ~low[s] : low[s];
            rot[s] = upper ? static_cast<uint32_t>(32 - j) : static_cast<uint32_t>(j);
        }
    }
    // lane l holds column l (bit r = row r); returns row `lane` (bit l = column l)
    __device__ __forceinline__ uint32_t apply(uint32_t x) const
    {
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            const int j = 16 >> s;
            const uint32_t t = __shfl_xor_sync(kFull, x, j);
            const uint32_t y = __funnelshift_l(t, t, rot[s]);
            x = (x & keep[s]) | (y & ~keep[s]);
        }
        return x;
    }
};

// Write pass over one tile.  mk[k*32 + lane] is this lane's column mask of
// block k; the tile's matches go to pos[off ...] in index order (only those
// below `capacity`).  First, for all blocks at once (independent chains, so
// their shuffle latencies overlap): a 32 x 32 bit transpose turns column masks
// into row masks (lane r holds row r, i.e. values 32r..32r+31 in index order)
// and a warp scan of the row counts says where each row's matches start.
// Then per block with a match: lane r writes its row's in-block indices to
// the warp's stage, and the warp copies the stage out with consecutive lanes
// on consecutive positions.
//   branch-free: every row visits its 32 bits with a predicated store;
//   branchy    : every row loops over its set bits only (rows diverge).
template <int TB, bool BRANCHY>
__device__ __forceinline__ uint32_t sel_write_tile(const uint32_t* mk, uint32_t nb, uint32_t blk0, int lane,
                                                  uint32_t off, uint32_t* pos, uint64_t capacity,
                                                  uint16_t* stage, const Transpose& T)
{
    uint32_t rm[TB], incl[TB];
#pragma unroll
    for (int k = 0; k < TB; ++k) {
        const uint32_t pm = static_cast<uint32_t>(k) < nb ? mk[k * 32 + lane] : 0u;
        rm[k] = T.apply(pm);
        incl[k] = static_cast<uint32_t>(__popc(rm[k]));
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int k = 0; k < TB; ++k) {
            const uint32_t v = __shfl_up_sync(kFull, incl[k], o);
            if (lane >= o) incl[k] += v;
        }
    }
#pragma unroll
    for (int k = 0; k < TB; ++k) {
        const uint32_t total = __shfl_sync(kFull, incl[k], 31);
        if (total == 0u) continue;
        uint32_t at = incl[k] - static_cast<uint32_t>(__popc(rm[k]));  // where row `lane` starts
        const uint32_t row0 = 32u * static_cast<uint32_t>(lane);
        if constexpr (BRANCHY) {
            uint32_t m = rm[k];
            while (m) {
                const uint32_t j = static_cast<uint32_t>(__ffs(m) - 1);
                m &= m - 1u;
                stage[at + ((at >> 5) << 1)] = static_cast<uint16_t>(row0 + j);
                ++at;
            }
        } else {
            // four independent chains over the row's bytes, each starting
            // where the matches of the bytes below it end
            const uint32_t r = rm[k];
            uint32_t a[4] = {at, at + static_cast<uint32_t>(__popc(r & 0xffu)),
                             at + static_cast<uint32_t>(__popc(r & 0xffffu)),
                             at + static_cast<uint32_t>(__popc(r & 0xffffffu))};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int bit = 8 * c + j;
                    if ((r >> bit) & 1u) {  // predicated, no branch
                        stage[a[c] + ((a[c] >> 5) << 1)] = static_cast<uint16_t>(row0 + static_cast<uint32_t>(bit));
                        ++a[c];
                    }
                }
            }
        }
        __syncwarp();
        const uint64_t room = capacity > off ? capacity - off : 0u;
        const uint32_t lim = room < total ? static_cast<uint32_t>(room) : total;
        const uint32_t first = (blk0 + static_cast<uint32_t>(k)) * 1024u;
        // copy out 128 positions per step: the four stage loads first, then the stores
        for (uint32_t q0 = 0; q0 < lim; q0 += 128u) {
            uint32_t v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t q = q0 + 32u * u + static_cast<uint32_t>(lane);
                v[u] = q < lim ? stage[q + ((q >> 5) << 1)] : 0u;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t q = q0 + 32u * u + static_cast<uint32_t>(lane);
                if (q < lim) pos[off + q] = first + v[u];
            }
        }
        __syncwarp();
        off += total;
    }
    return off;
}

template <int B, bool BRANCHY>
__global__ void __launch_bounds__(kSelWarps * 32, 1) k_select(const SelectParams p)
{
    using S = SelShape<B>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t cta_cnt[kSelRing][kSelWarps];
    __shared__ uint32_t cta_arrive[kSelRing];
    __shared__ uint32_t grid_tot[kSelRing], grid_before[kSelRing], grid_seq[kSelRing];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* slots = smem + static_cast<size_t>(warp) * S::kStages * S::kTileBytes;
    uint32_t* masks = reinterpret_cast<uint32_t*>(smem + S::kDataBytes) + warp * (kSelLag + 1) * S::kIB * 32;
    uint16_t* stage = reinterpret_cast<uint16_t*>(smem + S::kDataBytes + S::kMaskBytes) + warp * kSelStageHalfs;
    uint64_t* bars =
        reinterpret_cast<uint64_t*>(smem + S::kDataBytes + S::kMaskBytes + S::kStageBytes) + warp * S::kStages;

    const uint64_t nblocks = (p.n + 1023u) >> 10;
    const uint32_t ntiles = static_cast<uint32_t>((nblocks + S::kTB - 1) / S::kTB);
    const uint32_t tail = static_cast<uint32_t>(p.n & 1023u);
    const uint32_t gw = blockIdx.x * kSelWarps + warp;
    const uint32_t GW = gridDim.x * kSelWarps;
    const Transpose T(lane);

    if (threadIdx.x < kSelRing) {
        cta_arrive[threadIdx.x] = 0u;
        grid_seq[threadIdx.x] = 0u;
    }
    if (lane == 0) {
        for (int s = 0; s < S::kStages; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto tile_blocks = [&](uint32_t t) -> uint32_t {
        const uint64_t left = nblocks - static_cast<uint64_t>(t) * S::kTB;
        return left < S::kTB ? static_cast<uint32_t>(left) : static_cast<uint32_t>(S::kTB);
    };
    // q-th tile of this warp: iteration q / M, tile q % M of the warp's run
    // (increasing in q, so once past the last tile every later q is too)
    auto tile_of = [&](uint32_t q) -> uint64_t {
        return (static_cast<uint64_t>(q / S::kM) * GW + gw) * S::kM + q % S::kM;
    };
    auto issue = [&](uint32_t t, int s) {
        const uint32_t bytes = tile_blocks(t) * S::kBlockBytes;
        mbar_arrive_expect_tx(&bars[s], bytes);
        bulk_g2s(slots + s * S::kTileBytes, p.packed + static_cast<uint64_t>(t) * S::kTB * 32u * B, bytes,
                 &bars[s]);
    };
    if (lane == 0) {
        for (int s = 0; s < S::kStages; ++s) {
            const uint64_t t = tile_of(static_cast<uint32_t>(s));
            if (t < ntiles) issue(static_cast<uint32_t>(t), s);
        }
    }
    __syncwarp();

    uint32_t base = 0;      // matches in all iterations before the one being written
    uint32_t consumed = 0;  // tiles this warp has counted (data ring position)
    bool failed = false;
    // Every CTA's total for the iteration written next.  One warp of the CTA
    // (a different one each iteration) reads them and shares the sums through
    // shared memory; its loads are issued before the count pass so that their
    // latency hides behind it.
    constexpr int kPer = 8;  // up to 256 CTAs
    unsigned long long v[kPer];
#pragma unroll 1
    for (uint32_t i = 0; i < p.niter + kSelLag; ++i) {
        if (i >= kSelLag && (i - kSelLag) % kSelWarps == static_cast<uint32_t>(warp)) {
            const unsigned long long* row = p.agg + static_cast<uint64_t>(i - kSelLag) * gridDim.x;
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const uint32_t c = static_cast<uint32_t>(lane) + 32u * q;
                v[q] = c < gridDim.x ? ld_relaxed(row + c) : (static_cast<unsigned long long>(p.epoch) << 32);
            }
        }
        // ---------------------------------------------------- count pass (i)
        if (i < p.niter) {
            uint32_t cnt = 0;
            uint32_t* mk = masks + (i % (kSelLag + 1)) * S::kIB * 32;
#pragma unroll 1
            for (uint32_t m = 0; m < static_cast<uint32_t>(S::kM); ++m) {
                const uint64_t t = tile_of(i * S::kM + m);
                if (t >= ntiles) break;
                const int s = static_cast<int>(consumed % S::kStages);
                const uint32_t parity = (consumed / S::kStages) & 1u;
                const bool ok = mbar_wait(&bars[s], parity, p.wait_limit_ns);
                if (!__all_sync(kFull, ok)) {
                    failed = true;
                    break;
                }
                const uint32_t nb = tile_blocks(static_cast<uint32_t>(t));
                const uint32_t* tw = reinterpret_cast<const uint32_t*>(slots + s * S::kTileBytes);
#pragma unroll 1
                for (uint32_t k = 0; k < nb; ++k) {
                    const uint64_t blk = t * S::kTB + k;
                    const uint32_t limit = (tail && blk == nblocks - 1) ? tail : 1024u;
                    const uint32_t pm = sel_block_mask<B>(tw + k * 32u * B, lane, p.lo, p.wm1, limit);
                    mk[(m * S::kTB + k) * 32 + lane] = pm;
                    cnt += static_cast<uint32_t>(__popc(pm));
                }
                __syncwarp();
                const uint64_t tn = tile_of(consumed + S::kStages);
                ++consumed;
                if (lane == 0 && tn < ntiles) {
                    fence_proxy_async_smem();
                    issue(static_cast<uint32_t>(tn), s);
                }
            }
            if (failed) break;
#pragma unroll
            for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
            if (lane == 0) {
                volatile uint32_t* cc = cta_cnt[i % kSelRing];
                cc[warp] = cnt;
                __threadfence_block();
                const uint32_t old = atomicAdd(&cta_arrive[i % kSelRing], 1u);
                if (old == kSelWarps * (i / kSelRing) + (kSelWarps - 1)) {  // last warp of the CTA for i
                    __threadfence_block();
                    uint32_t sum = 0;
                    for (int w = 0; w < kSelWarps; ++w) sum += cc[w];
                    if (static_cast<int32_t>(blockIdx.x) != p.silent_cta)
                        st_relaxed(&p.agg[static_cast<uint64_t>(i) * gridDim.x + blockIdx.x],
                                   (static_cast<unsigned long long>(p.epoch) << 32) | sum);
                }
            }
            __syncwarp();
        }
        // ----------------------------------------- write pass (i - kSelLag)
        if (i >= kSelLag) {
            const uint32_t wi = i - kSelLag;
            const uint32_t slot = wi % kSelRing;
            bool ok = true;
            if (wi % kSelWarps == static_cast<uint32_t>(warp)) {
                // this warp polls: re-read the totals not yet published when
                // prefetched, backing off so that waiting CTAs do not flood L2
                const unsigned long long* row = p.agg + static_cast<uint64_t>(wi) * gridDim.x;
#pragma unroll
                for (int q = 0; q < kPer; ++q) {
                    const uint32_t c = static_cast<uint32_t>(lane) + 32u * q;
                    if (static_cast<uint32_t>(v[q] >> 32) != p.epoch) {
                        const uint64_t t0 = global_ns();
                        uint32_t nap = 64;
                        do {
                            if (global_ns() - t0 > p.wait_limit_ns) {
                                ok = false;
                                break;
                            }
                            __nanosleep(nap);
                            nap = nap < 1024u ? nap * 2u : nap;
                            v[q] = ld_relaxed(row + c);
                        } while (static_cast<uint32_t>(v[q] >> 32) != p.epoch);
                    }
                }
                uint32_t tot = 0, before = 0;
#pragma unroll
                for (int q = 0; q < kPer; ++q) {
                    const uint32_t c = static_cast<uint32_t>(lane) + 32u * q;
                    const uint32_t a = c < gridDim.x ? static_cast<uint32_t>(v[q]) : 0u;
                    tot += a;
                    before += c < blockIdx.x ? a : 0u;
                }
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    tot += __shfl_xor_sync(kFull, tot, o);
                    before += __shfl_xor_sync(kFull, before, o);
                }
                // Our own CTA's total for wi is among those seen, so every warp
                // of the CTA has stored its count for wi.
                __syncwarp();
                if (lane == 0) {
                    volatile uint32_t* gt = grid_tot;
                    volatile uint32_t* gb = grid_before;
                    gt[slot] = tot;
                    gb[slot] = before;
                    __threadfence_block();
                    *reinterpret_cast<volatile uint32_t*>(&grid_seq[slot]) = ok ? wi + 1u : ~0u;
                }
                __syncwarp();
            }
            // every warp: wait for the polling warp's sums of iteration wi
            {
                const volatile uint32_t* seq = grid_seq;
                uint32_t got = seq[slot];
                if (got != wi + 1u && got != ~0u) {
                    const uint64_t t0 = global_ns();
                    do {
                        if (global_ns() - t0 > p.wait_limit_ns) {
                            ok = false;
                            break;
                        }
                        __nanosleep(64);
                        got = seq[slot];
                    } while (got != wi + 1u && got != ~0u);
                }
                if (got == ~0u) ok = false;
            }
            if (!__all_sync(kFull, ok)) {
                failed = true;
                break;
            }
            // the CTA-scope fence orders the reads of the shared sums and of
            // the CTA's warp counts after the polling warp's publication
            __threadfence_block();
            const uint32_t tot = *reinterpret_cast<volatile uint32_t*>(&grid_tot[slot]);
            const uint32_t before = *reinterpret_cast<volatile uint32_t*>(&grid_before[slot]);
            const volatile uint32_t* cc = cta_cnt[wi % kSelRing];
            uint32_t off = base + before;
            for (int w = 0; w < warp; ++w) off += cc[w];
            const uint64_t blk0 = tile_of(wi * S::kM) * S::kTB;  // the iteration's blocks are consecutive
            // a warp with no match in the iteration skips the transposes and scans
            if (cc[warp] != 0u && blk0 < nblocks && off < p.capacity) {
                const uint32_t* mk = masks + (wi % (kSelLag + 1)) * S::kIB * 32;
                const uint64_t left = nblocks - blk0;
                const uint32_t nb = left < S::kIB ? static_cast<uint32_t>(left) : static_cast<uint32_t>(S::kIB);
                sel_write_tile<S::kIB, BRANCHY>(mk, nb, static_cast<uint32_t>(blk0), lane, off, p.pos, p.capacity,
                                                stage, T);
            }
            base += tot;
        }
    }
    if (failed) {
        if (lane == 0) atomicOr(p.status, kSelSelectErr);
        // Let this warp's copies still in flight land before shared memory
        // goes away: ring positions consumed .. consumed + stages - 1 that name a tile.
        for (uint32_t j = 0; j < static_cast<uint32_t>(S::kStages); ++j) {
            const uint32_t jt = consumed + j;
            if (tile_of(jt) >= ntiles) break;
            mbar_wait(&bars[jt % S::kStages], (jt / S::kStages) & 1u, kDrainLimitNs);
        }
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *p.count = base;
}

}  // namespace gb
