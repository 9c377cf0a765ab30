// Fused columnar-scan kernels, templated on the bit width B (1..32).
//
// Paper §3: 1024-value blocks transposed over 32 lanes so that every lane
// extracts its values with the same shifts and masks.  On the GPU a block is
// B rows of 32 words (128*B contiguous bytes); row w holds word w of every
// lane.  Eight threads cover one block: thread q of the group owns lanes
// 4q..4q+3 and reads one 16-byte vector per row, so a warp works on four
// blocks at once and every shared-memory read is conflict-free.
//
// Data movement is the GB300 part: each warp runs its own pipeline of
// kStages shared-memory slots, filled by the bulk TMA engine
// (cp.async.bulk + mbarrier transaction counts), so ~100 KB per SM stay in
// flight without holding registers.  The full scan walks tiles in a static
// persistent order; the zone-skip scan pops candidate blocks from a device
// queue (one atomic per tile).  Per-thread partials are reduced by warp
// shuffles, then per CTA, then by the last CTA to finish (no second launch).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "gb_ptx.cuh"

namespace gb {

enum : uint32_t { kErrTimeout = 1u, kErrRange = 2u };
enum : uint32_t { kFlagAgg = 1u };

struct ScanParams {
    const uint32_t* packed;       // lane-interleaved words, 16-byte aligned
    uint64_t n;                   // number of values
    uint32_t base;                // frame-of-reference base
    uint32_t lo;                  // predicate lower bound in code space
    uint32_t wm1;                 // predicate width minus one (width >= 1)
    uint32_t flags;               // kFlagAgg: answer wholly-inside blocks from their metadata
    uint64_t zlo, zhi;            // predicate [zlo, zhi) on decoded values, for zone tests
    const uint2* zonemap;         // (min, max) of decoded values per block
    uint2* zonemap_out;           // zone-map build output
    unsigned long long* blocksum; // sum of decoded values per block (written by the build)
    unsigned long long* partials; // 2 words per CTA
    unsigned int* done;           // grid-finish ticket, reset by the last CTA
    unsigned int* status;         // error bits (kErr*)
    unsigned int* cand;           // zone-skip candidate block ids
    unsigned long long* qctl;     // [0] candidates, [1] queue head, [2] tail kept,
                                  // [3] count and [4] code sum of wholly-inside blocks
    long long* result;            // count, sum, blocks_scanned, reserved
    uint32_t tile_blocks;         // pipeline shape: blocks per tile (a multiple of the warp step)
    uint32_t stages;              // and slots per warp; warps per CTA = blockDim.x / 32
};

// Launch shape for width B: warps per CTA, pipeline depth, blocks per tile.
template <int B>
struct Shape;

// ------------------------------------------------------------- geometry
// Threads per block: a thread owns LPT consecutive lanes and reads them as one
// vector per row; a warp step covers LPT blocks.  By default 4 lanes (16 bytes
// per row) for b <= 16 and 2 (8 bytes) above, where four blocks per warp step
// would not fit an 8 KB slot.  The 2-lane geometry at b = 9..16 is a tuned
// variant: its smaller warp step lets 16 warps fit in shared memory there.
__host__ __device__ constexpr int default_lpt(int b) { return b <= 16 ? 4 : 2; }

template <int B, int LPT = default_lpt(B)>
struct Geo {
    static_assert(LPT == 2 || LPT == 4, "2 or 4 lanes per thread");
    static constexpr int kLpt = LPT;
    static constexpr int kTpb = 32 / kLpt;
    using Vec = typename std::conditional<kLpt == 4, uint4, uint2>::type;
};

// Default launch shape for width B (used until a tuned shape is installed):
// 8 warps per CTA, each with kStages slots of up to 8 KB; a tile is the
// largest multiple of the warp step (kLpt blocks) that fits a slot, and at
// most 16 blocks: below b = 4 a full slot would hold 32-64 K values (~10-20 us
// of decode per warp), too coarse to share a column's work evenly among the
// warps.  The kernels take the shape at run time (ScanParams::tile_blocks,
// ::stages and the block size), so the autotuner can replace it per width.
template <int B>
struct Shape {
    static constexpr int kWarps = 8;
    static constexpr int kStages = 3;
    static constexpr int kBlockBytes = 128 * B;
    static constexpr int kSlotMax = 8 * 1024;
    static constexpr int kStep = Geo<B>::kLpt;
    static constexpr int kTbRaw = (kSlotMax / kBlockBytes) / kStep * kStep;
    static constexpr int kTB = kTbRaw < kStep ? kStep : (kTbRaw > 16 ? 16 : kTbRaw);
    static constexpr int kTileBytes = kTB * kBlockBytes;
    static constexpr int kSlotBytes = kWarps * kStages * kTileBytes;
    static constexpr int kSmemBytes = kSlotBytes + kWarps * kStages * 8 + kWarps * kStages * 4;
    static_assert(kSmemBytes <= 227 * 1024, "shared-memory budget");
    static_assert(kTileBytes % 16 == 0, "bulk copies move multiples of 16 bytes");
};

// Shared memory of a runtime-shaped pipeline: every warp owns `stages` slots of
// tile_blocks * 128 * B bytes; then the slots' transaction barriers (8 bytes
// each) and, for the queue kernel, the blocks held per slot (4 bytes each).
// The dynamic part may take 226 KB: 1 KB of the 227 KB a CTA can use stays
// for the kernels' static shared memory (the grid reduction's array).
constexpr int kSmemMax = 226 * 1024;
__host__ __device__ constexpr uint32_t pipe_smem_bytes(uint32_t b, uint32_t warps, uint32_t stages,
                                                       uint32_t tile_blocks)
{
    return warps * stages * (tile_blocks * 128u * b + 8u + 4u);
}

struct Pipe {
    unsigned char* slots;  // this warp's first slot
    uint64_t* bars;        // this warp's barriers
    uint32_t* slot_n;      // this warp's per-slot block counts
    uint32_t tile_bytes;   // bytes of a full tile
    uint32_t stages;
    uint32_t tb;           // blocks per full tile
};

template <int B>
__device__ __forceinline__ Pipe pipe_of(unsigned char* smem, const ScanParams& p, int warp, int nwarps)
{
    Pipe q;
    q.tb = p.tile_blocks;
    q.stages = p.stages;
    q.tile_bytes = q.tb * 128u * B;
    const size_t slot_area = static_cast<size_t>(nwarps) * q.stages * q.tile_bytes;
    q.slots = smem + static_cast<size_t>(warp) * q.stages * q.tile_bytes;
    q.bars = reinterpret_cast<uint64_t*>(smem + slot_area) + warp * q.stages;
    q.slot_n = reinterpret_cast<uint32_t*>(smem + slot_area + static_cast<size_t>(nwarps) * q.stages * 8u) +
               warp * q.stages;
    return q;
}

// ------------------------------------------------------------- extraction
__device__ __forceinline__ uint32_t lane_word(const uint4& v, int k)
{
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}
__device__ __forceinline__ uint32_t lane_word(const uint2& v, int k) { return k == 0 ? v.x : v.y; }

// Code of row r for the thread's lane k (r, k compile-time after unrolling).
template <int B, int LPT = default_lpt(B)>
__device__ __forceinline__ uint32_t code_of(const typename Geo<B, LPT>::Vec (&W)[B], int r, int k)
{
    const int bit = r * B;
    const int w0 = bit >> 5;
    const int s = bit & 31;
    const uint32_t lw = lane_word(W[w0], k);
    if constexpr (B == 32) {
        return lw;
    } else {
        constexpr uint32_t kMask = (1u << B) - 1u;
        if (s + B <= 32) return (lw >> s) & kMask;
        const int w1 = (w0 + 1 < B) ? w0 + 1 : w0;
        return __funnelshift_r(lw, lane_word(W[w1], k), s) & kMask;
    }
}

template <int B, int LPT = default_lpt(B)>
__device__ __forceinline__ void load_rows(typename Geo<B, LPT>::Vec (&W)[B], const typename Geo<B, LPT>::Vec* rows)
{
#pragma unroll
    for (int w = 0; w < B; ++w) W[w] = rows[w * Geo<B, LPT>::kTpb];
}

// -------------------------------------------------------------- aggregate
// Per value the decode needs an extraction, a range test and one add.  The
// integer ALU pipe and the FMA-heavy pipe (IMAD) each retire 16 lanes per
// cycle on this SM (the ncu pipe counters of the b = 8 scan: 2 cycles per warp
// instruction on both), so the decode spreads its work over both: extraction
// (shift, funnel shift, LOP3 mask) and one ISETP per value stay on the ALU;
// the subtract of the range test and the accumulation are IMADs by an opaque
// 1 (%nctaid.z, which the compiler cannot fold), and a field at the top of its
// word is extracted by IMAD.HI by 2^B with the added constant folded in.
struct Lanes {
    uint32_t one;     // 1, opaque to the compiler
    uint32_t pow2b;   // 2^B (B < 32)
    uint32_t add;     // constant added to every extracted code (packed count bit)
    uint32_t mask;    // 2^B - 1
    uint32_t loi;     // lo' + add
    uint32_t hii;     // hi' + add (B < 32)
    uint32_t negloi;  // -(lo' + add)
    uint32_t wm1;     // hi' - lo' - 1
};

__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ uint32_t opaque_one()
{
    uint32_t v;
    asm("mov.u32 %0, %%nctaid.z;" : "=r"(v));
    return v;
}

template <int B>
__device__ __forceinline__ Lanes make_lanes(uint32_t lo, uint32_t wm1)
{
    Lanes L;
    L.one = opaque_one();
    L.pow2b = B < 32 ? (L.one << (B & 31)) : 0u;
    L.add = B <= 21 ? (1u << ((B + 5) & 31)) : 0u;
    L.mask = B < 32 ? ((1u << (B & 31)) - 1u) : 0xffffffffu;
    L.loi = lo + L.add;
    L.hii = lo + wm1 + 1u + L.add;  // only used for B < 32, where it cannot wrap
    L.negloi = 0u - L.loi;
    L.wm1 = wm1;
    return L;
}

// True when row r's field sits at the top of its word (extracted by IMAD.HI).
template <int B>
__device__ __forceinline__ bool top_field(int r)
{
    const int s = (r * B) & 31;
    return B < 32 && s != 0 && s + B == 32;
}

// Code of row r, lane k, plus L.add (r, k compile-time after unrolling).
template <int B, int LPT = default_lpt(B)>
__device__ __forceinline__ uint32_t field_add(const typename Geo<B, LPT>::Vec (&W)[B], int r, int k,
                                              const Lanes& L)
{
    const int bit = r * B;
    const int w0 = bit >> 5;
    const int s = bit & 31;
    const uint32_t lw = lane_word(W[w0], k);
    if constexpr (B == 32) {
        return lw;
    } else {
        uint32_t v;
        if (top_field<B>(r)) {  // hi32(w * 2^B) + add = (w >> s) + add
            asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(v) : "r"(lw), "r"(L.pow2b), "r"(L.add));
            return v;
        }
        uint32_t x;
        if (s + B <= 32) {
            x = lw >> s;
        } else {
            const int w1 = (w0 + 1 < B) ? w0 + 1 : w0;
            x = __funnelshift_r(lw, lane_word(W[w1], k), s);
        }
        asm("lop3.b32 %0, %1, %2, %3, 0xEA;" : "=r"(v) : "r"(x), "r"(L.mask), "r"(L.add));  // (x & mask) | add
        return v;
    }
}

// Mode 1 (32-bit sums plus a count): for a field in the middle of its word
// or straddling two words the extraction already costs two ALU operations;
// every other such value moves its subtraction to the FMA pipe (one compare
// left on the ALU).
template <int B>
__device__ __forceinline__ bool sub_on_fma(int r, int k)
{
    const int s = (r * B) & 31;
    return B < 32 && s != 0 && !top_field<B>(r) && ((r + k) & 1) != 0;
}

__device__ __forceinline__ void acc0_fma(uint32_t& a, uint32_t ui, const Lanes& L)
{
    asm("{\n\t.reg .pred p;\n\t.reg .b32 t;\n\t"
        "mad.lo.u32 t, %1, %4, %2;\n\t"
        "setp.le.u32 p, t, %3;\n\t"
        "@p mad.lo.u32 %0, %1, %4, %0;\n\t}"
        : "+r"(a) : "r"(ui), "r"(L.negloi), "r"(L.wm1), "r"(L.one));
}
__device__ __forceinline__ void acc1_fma(uint32_t& c, uint32_t& a, uint32_t ui, const Lanes& L)
{
    asm("{\n\t.reg .pred p;\n\t.reg .b32 t;\n\t"
        "mad.lo.u32 t, %2, %5, %3;\n\t"
        "setp.le.u32 p, t, %4;\n\t"
        "@p add.u32 %0, %0, 1;\n\t"
        "@p mad.lo.u32 %1, %2, %5, %1;\n\t}"
        : "+r"(c), "+r"(a) : "r"(ui), "r"(L.negloi), "r"(L.wm1), "r"(L.one));
}

// packed accumulator: a += v + add when lo <= v < hi (compares on the ALU)
__device__ __forceinline__ void acc0_imad(uint32_t& a, uint32_t ui, const Lanes& L)
{
    asm("{\n\t.reg .pred p;\n\t"
        "setp.ge.u32 p, %1, %2;\n\t"
        "setp.lt.and.u32 p, %1, %3, p;\n\t"
        "@p mad.lo.u32 %0, %1, %4, %0;\n\t}"
        : "+r"(a) : "r"(ui), "r"(L.loi), "r"(L.hii), "r"(L.one));
}
// subtract on the FMA pipe, compare and add on the ALU (a top-of-word field,
// whose extraction was already an IMAD)
__device__ __forceinline__ void acc0_fsub(uint32_t& a, uint32_t ui, const Lanes& L)
{
    asm("{\n\t.reg .pred p;\n\t.reg .b32 t;\n\t"
        "mad.lo.u32 t, %1, %4, %2;\n\t"
        "setp.le.u32 p, t, %3;\n\t"
        "@p add.u32 %0, %0, %1;\n\t}"
        : "+r"(a) : "r"(ui), "r"(L.negloi), "r"(L.wm1), "r"(L.one));
}
__device__ __forceinline__ void acc0_alu(uint32_t& a, uint32_t ui, const Lanes& L)
{
    asm("{\n\t.reg .pred p;\n\t"
        "setp.ge.u32 p, %1, %2;\n\t"
        "setp.lt.and.u32 p, %1, %3, p;\n\t"
        "@p add.u32 %0, %0, %1;\n\t}"
        : "+r"(a) : "r"(ui), "r"(L.loi), "r"(L.hii));
}
// 32-bit sum + count
__device__ __forceinline__ void acc1_imad(uint32_t& c, uint32_t& a, uint32_t ui, const Lanes& L)
{
    asm("{\n\t.reg .pred p;\n\t"
        "setp.ge.u32 p, %2, %3;\n\t"
        "setp.lt.and.u32 p, %2, %4, p;\n\t"
        "@p add.u32 %0, %0, 1;\n\t"
        "@p mad.lo.u32 %1, %2, %5, %1;\n\t}"
        : "+r"(c), "+r"(a) : "r"(ui), "r"(L.loi), "r"(L.hii), "r"(L.one));
}
__device__ __forceinline__ void acc1_alu(uint32_t& c, uint32_t& a, uint32_t ui, const Lanes& L)
{
    asm("{\n\t.reg .pred p;\n\t"
        "setp.ge.u32 p, %2, %3;\n\t"
        "setp.lt.and.u32 p, %2, %4, p;\n\t"
        "@p add.u32 %0, %0, 1;\n\t"
        "@p add.u32 %1, %1, %2;\n\t}"
        : "+r"(c), "+r"(a) : "r"(ui), "r"(L.loi), "r"(L.hii));
}

// 64-bit accumulation on the FMA pipe: s += u (IMAD.WIDE by an opaque 1).
__device__ __forceinline__ uint64_t imad_wide(uint32_t u, uint32_t one, uint64_t s)
{
    uint64_t d;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(u), "r"(one), "l"(s));
    return d;
}

// Mode 2 (64-bit sums): the compare stays on the ALU; the subtract (unless
// `alu_sub`), the count and the 64-bit add are IMADs on the FMA pipe.
template <bool ALU_SUB>
__device__ __forceinline__ void acc2(uint32_t& c, uint64_t& s, uint32_t ui, const Lanes& L)
{
    if constexpr (ALU_SUB)
        asm("{\n\t.reg .pred p;\n\t.reg .b32 t;\n\t"
            "sub.u32 t, %2, %3;\n\t"
            "setp.le.u32 p, t, %4;\n\t"
            "@p mad.lo.u32 %0, %5, %5, %0;\n\t"
            "@p mad.wide.u32 %1, %2, %5, %1;\n\t}"
            : "+r"(c), "+l"(s) : "r"(ui), "r"(L.loi), "r"(L.wm1), "r"(L.one));
    else
        asm("{\n\t.reg .pred p;\n\t.reg .b32 t;\n\t"
            "mad.lo.u32 t, %2, %5, %3;\n\t"
            "setp.le.u32 p, t, %4;\n\t"
            "@p mad.lo.u32 %0, %5, %5, %0;\n\t"
            "@p mad.wide.u32 %1, %2, %5, %1;\n\t}"
            : "+r"(c), "+l"(s) : "r"(ui), "r"(L.negloi), "r"(L.wm1), "r"(L.one));
}

// One branchy row of mode 0 (packed accumulators) as a single PTX block: the
// thread's kLpt tests t = u - lo' <= w - 1 (subtract on the FMA pipe unless
// the field was extracted there, TOP), OR-ed into one predicate, one warp vote,
// and a uniform branch that skips the kLpt predicated adds when no lane of the
// warp matches anywhere in the row.
template <bool TOP, int LPT>
__device__ __forceinline__ void branchy_row(uint32_t (&a)[LPT], const uint32_t (&u)[LPT], const Lanes& L);

template <>
__device__ __forceinline__ void branchy_row<true, 4>(uint32_t (&a)[4], const uint32_t (&u)[4], const Lanes& L)
{
    asm volatile(
        "{\n\t.reg .pred p0, p1, p2, p3, q;\n\t.reg .b32 t0, t1, t2, t3;\n\t"
        "sub.u32 t0, %4, %8;\n\tsub.u32 t1, %5, %8;\n\tsub.u32 t2, %6, %8;\n\tsub.u32 t3, %7, %8;\n\t"
        "setp.le.u32 p0, t0, %9;\n\tsetp.le.u32 p1, t1, %9;\n\t"
        "setp.le.u32 p2, t2, %9;\n\tsetp.le.u32 p3, t3, %9;\n\t"
        "or.pred q, p0, p1;\n\tor.pred q, q, p2;\n\tor.pred q, q, p3;\n\t"
        "vote.sync.any.pred q, q, 0xffffffff;\n\t"
        "@!q bra.uni BR_SKIP;\n\t"
        "@p0 add.u32 %0, %0, %4;\n\t@p1 add.u32 %1, %1, %5;\n\t"
        "@p2 add.u32 %2, %2, %6;\n\t@p3 add.u32 %3, %3, %7;\n\t"
        "BR_SKIP:\n\t}"
        : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3])
        : "r"(u[0]), "r"(u[1]), "r"(u[2]), "r"(u[3]), "r"(L.loi), "r"(L.wm1));
}
template <>
__device__ __forceinline__ void branchy_row<false, 4>(uint32_t (&a)[4], const uint32_t (&u)[4], const Lanes& L)
{
    asm volatile(
        "{\n\t.reg .pred p0, p1, p2, p3, q;\n\t.reg .b32 t0, t1, t2, t3;\n\t"
        "mad.lo.u32 t0, %4, %10, %8;\n\tmad.lo.u32 t1, %5, %10, %8;\n\t"
        "mad.lo.u32 t2, %6, %10, %8;\n\tmad.lo.u32 t3, %7, %10, %8;\n\t"
        "setp.le.u32 p0, t0, %9;\n\tsetp.le.u32 p1, t1, %9;\n\t"
        "setp.le.u32 p2, t2, %9;\n\tsetp.le.u32 p3, t3, %9;\n\t"
        "or.pred q, p0, p1;\n\tor.pred q, q, p2;\n\tor.pred q, q, p3;\n\t"
        "vote.sync.any.pred q, q, 0xffffffff;\n\t"
        "@!q bra.uni BR_SKIP;\n\t"
        "@p0 mad.lo.u32 %0, %4, %10, %0;\n\t@p1 mad.lo.u32 %1, %5, %10, %1;\n\t"
        "@p2 mad.lo.u32 %2, %6, %10, %2;\n\t@p3 mad.lo.u32 %3, %7, %10, %3;\n\t"
        "BR_SKIP:\n\t}"
        : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3])
        : "r"(u[0]), "r"(u[1]), "r"(u[2]), "r"(u[3]), "r"(L.negloi), "r"(L.wm1), "r"(L.one));
}
template <>
__device__ __forceinline__ void branchy_row<true, 2>(uint32_t (&a)[2], const uint32_t (&u)[2], const Lanes& L)
{
    asm volatile(
        "{\n\t.reg .pred p0, p1, q;\n\t.reg .b32 t0, t1;\n\t"
        "sub.u32 t0, %2, %4;\n\tsub.u32 t1, %3, %4;\n\t"
        "setp.le.u32 p0, t0, %5;\n\tsetp.le.u32 p1, t1, %5;\n\t"
        "or.pred q, p0, p1;\n\t"
        "vote.sync.any.pred q, q, 0xffffffff;\n\t"
        "@!q bra.uni BR_SKIP;\n\t"
        "@p0 add.u32 %0, %0, %2;\n\t@p1 add.u32 %1, %1, %3;\n\t"
        "BR_SKIP:\n\t}"
        : "+r"(a[0]), "+r"(a[1])
        : "r"(u[0]), "r"(u[1]), "r"(L.loi), "r"(L.wm1));
}
template <>
__device__ __forceinline__ void branchy_row<false, 2>(uint32_t (&a)[2], const uint32_t (&u)[2], const Lanes& L)
{
    asm volatile(
        "{\n\t.reg .pred p0, p1, q;\n\t.reg .b32 t0, t1;\n\t"
        "mad.lo.u32 t0, %2, %6, %4;\n\tmad.lo.u32 t1, %3, %6, %4;\n\t"
        "setp.le.u32 p0, t0, %5;\n\tsetp.le.u32 p1, t1, %5;\n\t"
        "or.pred q, p0, p1;\n\t"
        "vote.sync.any.pred q, q, 0xffffffff;\n\t"
        "@!q bra.uni BR_SKIP;\n\t"
        "@p0 mad.lo.u32 %0, %2, %6, %0;\n\t@p1 mad.lo.u32 %1, %3, %6, %1;\n\t"
        "BR_SKIP:\n\t}"
        : "+r"(a[0]), "+r"(a[1])
        : "r"(u[0]), "r"(u[1]), "r"(L.negloi), "r"(L.wm1), "r"(L.one));
}

// Two branchy rows of mode 0 as one PTX block (ROWVOTE = 3): both rows' tests
// and both votes come before the first branch, so the scheduler has 2 * kLpt
// independent tests and two votes in one basic block; then, per row, a uniform
// branch around its predicated adds.  Operands: %0.. the kLpt accumulators,
// then the row-A codes, the row-B codes, lo', -lo', w - 1, an opaque 1.
#define GB_BR_SUB_ALU(t, u, LOI, NLOI, ONE) "sub.u32 " t ", " u ", " LOI ";\n\t"
#define GB_BR_SUB_FMA(t, u, LOI, NLOI, ONE) "mad.lo.u32 " t ", " u ", " ONE ", " NLOI ";\n\t"
#define GB_BR_ADD_ALU(p, a, u, ONE) "@" p " add.u32 " a ", " a ", " u ";\n\t"
#define GB_BR_ADD_FMA(p, a, u, ONE) "@" p " mad.lo.u32 " a ", " u ", " ONE ", " a ";\n\t"
#define GB_BR_TWO_ROWS4(SUBA, ADDA, SUBB, ADDB)                                                           \
    asm volatile("{\n\t.reg .pred pa0, pa1, pa2, pa3, pb0, pb1, pb2, pb3, qa, qb;\n\t"                     \
                 ".reg .b32 ta0, ta1, ta2, ta3, tb0, tb1, tb2, tb3;\n\t"                                  \
                 SUBA("ta0", "%4", "%12", "%13", "%15") SUBA("ta1", "%5", "%12", "%13", "%15")            \
                 SUBA("ta2", "%6", "%12", "%13", "%15") SUBA("ta3", "%7", "%12", "%13", "%15")            \
                 SUBB("tb0", "%8", "%12", "%13", "%15") SUBB("tb1", "%9", "%12", "%13", "%15")            \
                 SUBB("tb2", "%10", "%12", "%13", "%15") SUBB("tb3", "%11", "%12", "%13", "%15")          \
                 "setp.le.u32 pa0, ta0, %14;\n\tsetp.le.u32 pa1, ta1, %14;\n\t"                           \
                 "setp.le.u32 pa2, ta2, %14;\n\tsetp.le.u32 pa3, ta3, %14;\n\t"                           \
                 "setp.le.u32 pb0, tb0, %14;\n\tsetp.le.u32 pb1, tb1, %14;\n\t"                           \
                 "setp.le.u32 pb2, tb2, %14;\n\tsetp.le.u32 pb3, tb3, %14;\n\t"                           \
                 "or.pred qa, pa0, pa1;\n\tor.pred qa, qa, pa2;\n\tor.pred qa, qa, pa3;\n\t"              \
                 "or.pred qb, pb0, pb1;\n\tor.pred qb, qb, pb2;\n\tor.pred qb, qb, pb3;\n\t"              \
                 "vote.sync.any.pred qa, qa, 0xffffffff;\n\tvote.sync.any.pred qb, qb, 0xffffffff;\n\t"  \
                 "@!qa bra.uni BR_SKIP_A;\n\t"                                                            \
                 ADDA("pa0", "%0", "%4", "%15") ADDA("pa1", "%1", "%5", "%15")                            \
                 ADDA("pa2", "%2", "%6", "%15") ADDA("pa3", "%3", "%7", "%15")                            \
                 "BR_SKIP_A:\n\t@!qb bra.uni BR_SKIP_B;\n\t"                                              \
                 ADDB("pb0", "%0", "%8", "%15") ADDB("pb1", "%1", "%9", "%15")                            \
                 ADDB("pb2", "%2", "%10", "%15") ADDB("pb3", "%3", "%11", "%15")                          \
                 "BR_SKIP_B:\n\t}"                                                                        \
                 : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3])                                         \
                 : "r"(ua[0]), "r"(ua[1]), "r"(ua[2]), "r"(ua[3]), "r"(ub[0]), "r"(ub[1]), "r"(ub[2]),   \
                   "r"(ub[3]), "r"(L.loi), "r"(L.negloi), "r"(L.wm1), "r"(L.one))
#define GB_BR_TWO_ROWS2(SUBA, ADDA, SUBB, ADDB)                                                           \
    asm volatile("{\n\t.reg .pred pa0, pa1, pb0, pb1, qa, qb;\n\t.reg .b32 ta0, ta1, tb0, tb1;\n\t"       \
                 SUBA("ta0", "%2", "%6", "%7", "%9") SUBA("ta1", "%3", "%6", "%7", "%9")                  \
                 SUBB("tb0", "%4", "%6", "%7", "%9") SUBB("tb1", "%5", "%6", "%7", "%9")                  \
                 "setp.le.u32 pa0, ta0, %8;\n\tsetp.le.u32 pa1, ta1, %8;\n\t"                             \
                 "setp.le.u32 pb0, tb0, %8;\n\tsetp.le.u32 pb1, tb1, %8;\n\t"                             \
                 "or.pred qa, pa0, pa1;\n\tor.pred qb, pb0, pb1;\n\t"                                     \
                 "vote.sync.any.pred qa, qa, 0xffffffff;\n\tvote.sync.any.pred qb, qb, 0xffffffff;\n\t"  \
                 "@!qa bra.uni BR_SKIP_A;\n\t"                                                            \
                 ADDA("pa0", "%0", "%2", "%9") ADDA("pa1", "%1", "%3", "%9")                              \
                 "BR_SKIP_A:\n\t@!qb bra.uni BR_SKIP_B;\n\t"                                              \
                 ADDB("pb0", "%0", "%4", "%9") ADDB("pb1", "%1", "%5", "%9")                              \
                 "BR_SKIP_B:\n\t}"                                                                        \
                 : "+r"(a[0]), "+r"(a[1])                                                                 \
                 : "r"(ua[0]), "r"(ua[1]), "r"(ub[0]), "r"(ub[1]), "r"(L.loi), "r"(L.negloi), "r"(L.wm1), \
                   "r"(L.one))

// TOPA / TOPB: the row's fields sit at the top of their words (extracted on
// the FMA pipe), so its subtract and add go to the ALU.
template <bool TOPA, bool TOPB, int LPT>
__device__ __forceinline__ void branchy_two_rows(uint32_t (&a)[LPT], const uint32_t (&ua)[LPT],
                                                 const uint32_t (&ub)[LPT], const Lanes& L)
{
    if constexpr (LPT == 4) {
        if constexpr (TOPA && TOPB) GB_BR_TWO_ROWS4(GB_BR_SUB_ALU, GB_BR_ADD_ALU, GB_BR_SUB_ALU, GB_BR_ADD_ALU);
        else if constexpr (TOPA) GB_BR_TWO_ROWS4(GB_BR_SUB_ALU, GB_BR_ADD_ALU, GB_BR_SUB_FMA, GB_BR_ADD_FMA);
        else if constexpr (TOPB) GB_BR_TWO_ROWS4(GB_BR_SUB_FMA, GB_BR_ADD_FMA, GB_BR_SUB_ALU, GB_BR_ADD_ALU);
        else GB_BR_TWO_ROWS4(GB_BR_SUB_FMA, GB_BR_ADD_FMA, GB_BR_SUB_FMA, GB_BR_ADD_FMA);
    } else {
        static_assert(LPT == 2, "two-row blocks are written for 2 or 4 lanes per thread");
        if constexpr (TOPA && TOPB) GB_BR_TWO_ROWS2(GB_BR_SUB_ALU, GB_BR_ADD_ALU, GB_BR_SUB_ALU, GB_BR_ADD_ALU);
        else if constexpr (TOPA) GB_BR_TWO_ROWS2(GB_BR_SUB_ALU, GB_BR_ADD_ALU, GB_BR_SUB_FMA, GB_BR_ADD_FMA);
        else if constexpr (TOPB) GB_BR_TWO_ROWS2(GB_BR_SUB_FMA, GB_BR_ADD_FMA, GB_BR_SUB_ALU, GB_BR_ADD_ALU);
        else GB_BR_TWO_ROWS2(GB_BR_SUB_FMA, GB_BR_ADD_FMA, GB_BR_SUB_FMA, GB_BR_ADD_FMA);
    }
}

// One block, this thread's 4 lanes x 32 rows, every value valid.
// Accumulators stay 32-bit inside the block:
//   B <= 21: one word per lane packs (count << (B+5)) + sum  (mode 0);
//   B <= 27: a 32-bit sum per lane plus a count              (mode 1);
//   else   : a 64-bit sum plus a count                       (mode 2).
// BRANCHY adds a warp vote and skips the aggregation when no value of the
// voting group matches.  The group is one value per thread (32 values) by
// default (ROWVOTE = 0); with ROWVOTE = 1 or 2 it is a whole row of the
// thread's kLpt lanes (32 * kLpt values over kLpt blocks): one vote per kLpt
// values, but all kLpt tests must be held across the vote.  ROWVOTE = 2 writes
// the row as one PTX block (branchy_row): tests combined by or.pred, one
// vote.sync.any, one uniform branch around the predicated adds.  Which form is
// faster depends on the width and on how many warps share an SM (the
// autotuner picks per width).
template <int B, bool BRANCHY, int ROWVOTE = 0, int LPT = default_lpt(B)>
__device__ __forceinline__ void agg_block(const typename Geo<B, LPT>::Vec* rows, const Lanes& L,
                                          uint64_t& cnt, uint64_t& sum)
{
    constexpr int kMode = B <= 21 ? 0 : (B <= 27 ? 1 : 2);
    constexpr int kLpt = LPT;
    typename Geo<B, LPT>::Vec W[B];
    load_rows<B, LPT>(W, rows);
    uint32_t a[kLpt] = {};
    uint32_t c = 0u;
    uint64_t s64 = 0u;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        if constexpr (BRANCHY && ROWVOTE == 3) {
            static_assert(kMode == 0 && (kLpt == 2 || kLpt == 4), "the PTX row vote is written for mode 0");
            if ((r & 1) == 0) {  // rows r and r + 1 (32 rows: always a pair)
                uint32_t ua[kLpt], ub[kLpt];
#pragma unroll
                for (int k = 0; k < kLpt; ++k) {
                    ua[k] = field_add<B, LPT>(W, r, k, L);
                    ub[k] = field_add<B, LPT>(W, r + 1, k, L);
                }
                const bool ta = top_field<B>(r), tb = top_field<B>(r + 1);  // folded after unrolling
                if (ta && tb) branchy_two_rows<true, true, kLpt>(a, ua, ub, L);
                else if (ta) branchy_two_rows<true, false, kLpt>(a, ua, ub, L);
                else if (tb) branchy_two_rows<false, true, kLpt>(a, ua, ub, L);
                else branchy_two_rows<false, false, kLpt>(a, ua, ub, L);
            }
        } else if constexpr (BRANCHY && ROWVOTE == 2) {
            static_assert(kMode == 0 && (kLpt == 2 || kLpt == 4), "the PTX row vote is written for mode 0");
            uint32_t ui[kLpt];
#pragma unroll
            for (int k = 0; k < kLpt; ++k) ui[k] = field_add<B, LPT>(W, r, k, L);
            if (top_field<B>(r)) branchy_row<true, kLpt>(a, ui, L);  // folded after unrolling
            else branchy_row<false, kLpt>(a, ui, L);
        } else if constexpr (BRANCHY && ROWVOTE == 1) {
            // subtract on the FMA pipe unless the extraction already used it
            const bool top = top_field<B>(r);
            uint32_t ui[kLpt];
            bool m[kLpt];
            bool any = false;
#pragma unroll
            for (int k = 0; k < kLpt; ++k) {
                ui[k] = field_add<B, LPT>(W, r, k, L);
                const uint32_t t = top ? ui[k] - L.loi : imad(ui[k], L.one, L.negloi);
                m[k] = t <= L.wm1;
                any = any || m[k];
            }
            if (__any_sync(kFull, any)) {
#pragma unroll
                for (int k = 0; k < kLpt; ++k) {
                    if (m[k]) {
                        if constexpr (kMode != 0) c = imad(L.one, L.one, c);
                        if constexpr (kMode == 2) s64 = imad_wide(ui[k], L.one, s64);
                        else a[k] = top ? a[k] + ui[k] : imad(ui[k], L.one, a[k]);
                    }
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < kLpt; ++k) {
                const uint32_t ui = field_add<B, LPT>(W, r, k, L);
                if constexpr (BRANCHY) {
                    // subtract and add on the FMA pipe unless the extraction already used it
                    const bool top = top_field<B>(r);
                    const uint32_t t = top ? ui - L.loi : imad(ui, L.one, L.negloi);
                    const bool m = t <= L.wm1;
                    if (__any_sync(kFull, m)) {  // vote.any: the predicate directly, no compare
                        if (m) {
                            if constexpr (kMode != 0) c += 1u;
                            if constexpr (kMode == 2) s64 += ui;
                            else a[k] = top ? a[k] + ui : imad(ui, L.one, a[k]);
                        }
                    }
                } else if constexpr (kMode == 0) {
                    // Every compare keeps one ISETP on the ALU; the subtract and the
                    // add go to the FMA pipe, except that half the top-of-word
                    // fields (already extracted by IMAD.HI) add on the ALU: about
                    // 2.9 ALU and 2.0 IMAD per value (2.4 / 2.1 at b = 8).
                    if (top_field<B>(r) && ((r + k) & 1) == 0) acc0_fsub(a[k], ui, L);
                    else acc0_fma(a[k], ui, L);
                } else if constexpr (kMode == 1) {
                    if (top_field<B>(r)) acc1_alu(c, a[k], ui, L);
                    else if (sub_on_fma<B>(r, k)) acc1_fma(c, a[k], ui, L);
                    else acc1_imad(c, a[k], ui, L);
                } else if constexpr (B < 32) {
                    // 64-bit sums: count and sum on the FMA pipe (IMAD.WIDE); a
                    // top-of-word field (extracted by IMAD.HI) subtracts on the
                    // ALU.  At b = 28..31 this ran 1.5-6% faster than ALU adds.
                    if (top_field<B>(r)) acc2<true>(c, s64, ui, L);
                    else acc2<false>(c, s64, ui, L);
                } else {
                    // b = 32 (no extraction): plain compare and ALU adds, 2% faster
                    // than the FMA form above
                    if ((ui - L.loi) <= L.wm1) {
                        c += 1u;
                        s64 += ui;
                    }
                }
            }
        }
    }
    if constexpr (kMode == 0) {
        constexpr int kSB = (B + 5) & 31;
        constexpr uint32_t kSumMask = (1u << kSB) - 1u;
#pragma unroll
        for (int k = 0; k < kLpt; ++k) {
            cnt += a[k] >> kSB;
            sum += a[k] & kSumMask;
        }
    } else if constexpr (kMode == 1) {
        cnt += c;
#pragma unroll
        for (int k = 0; k < kLpt; ++k) sum += a[k];
    } else {
        cnt += c;
        sum += s64;
    }
}

// Same with a validity mask: value (r, lane kLpt*q + k) counts iff `ok` and
// its index in the block, 32r + kLpt*q + k, is below `limit`.  Used for the
// last partial warp step of a tile and for the zero-padded tail block.
template <int B, int LPT = default_lpt(B)>
__device__ __forceinline__ void agg_block_masked(const typename Geo<B, LPT>::Vec* rows, uint32_t lo,
                                                 uint32_t wm1, uint64_t& cnt, uint64_t& sum, bool ok,
                                                 uint32_t limit, int q)
{
    constexpr int kLpt = LPT;
    typename Geo<B, LPT>::Vec W[B];
    load_rows<B, LPT>(W, rows);
    uint32_t c = 0u;
    uint64_t s = 0u;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
#pragma unroll
        for (int k = 0; k < kLpt; ++k) {
            const uint32_t u = code_of<B, LPT>(W, r, k);
            const uint32_t j = 32u * r + static_cast<uint32_t>(kLpt * q + k);
            if (ok && j < limit && (u - lo) <= wm1) {
                c += 1u;
                s += u;
            }
        }
    }
    cnt += c;
    sum += s;
}

// (min, max) and sum of the codes of one block over valid positions.
template <int B>
__device__ __forceinline__ void minmax_block(const typename Geo<B>::Vec* rows, uint32_t limit, int q,
                                             uint32_t& mn, uint32_t& mx, uint64_t& sm)
{
    constexpr int kLpt = Geo<B>::kLpt;
    typename Geo<B>::Vec W[B];
    load_rows<B>(W, rows);
#pragma unroll
    for (int r = 0; r < 32; ++r) {
#pragma unroll
        for (int k = 0; k < kLpt; ++k) {
            const uint32_t u = code_of<B>(W, r, k);
            const uint32_t j = 32u * r + static_cast<uint32_t>(kLpt * q + k);
            if (j < limit) {
                mn = min(mn, u);
                mx = max(mx, u);
                sm += u;
            }
        }
    }
}

template <int B, int LPT = default_lpt(B)>
__device__ __forceinline__ const typename Geo<B, LPT>::Vec* block_rows(const unsigned char* blk, int q)
{
    return reinterpret_cast<const typename Geo<B, LPT>::Vec*>(blk) + q;
}

// ------------------------------------------- the other layouts (§3 i, iii)
// A column's 1024-value blocks occupy the same 128*b bytes in every layout;
// only the order of the codes inside a block differs:
//   kLayLanes : lane-interleaved (strategy ii, everything above);
//   kLayRow   : row-major bit stream, value j of the block at bits
//               [j*b, j*b + b) of the block's 32*b words (strategy i);
//   kLayBytes : b in {8, 16}: the codes as a plain uint8/uint16 array
//               (strategy iii; b = 32 is the lane layout byte for byte).
// The staging pipeline is shared; these consumers put all 32 lanes on one
// block at a time, 32 codes per lane, with the accumulators of agg_block.
enum Layout : int { kLayLanes = 0, kLayRow = 1, kLayBytes = 2 };

template <int B, bool BRANCHY>
__device__ __forceinline__ void acc_one(uint32_t ui, const Lanes& L, uint32_t& a, uint32_t& c, uint64_t& s64)
{
    constexpr int kMode = B <= 21 ? 0 : (B <= 27 ? 1 : 2);
    if constexpr (BRANCHY) {
        const uint32_t t = imad(ui, L.one, L.negloi);
        const bool m = t <= L.wm1;
        if (__any_sync(kFull, m)) {
            if (m) {
                if constexpr (kMode != 0) c += 1u;
                if constexpr (kMode == 2) s64 += ui;
                else a = imad(ui, L.one, a);
            }
        }
    } else if constexpr (kMode == 0) {
        acc0_fma(a, ui, L);  // subtract and add on the FMA pipe, one ISETP on the ALU
    } else if constexpr (kMode == 1) {
        acc1_imad(c, a, ui, L);
    } else {
        if ((ui - L.loi) <= L.wm1) {
            c += 1u;
            s64 += ui;
        }
    }
}

// Fold one lane's 32 codes of accumulation into the 64-bit totals.
template <int B>
__device__ __forceinline__ void acc_flush(uint32_t a, uint32_t c, uint64_t s64, uint64_t& cnt, uint64_t& sum)
{
    constexpr int kMode = B <= 21 ? 0 : (B <= 27 ? 1 : 2);
    if constexpr (kMode == 0) {
        constexpr int kSB = (B + 5) & 31;
        cnt += a >> kSB;
        sum += a & ((1u << kSB) - 1u);
    } else if constexpr (kMode == 1) {
        cnt += c;
        sum += a;
    } else {
        cnt += c;
        sum += s64;
    }
}

// Row-major block: lane l takes values j = l + 32m (m = 0..31), whose bits
// start at l*B + 32*B*m: the word offset grows by B per m (an immediate) and
// the shift (l*B) mod 32 is fixed per lane -- a variable-shift extractor, one
// funnel shift over a two-word window per value.  The high word of the
// block's last value lies one word past the block; it is read from shared
// memory (the slot's neighbour) and contributes no bits.
template <int B, bool BRANCHY>
__device__ __forceinline__ void agg_block_row(const uint32_t* words, int lane, const Lanes& L, uint64_t& cnt,
                                              uint64_t& sum)
{
    const uint32_t bit0 = static_cast<uint32_t>(lane) * B;
    const uint32_t* w = words + (bit0 >> 5);
    const uint32_t sh = bit0 & 31u;
    uint32_t a = 0u, c = 0u;
    uint64_t s64 = 0u;
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        uint32_t ui;
        if constexpr (B == 32) {
            ui = w[32 * m];
        } else {
            const uint32_t x = __funnelshift_r(w[B * m], w[B * m + 1], sh);
            asm("lop3.b32 %0, %1, %2, %3, 0xEA;" : "=r"(ui) : "r"(x), "r"(L.mask), "r"(L.add));  // (x & mask) | add
        }
        acc_one<B, BRANCHY>(ui, L, a, c, s64);
    }
    acc_flush<B>(a, c, s64, cnt, sum);
}

// Byte-aligned block (B = 8 or 16): lane l reads the 16-byte chunks l and
// l + 32 (B = 8) or l + 32h, h < 4 (B = 16); one byte permute per value
// takes the code and ORs in the packed-count bit of L.add at once.
template <int B, bool BRANCHY>
__device__ __forceinline__ void agg_block_bytes(const unsigned char* blk, int lane, const Lanes& L,
                                                uint64_t& cnt, uint64_t& sum)
{
    static_assert(B == 8 || B == 16, "byte-aligned widths are 8 and 16 (32 is the lane layout)");
    const uint4* q4 = reinterpret_cast<const uint4*>(blk);
    uint32_t a = 0u, c = 0u;
    uint64_t s64 = 0u;
#pragma unroll
    for (int h = 0; h < B / 4; ++h) {
        const uint4 q = q4[lane + 32 * h];
        const uint32_t x[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
#pragma unroll
            for (int k = 0; k < 32 / B; ++k) {
                // B = 8 : bytes (x.k, add.1, add.0, add.0); add = 1 << 13 -> its byte 1 is 0x20
                // B = 16: bytes (x.2k, x.2k+1, add.2, add.0); add = 1 << 21 -> its byte 2 is 0x20
                constexpr unsigned kSel8 = 0x4450u;
                constexpr unsigned kSel16 = 0x4600u;
                const unsigned sel = B == 8 ? kSel8 + static_cast<unsigned>(k)
                                            : kSel16 + static_cast<unsigned>(2 * k) +
                                                  (static_cast<unsigned>(2 * k + 1) << 4);
                const uint32_t ui = __byte_perm(x[e], L.add, sel);
                acc_one<B, BRANCHY>(ui, L, a, c, s64);
            }
        }
    }
    acc_flush<B>(a, c, s64, cnt, sum);
}

// All `nb` blocks of a staged tile in a non-lane layout.
template <int B, bool BRANCHY, int LAY>
__device__ __forceinline__ void scan_tile_layout(const unsigned char* tile, uint32_t nb, int lane, const Lanes& L,
                                                 uint64_t& cnt, uint64_t& sum)
{
    constexpr uint32_t kBB = 128u * B;
#pragma unroll 1
    for (uint32_t g = 0; g < nb; ++g) {
        if constexpr (LAY == kLayRow) {
            agg_block_row<B, BRANCHY>(reinterpret_cast<const uint32_t*>(tile + g * kBB), lane, L, cnt, sum);
        } else if constexpr (LAY == kLayBytes && (B == 8 || B == 16)) {
            agg_block_bytes<B, BRANCHY>(tile + g * kBB, lane, L, cnt, sum);
        }
    }
}

// Tail block (n mod 1024 values) of a non-lane layout, from global memory.
template <int B, int LAY>
__device__ __forceinline__ void scan_tail_layout(const ScanParams& p, int lane, uint64_t& cnt, uint64_t& sum)
{
    const uint32_t* blk = p.packed + (p.n >> 10) * 32u * B;
    const uint32_t rem = static_cast<uint32_t>(p.n & 1023u);
    uint32_t c = 0u;
    uint64_t s = 0u;
    for (uint32_t j = static_cast<uint32_t>(lane); j < rem; j += 32u) {
        uint32_t u;
        if constexpr (LAY == kLayBytes && B == 8) {
            u = reinterpret_cast<const uint8_t*>(blk)[j];
        } else if constexpr (LAY == kLayBytes && B == 16) {
            u = reinterpret_cast<const uint16_t*>(blk)[j];
        } else if constexpr (B == 32) {
            u = blk[j];
        } else {
            const uint32_t bit = j * B;
            const uint32_t w = bit >> 5, sh = bit & 31u;
            const uint32_t hi = sh + B > 32u ? blk[w + 1] : 0u;  // within the block when the value straddles
            u = __funnelshift_r(blk[w], hi, sh) & ((1u << B) - 1u);
        }
        if ((u - p.lo) <= p.wm1) {
            c += 1u;
            s += u;
        }
    }
    cnt += c;
    sum += s;
}

// All `nb` blocks of a staged tile (blocks are contiguous in the slot).
template <int B, bool BRANCHY, int ROWVOTE = 0, int LPT = default_lpt(B)>
__device__ __forceinline__ void scan_tile(const unsigned char* tile, uint32_t nb, int lane,
                                          const Lanes& L, uint32_t lo, uint32_t wm1, uint64_t& cnt,
                                          uint64_t& sum)
{
    constexpr uint32_t kBB = 128u * B;
    constexpr uint32_t kStep = Geo<B, LPT>::kLpt;          // blocks per warp step
    const int q = lane % Geo<B, LPT>::kTpb;
    const uint32_t sub = static_cast<uint32_t>(lane / Geo<B, LPT>::kTpb);
    uint32_t g = 0;
#pragma unroll 1
    for (; g + kStep <= nb; g += kStep)
        agg_block<B, BRANCHY, ROWVOTE, LPT>(block_rows<B, LPT>(tile + (g + sub) * kBB, q), L, cnt, sum);
    if (g < nb) {
        const bool ok = g + sub < nb;
        agg_block_masked<B, LPT>(block_rows<B, LPT>(tile + (ok ? g + sub : g) * kBB, q), lo, wm1, cnt, sum, ok,
                            1024u, q);
    }
}

// --------------------------------------------------------- grid reduction
// Sum (count, sum) over the grid: warp shuffles, one word pair per CTA, and
// the last CTA to arrive folds the pairs, applies the frame of reference
// (SUM_v = SUM_u + base*COUNT) and resets the ticket for the next launch.
// WMAX bounds the CTA's warps (blockDim.x / 32 at run time).
template <int WMAX>
__device__ __forceinline__ void grid_finish(const ScanParams& p, uint64_t cnt, uint64_t sum,
                                            bool queue_mode, uint64_t full_blocks_scanned)
{
    __shared__ unsigned long long red[WMAX][2];
    __shared__ int is_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int WARPS = static_cast<int>(blockDim.x >> 5);
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        cnt += __shfl_xor_sync(kFull, cnt, o);
        sum += __shfl_xor_sync(kFull, sum, o);
    }
    if (lane == 0) {
        red[warp][0] = cnt;
        red[warp][1] = sum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long c = 0, s = 0;
        for (int w = 0; w < WARPS; ++w) {
            c += red[w][0];
            s += red[w][1];
        }
        p.partials[2 * blockIdx.x] = c;
        p.partials[2 * blockIdx.x + 1] = s;
        __threadfence();
        const unsigned t = atomicAdd(p.done, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    unsigned long long c = 0, s = 0;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
        c += __ldcg(&p.partials[2 * i]);
        s += __ldcg(&p.partials[2 * i + 1]);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        c += __shfl_xor_sync(kFull, c, o);
        s += __shfl_xor_sync(kFull, s, o);
    }
    __syncthreads();
    if (lane == 0) {
        red[warp][0] = c;
        red[warp][1] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tc = 0, ts = 0;
        for (int w = 0; w < WARPS; ++w) {
            tc += red[w][0];
            ts += red[w][1];
        }
        unsigned long long blocks = full_blocks_scanned;
        if (queue_mode) {
            blocks = __ldcg(&p.qctl[0]) + __ldcg(&p.qctl[2]);
            tc += __ldcg(&p.qctl[3]);  // wholly-inside blocks answered from metadata
            ts += __ldcg(&p.qctl[4]);
            p.qctl[0] = 0ull;
            p.qctl[1] = 0ull;
            p.qctl[2] = 0ull;
            p.qctl[3] = 0ull;
            p.qctl[4] = 0ull;
        }
        p.result[0] = static_cast<long long>(tc);
        p.result[1] = static_cast<long long>(ts + static_cast<unsigned long long>(p.base) * tc);
        p.result[2] = static_cast<long long>(blocks);
        p.result[3] = 0;
        __threadfence();
        *p.done = 0u;
    }
}

// Tail block (n mod 1024 values, zero padded) read straight from global memory.
template <int B, int LPT = default_lpt(B)>
__device__ __forceinline__ void scan_tail(const ScanParams& p, int lane, uint64_t& cnt,
                                          uint64_t& sum)
{
    const uint64_t tb = p.n >> 10;
    const uint32_t rem = static_cast<uint32_t>(p.n & 1023u);
    const int q = lane % Geo<B, LPT>::kTpb;
    const bool ok = lane < Geo<B, LPT>::kTpb;
    const auto* rows = block_rows<B, LPT>(reinterpret_cast<const unsigned char*>(p.packed + tb * 32u * B), q);
    agg_block_masked<B, LPT>(rows, p.lo, p.wm1, cnt, sum, ok, rem, q);
}

// ------------------------------------------------------------- full scan
// The static persistent walk over every full block: tile t of the column goes
// to warp t mod (all warps), numbered warp-major, through the warp's ring of
// slots.  Returns false when a bounded wait gave up (the warp's copies in
// flight have landed by then and the status bit is set).
template <int B, bool BRANCHY, int LAY, int ROWVOTE, int LPT = default_lpt(B)>
__device__ __forceinline__ bool walk_static(const ScanParams& p, const Pipe& P, int warp, int lane, int nwarps,
                                            uint64_t& cnt, uint64_t& sum)
{
    const uint64_t full_blocks = p.n >> 10;
    const uint64_t ntiles = (full_blocks + P.tb - 1) / P.tb;
    // Warp-major numbering: a round's last, partial stretch of tiles goes to
    // warp slot w of every CTA before slot w + 1 of any, so the CTAs (SMs) of
    // a small column get equal shares (CTA-major numbering gave the first
    // CTAs two tiles per warp and the rest one at 2^24 values, b = 8).
    const uint64_t gw = static_cast<uint64_t>(warp) * gridDim.x + blockIdx.x;
    const uint64_t GW = static_cast<uint64_t>(gridDim.x) * nwarps;

    auto issue = [&](uint64_t t, uint32_t s) {
        const uint64_t fb = t * P.tb;
        const uint64_t left = full_blocks - fb;
        const uint32_t nb = left < P.tb ? static_cast<uint32_t>(left) : P.tb;
        const uint32_t bytes = nb * (128u * B);
        mbar_arrive_expect_tx(&P.bars[s], bytes);
        bulk_g2s(P.slots + s * P.tile_bytes, p.packed + fb * 32u * B, bytes, &P.bars[s]);
    };
    if (lane == 0) {
        for (uint32_t s = 0; s < P.stages; ++s) {
            const uint64_t t = gw + s * GW;
            if (t < ntiles) issue(t, s);
        }
    }

    const Lanes L = make_lanes<B>(p.lo, p.wm1);
    uint32_t it = 0, s = 0, parity = 0;
    bool failed = false;
#pragma unroll 1
    for (uint64_t t = gw; t < ntiles; t += GW, ++it) {
        const bool ok = mbar_wait(&P.bars[s], parity, kWaitLimitNs);
        if (!__all_sync(kFull, ok)) {
            failed = true;
            break;
        }
        const uint64_t left = full_blocks - t * P.tb;
        const uint32_t nb = left < P.tb ? static_cast<uint32_t>(left) : P.tb;
        if constexpr (LAY == kLayLanes)
            scan_tile<B, BRANCHY, ROWVOTE, LPT>(P.slots + s * P.tile_bytes, nb, lane, L, p.lo, p.wm1, cnt, sum);
        else
            scan_tile_layout<B, BRANCHY, LAY>(P.slots + s * P.tile_bytes, nb, lane, L, cnt, sum);
        __syncwarp();
        const uint64_t tn = t + static_cast<uint64_t>(P.stages) * GW;
        if (lane == 0 && tn < ntiles) {
            fence_proxy_async_smem();
            issue(tn, s);
        }
        if (++s == P.stages) {
            s = 0;
            parity ^= 1u;
        }
    }
    if (failed) {
        if (lane == 0) atomicOr(p.status, kErrTimeout);
        // let copies still in flight land before the CTA's shared memory goes away
        for (uint32_t j = 0; j < P.stages; ++j) {
            const uint64_t t = gw + static_cast<uint64_t>(it + j) * GW;
            if (t >= ntiles) break;
            const uint32_t jt = it + j;
            mbar_wait(&P.bars[jt % P.stages], (jt / P.stages) & 1u, kDrainLimitNs);
        }
    }
    return !failed;
}

// WMAX: the largest CTA the instantiation is compiled for (launch bound; 8
// warps leave up to 255 registers per thread, 16 warps 128).  ROWVOTE: the
// branchy vote group (see agg_block).  LPT: lanes per thread (see Geo).
template <int B, bool BRANCHY, int LAY = kLayLanes, int WMAX = 8, int ROWVOTE = 0, int LPT = default_lpt(B)>
__global__ void __launch_bounds__(WMAX * 32, 1) k_scan_full(const ScanParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = static_cast<int>(blockDim.x >> 5);
    const Pipe P = pipe_of<B>(smem, p, warp, nwarps);
    if (lane == 0) {
        for (uint32_t s = 0; s < P.stages; ++s) mbar_init(&P.bars[s], 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint64_t cnt = 0, sum = 0;
    walk_static<B, BRANCHY, LAY, ROWVOTE, LPT>(p, P, warp, lane, nwarps, cnt, sum);
    const uint64_t gw = static_cast<uint64_t>(warp) * gridDim.x + blockIdx.x;
    if ((p.n & 1023u) && gw == static_cast<uint64_t>(gridDim.x) * nwarps - 1) {
        if constexpr (LAY == kLayLanes)
            scan_tail<B, LPT>(p, lane, cnt, sum);
        else
            scan_tail_layout<B, LAY>(p, lane, cnt, sum);
    }
    grid_finish<WMAX>(p, cnt, sum, false, (p.n + 1023u) >> 10);
}

// -------------------------------------------------------- zone-map build
template <int B>
__global__ void __launch_bounds__(Shape<B>::kWarps * 32, 1) k_zonemap_build(const ScanParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = static_cast<int>(blockDim.x >> 5);
    const int q = lane % Geo<B>::kTpb;
    const uint32_t sub = static_cast<uint32_t>(lane / Geo<B>::kTpb);
    const Pipe P = pipe_of<B>(smem, p, warp, nwarps);

    const uint64_t full_blocks = p.n >> 10;
    const uint64_t ntiles = (full_blocks + P.tb - 1) / P.tb;
    const uint64_t gw = static_cast<uint64_t>(blockIdx.x) * nwarps + warp;
    const uint64_t GW = static_cast<uint64_t>(gridDim.x) * nwarps;

    if (lane == 0) {
        for (uint32_t s = 0; s < P.stages; ++s) mbar_init(&P.bars[s], 1);
        fence_mbar_init();
    }
    __syncwarp();
    auto issue = [&](uint64_t t, uint32_t s) {
        const uint64_t fb = t * P.tb;
        const uint64_t left = full_blocks - fb;
        const uint32_t nb = left < P.tb ? static_cast<uint32_t>(left) : P.tb;
        const uint32_t bytes = nb * (128u * B);
        mbar_arrive_expect_tx(&P.bars[s], bytes);
        bulk_g2s(P.slots + s * P.tile_bytes, p.packed + fb * 32u * B, bytes, &P.bars[s]);
    };
    if (lane == 0) {
        for (uint32_t s = 0; s < P.stages; ++s) {
            const uint64_t t = gw + s * GW;
            if (t < ntiles) issue(t, s);
        }
    }
    auto emit = [&](uint64_t blk, bool ok, uint32_t mn, uint32_t mx, uint64_t sm, uint32_t valid) {
#pragma unroll
        for (int o = 1; o < Geo<B>::kTpb; o <<= 1) {
            mn = min(mn, __shfl_xor_sync(kFull, mn, o));
            mx = max(mx, __shfl_xor_sync(kFull, mx, o));
            sm += __shfl_xor_sync(kFull, sm, o);
        }
        if (ok && q == 0) {
            p.zonemap_out[blk] = make_uint2(mn + p.base, mx + p.base);
            p.blocksum[blk] = sm + static_cast<unsigned long long>(p.base) * valid;
        }
    };
    uint32_t it = 0, s = 0, parity = 0;
    bool failed = false;
#pragma unroll 1
    for (uint64_t t = gw; t < ntiles; t += GW, ++it) {
        const bool okw = mbar_wait(&P.bars[s], parity, kWaitLimitNs);
        if (!__all_sync(kFull, okw)) {
            failed = true;
            break;
        }
        const uint64_t fb = t * P.tb;
        const uint64_t left = full_blocks - fb;
        const uint32_t nb = left < P.tb ? static_cast<uint32_t>(left) : P.tb;
        const unsigned char* tile = P.slots + s * P.tile_bytes;
#pragma unroll 1
        for (uint32_t g = 0; g < nb; g += static_cast<uint32_t>(Geo<B>::kLpt)) {
            const bool ok = g + sub < nb;
            uint32_t mn = 0xffffffffu, mx = 0u;
            uint64_t sm = 0u;
            minmax_block<B>(block_rows<B>(tile + (ok ? g + sub : g) * (128u * B), q), 1024u, q, mn, mx, sm);
            emit(fb + g + sub, ok, mn, mx, sm, 1024u);
        }
        __syncwarp();
        const uint64_t tn = t + static_cast<uint64_t>(P.stages) * GW;
        if (lane == 0 && tn < ntiles) {
            fence_proxy_async_smem();
            issue(tn, s);
        }
        if (++s == P.stages) {
            s = 0;
            parity ^= 1u;
        }
    }
    if (failed) {
        if (lane == 0) atomicOr(p.status, kErrTimeout);
        for (uint32_t j = 0; j < P.stages; ++j) {
            const uint64_t t = gw + static_cast<uint64_t>(it + j) * GW;
            if (t >= ntiles) break;
            const uint32_t jt = it + j;
            mbar_wait(&P.bars[jt % P.stages], (jt / P.stages) & 1u, kDrainLimitNs);
        }
    }
    if ((p.n & 1023u) && gw == GW - 1) {
        const uint32_t rem = static_cast<uint32_t>(p.n & 1023u);
        const auto* rows =
            block_rows<B>(reinterpret_cast<const unsigned char*>(p.packed + full_blocks * 32u * B), q);
        uint32_t mn = 0xffffffffu, mx = 0u;
        uint64_t sm = 0u;
        minmax_block<B>(rows, sub == 0 ? rem : 0u, q, mn, mx, sm);
        emit(full_blocks, sub == 0, mn, mx, sm, rem);
    }
}

// ----------------------------------------------------- zone-map filtering
constexpr int kFilterThreads = 256;
constexpr int kFilterPerCta = 2048;
// k_zone_filter (not templated) is defined once, in the host library unit.
__global__ void k_zone_filter(const ScanParams p);

// ------------------------------------------------------- zone-skip scan
// The candidate list (the surviving blocks' ids, in order) is cut into tiles
// of tile_blocks (<= 32) ids; tile t goes to warp t mod (all warps), numbered
// warp-major as in the full scan, so the GPU reads the survivors in one
// front sweeping up the column and every warp gets the same number of
// blocks.  A tile's ids are loaded one iteration ahead (overlapping the decode
// of the current slot); consecutive ids are merged into single bulk copies.
// An earlier form popped tiles from an atomic counter: with one tile per pop,
// a column whose 2^20 blocks all survived spent more time in pops on the one
// counter (~1.75 ns each) than in reading; with eight tiles per pop the warps
// read scattered 64 KB runs and the scan ran 13% slower than the full scan.
template <int B, bool BRANCHY>
__global__ void __launch_bounds__(Shape<B>::kWarps * 32, 1) k_scan_queue(const ScanParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = static_cast<int>(blockDim.x >> 5);
    const Pipe P = pipe_of<B>(smem, p, warp, nwarps);

    const uint64_t ncand = __ldcg(&p.qctl[0]);
    const uint64_t ntiles = (ncand + P.tb - 1) / P.tb;
    const uint64_t gw = static_cast<uint64_t>(warp) * gridDim.x + blockIdx.x;
    const uint64_t GW = static_cast<uint64_t>(gridDim.x) * nwarps;
    if (lane == 0) {
        for (uint32_t s = 0; s < P.stages; ++s) mbar_init(&P.bars[s], 1);
        fence_mbar_init();
    }
    __syncwarp();

    // Tile t of the candidate list: its block count and this lane's id.
    auto ids_of = [&](uint64_t t, uint32_t& id) -> uint32_t {
        const uint64_t first = t * P.tb;
        const uint64_t left = ncand - first;
        const uint32_t nb = left < P.tb ? static_cast<uint32_t>(left) : P.tb;
        id = static_cast<uint32_t>(lane) < nb ? __ldcg(&p.cand[first + lane]) : 0u;
        return nb;
    };
    // Stage a tile into slot s (one bulk copy per run of consecutive ids).
    auto stage = [&](uint32_t nb, uint32_t id, uint32_t s) {
        if (lane == 0) mbar_arrive_expect_tx(&P.bars[s], nb * (128u * B));
        __syncwarp();
        fence_proxy_async_smem();
        unsigned char* dst = P.slots + s * P.tile_bytes;
        const bool valid = static_cast<uint32_t>(lane) < nb;
        const uint32_t prev = __shfl_up_sync(kFull, id, 1);
        const bool head = valid && (lane == 0 || prev + 1u != id);
        const uint32_t heads = __ballot_sync(kFull, head);
        const uint32_t vmask = __ballot_sync(kFull, valid);
        if (head) {
            const uint32_t later = heads & ~((2u << lane) - 1u);
            const uint32_t end = later ? static_cast<uint32_t>(__ffs(later) - 1)
                                       : static_cast<uint32_t>(32 - __clz(vmask));
            const uint32_t len = end - static_cast<uint32_t>(lane);
            bulk_g2s(dst + lane * (128u * B), p.packed + static_cast<uint64_t>(id) * 32u * B, len * (128u * B),
                     &P.bars[s]);
        }
    };

    for (uint32_t s = 0; s < P.stages; ++s) {
        const uint64_t t = gw + s * GW;
        if (t >= ntiles) break;
        uint32_t id;
        const uint32_t nb = ids_of(t, id);
        stage(nb, id, s);
    }
    // the ids of the tile that refills the current slot, loaded one iteration ahead
    uint64_t tn = gw + static_cast<uint64_t>(P.stages) * GW;
    uint32_t next_id = 0;
    uint32_t next_nb = tn < ntiles ? ids_of(tn, next_id) : 0u;

    const Lanes L = make_lanes<B>(p.lo, p.wm1);
    uint64_t cnt = 0, sum = 0;
    uint32_t it = 0, s = 0, parity = 0;
    bool failed = false;
#pragma unroll 1
    for (uint64_t t = gw; t < ntiles; t += GW, ++it) {
        const bool ok = mbar_wait(&P.bars[s], parity, kWaitLimitNs);
        if (!__all_sync(kFull, ok)) {
            failed = true;
            break;
        }
        const uint64_t left = ncand - t * P.tb;
        const uint32_t nb = left < P.tb ? static_cast<uint32_t>(left) : P.tb;
        scan_tile<B, BRANCHY>(P.slots + s * P.tile_bytes, nb, lane, L, p.lo, p.wm1, cnt, sum);
        __syncwarp();
        if (next_nb) stage(next_nb, next_id, s);
        tn += GW;
        next_nb = tn < ntiles ? ids_of(tn, next_id) : 0u;
        if (++s == P.stages) {
            s = 0;
            parity ^= 1u;
        }
    }
    if (failed) {
        if (lane == 0) atomicOr(p.status, kErrTimeout);
        // let copies still in flight land before the CTA's shared memory goes away
        for (uint32_t j = 0; j < P.stages; ++j) {
            const uint64_t t = gw + static_cast<uint64_t>(it + j) * GW;
            if (t >= ntiles) break;
            const uint32_t jt = it + j;
            mbar_wait(&P.bars[jt % P.stages], (jt / P.stages) & 1u, kDrainLimitNs);
        }
    }
    // the zero-padded tail block is tested and scanned by CTA 0, warp 0
    if ((p.n & 1023u) && blockIdx.x == 0 && warp == 0) {
        const uint2 z = p.zonemap[p.n >> 10];
        if (static_cast<uint64_t>(z.y) >= p.zlo && static_cast<uint64_t>(z.x) < p.zhi) {
            if ((p.flags & kFlagAgg) && static_cast<uint64_t>(z.x) >= p.zlo && static_cast<uint64_t>(z.y) < p.zhi) {
                // every value of the tail matches: count and (code) sum from the metadata
                if (lane == 0) {
                    const uint64_t rem = p.n & 1023u;
                    cnt += rem;
                    sum += p.blocksum[p.n >> 10] - static_cast<uint64_t>(p.base) * rem;
                }
            } else {
                scan_tail<B>(p, lane, cnt, sum);
                if (lane == 0) p.qctl[2] = 1ull;
            }
        }
    }
    grid_finish<Shape<B>::kWarps>(p, cnt, sum, true, 0);
}

// ----------------------------------------------------------- dispatching
enum OpKind : int {
    kOpFullBF = 0,
    kOpFullBR = 1,
    kOpQueueBF = 2,
    kOpQueueBR = 3,
    kOpZoneBuild = 4,
    kOpRowBF = 5,     // row-major layout (§3 strategy i)
    kOpRowBR = 6,
    kOpBytesBF = 7,   // byte-aligned layout, b = 8 or 16 (§3 strategy iii)
    kOpBytesBR = 8,
    kOpBatchBF = 9,   // batched scans (one width group of a batch); only their shapes
    kOpBatchBR = 10,  // are kept here, the kernels live with the batch
};

struct ShapeInfo {
    int warps, stages, tile_blocks, smem_bytes;
};

// A runtime launch shape: CTAs of `warps` warps (one per SM for single-column
// scans, two for batched ones), each warp with `stages` slots of `tile_blocks`
// blocks (the zone-skip kernels take that many candidates per tile); vote_rows
// picks the branchy vote form (0 per value, 1 per row, 2 and 3 the PTX row
// blocks; full branchy scans at b <= 21 only); vec_lanes = 2 the 2-lane
// geometry (full scans at b = 9..16, compiled with the 16-warp bound).  Full
// scans take 8..16 warps (above 8, and for vote forms 2 and 3, the
// 16-warp-bound instantiation, <= 128 registers per thread); every other
// single-column kernel 1..8.
struct LaunchShape {
    int warps, stages, tile_blocks, vote_rows;
    int vec_lanes;  // lanes per thread and row (4 or 2; 0 = the width's default); full scans only
};

template <int LO, int HI>
__host__ inline ShapeInfo shape_range(int b)
{
    if constexpr (LO > HI) {
        return ShapeInfo{0, 0, 0, 0};
    } else {
        if (b == LO) return ShapeInfo{Shape<LO>::kWarps, Shape<LO>::kStages, Shape<LO>::kTB,
                                      Shape<LO>::kSmemBytes};
        return shape_range<LO + 1, HI>(b);
    }
}
inline ShapeInfo shape_of(int b) { return shape_range<1, 32>(b); }

}  // namespace gb

// One translation unit per width range instantiates the kernels; these are
// the entry points the host library dispatches to.
// The shape's tile_blocks and stages override those fields of p.
#define GB_DECLARE_RANGE(lo, hi)                                                                          \
    cudaError_t gb_launch_range_##lo##_##hi(int b, int op, const gb::ScanParams& p, const gb::LaunchShape& sh, \
                                            int grid, cudaStream_t st);
GB_DECLARE_RANGE(1, 4)
GB_DECLARE_RANGE(5, 8)
GB_DECLARE_RANGE(9, 12)
GB_DECLARE_RANGE(13, 16)
GB_DECLARE_RANGE(17, 20)
GB_DECLARE_RANGE(21, 24)
GB_DECLARE_RANGE(25, 28)
GB_DECLARE_RANGE(29, 32)
#undef GB_DECLARE_RANGE

// Dispatch to the range's launcher.
inline cudaError_t gb_launch(int b, int op, const gb::ScanParams& p, const gb::LaunchShape& sh, int grid,
                             cudaStream_t st)
{
    switch ((b - 1) / 4) {
    case 0: return gb_launch_range_1_4(b, op, p, sh, grid, st);
    case 1: return gb_launch_range_5_8(b, op, p, sh, grid, st);
    case 2: return gb_launch_range_9_12(b, op, p, sh, grid, st);
    case 3: return gb_launch_range_13_16(b, op, p, sh, grid, st);
    case 4: return gb_launch_range_17_20(b, op, p, sh, grid, st);
    case 5: return gb_launch_range_21_24(b, op, p, sh, grid, st);
    case 6: return gb_launch_range_25_28(b, op, p, sh, grid, st);
    case 7: return gb_launch_range_29_32(b, op, p, sh, grid, st);
    default: return cudaErrorInvalidValue;
    }
}
