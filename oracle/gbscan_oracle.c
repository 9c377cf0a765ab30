/*
 * Plain, slow, single-threaded CPU oracle for the fused columnar scan.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or
 * load this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it. It shares no code, header or constant with the CUDA
 * library; both sides only receive inputs from the seeded generators.
 *
 * What it computes (paper §2 "Problem and Model", §3 "Method"): a column of
 * N unsigned 32-bit values v_i, each stored in b bits (1 <= b <= 32), is
 * decoded, filtered by a predicate and aggregated in one pass.  The paper's
 * predicates are equality counts; the scan here takes the half-open range
 * lo <= v < hi (equality c is the range [c, c+1)) and returns
 *     COUNT = #{ i : lo <= v_i < hi }
 *     SUM   = sum of v_i over those i, exact in int64.
 *
 * Readings of what the paper leaves open (each one is a choice, listed with
 * its reason in the design notes):
 *   - Frame of reference: the stored code is u_i = v_i - base, 0 <= u_i < 2^b,
 *     and base + 2^b - 1 must fit in 32 bits (so b = 32 forces base = 0).
 *   - Transposed layout (§3, "FastLanes-style", 1024-value blocks over 32
 *     lanes): value j of block k goes to lane j mod 32 at row floor(j/32).
 *     Each lane owns a stream of 32*b bits; row r occupies stream bits
 *     [r*b, r*b + b), least significant bit first, and stream bit p lives in
 *     bit (p mod 32) of the lane's word floor(p/32).  Lane word w of block k
 *     is stored at 32-bit offset 32*b*k + 32*w + lane.  No row reordering.
 *   - The last block is padded with zero codes; padding is never counted.
 *   - Zone maps (§3, "per-block zone maps (min/max skipping)"): one
 *     (min, max) pair of decoded values per 1024-value block, over valid
 *     positions only.  A block is skipped iff max < lo or min >= hi, which
 *     cannot change COUNT or SUM.
 *
 * Parity pins for every function live in tests/test_oracle.py.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <pthread.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL 1

#define BLOCK_VALUES 1024u
#define LANES 32u

uint64_t oracle_n_blocks(uint64_t n) { return (n + BLOCK_VALUES - 1) / BLOCK_VALUES; }

/* Number of 32-bit words of the packed column: b words per lane, 32 lanes per block. */
uint64_t oracle_packed_words(uint64_t n, uint32_t b)
{
    return oracle_n_blocks(n) * (uint64_t)LANES * (uint64_t)b;
}

static int width_ok(uint32_t b, uint32_t base)
{
    if (b < 1 || b > 32) return 0;
    /* the largest code must still decode to a 32-bit value */
    if ((uint64_t)base + ((1ull << b) - 1ull) > 0xFFFFFFFFull) return 0;
    return 1;
}

/* Offset of lane word `w` (0 <= w < b) of block `k`. */
static uint64_t word_at(uint64_t k, uint32_t b, uint64_t w, uint32_t lane)
{
    return k * (uint64_t)LANES * b + (uint64_t)LANES * w + lane;
}

/* Encode: FOR subtraction, then place each code in its lane stream. */
int oracle_pack(const uint32_t *values, uint64_t n, uint32_t b, uint32_t base, uint32_t *out)
{
    uint64_t i;
    if (!width_ok(b, base)) return ORACLE_EINVAL;
    if (n > 0 && (values == NULL || out == NULL)) return ORACLE_EINVAL;
    for (i = 0; i < n; ++i) {
        if (values[i] < base) return ORACLE_EINVAL;
        if ((uint64_t)(values[i] - base) >> b) return ORACLE_EINVAL;
    }
    if (n == 0) return ORACLE_OK;
    memset(out, 0, oracle_packed_words(n, b) * sizeof(uint32_t));
    for (i = 0; i < n; ++i) {
        uint64_t u = (uint64_t)(values[i] - base);
        uint64_t k = i / BLOCK_VALUES;
        uint64_t j = i % BLOCK_VALUES;
        uint32_t lane = (uint32_t)(j % LANES);
        uint64_t row = j / LANES;
        uint64_t p = row * b;            /* first stream bit of this value */
        uint64_t w = p / 32;
        uint32_t off = (uint32_t)(p % 32);
        out[word_at(k, b, w, lane)] |= (uint32_t)(u << off);
        if (off + b > 32) /* the value continues in the lane's next word */
            out[word_at(k, b, w + 1, lane)] |= (uint32_t)(u >> (32 - off));
    }
    return ORACLE_OK;
}

/* Code of value i, read back from its lane stream. */
static uint32_t code_at(const uint32_t *words, uint64_t i, uint32_t b)
{
    uint64_t k = i / BLOCK_VALUES;
    uint64_t j = i % BLOCK_VALUES;
    uint32_t lane = (uint32_t)(j % LANES);
    uint64_t row = j / LANES;
    uint64_t p = row * b;
    uint64_t w = p / 32;
    uint32_t off = (uint32_t)(p % 32);
    uint64_t window = words[word_at(k, b, w, lane)];
    if (off + b > 32) window |= (uint64_t)words[word_at(k, b, w + 1, lane)] << 32;
    return (uint32_t)((window >> off) & ((1ull << b) - 1ull));
}

/* Decode: code plus base. */
int oracle_unpack(const uint32_t *words, uint64_t n, uint32_t b, uint32_t base, uint32_t *values)
{
    uint64_t i;
    if (!width_ok(b, base)) return ORACLE_EINVAL;
    for (i = 0; i < n; ++i) values[i] = code_at(words, i, b) + base;
    return ORACLE_OK;
}

/* The plain definition over raw values: brute force, no packing involved. */
void oracle_scan_values(const uint32_t *values, uint64_t n, int64_t lo, int64_t hi,
                        int64_t *count, int64_t *sum)
{
    int64_t c = 0, s = 0;
    uint64_t i;
    for (i = 0; i < n; ++i) {
        int64_t v = (int64_t)values[i];
        if (lo <= v && v < hi) {
            c += 1;
            s += v;
        }
    }
    *count = c;
    *sum = s;
}

/* Fused decode -> filter -> aggregate over values [first, last) of a packed column. */
static void scan_range(const uint32_t *words, uint64_t first, uint64_t last, uint32_t b,
                       uint32_t base, int64_t lo, int64_t hi, int64_t *count, int64_t *sum)
{
    int64_t c = 0, s = 0;
    uint64_t i;
    for (i = first; i < last; ++i) {
        int64_t v = (int64_t)code_at(words, i, b) + (int64_t)base;
        if (lo <= v && v < hi) {
            c += 1;
            s += v;
        }
    }
    *count = c;
    *sum = s;
}

int oracle_scan_packed(const uint32_t *words, uint64_t n, uint32_t b, uint32_t base,
                       int64_t lo, int64_t hi, int64_t *count, int64_t *sum)
{
    if (!width_ok(b, base)) return ORACLE_EINVAL;
    scan_range(words, 0, n, b, base, lo, hi, count, sum);
    return ORACLE_OK;
}

/* Per-block (min, max) of decoded values over the block's valid positions. */
int oracle_zonemap(const uint32_t *words, uint64_t n, uint32_t b, uint32_t base,
                   uint32_t *zmin, uint32_t *zmax)
{
    uint64_t k, i, nb = oracle_n_blocks(n);
    if (!width_ok(b, base)) return ORACLE_EINVAL;
    for (k = 0; k < nb; ++k) {
        uint64_t first = k * BLOCK_VALUES;
        uint64_t last = first + BLOCK_VALUES < n ? first + BLOCK_VALUES : n;
        uint32_t mn = 0xFFFFFFFFu, mx = 0;
        for (i = first; i < last; ++i) {
            uint32_t v = code_at(words, i, b) + base;
            if (v < mn) mn = v;
            if (v > mx) mx = v;
        }
        zmin[k] = mn;
        zmax[k] = mx;
    }
    return ORACLE_OK;
}

/* Zone-map skipping: scan only the blocks whose [min, max] meets [lo, hi). */
int oracle_scan_zoneskip(const uint32_t *words, const uint32_t *zmin, const uint32_t *zmax,
                         uint64_t n, uint32_t b, uint32_t base, int64_t lo, int64_t hi,
                         int64_t *count, int64_t *sum, uint64_t *blocks_scanned)
{
    uint64_t k, nb = oracle_n_blocks(n), touched = 0;
    int64_t c = 0, s = 0;
    if (!width_ok(b, base)) return ORACLE_EINVAL;
    for (k = 0; k < nb; ++k) {
        uint64_t first = k * BLOCK_VALUES;
        uint64_t last = first + BLOCK_VALUES < n ? first + BLOCK_VALUES : n;
        int64_t bc, bs;
        if ((int64_t)zmax[k] < lo || (int64_t)zmin[k] >= hi) continue;
        touched += 1;
        scan_range(words, first, last, b, base, lo, hi, &bc, &bs);
        c += bc;
        s += bs;
    }
    *count = c;
    *sum = s;
    *blocks_scanned = touched;
    return ORACLE_OK;
}

/*
 * Conjunctive predicate over k columns of one table (the problem statement
 * of paper §2 extended to several columns of equal length; rows are shared
 * positions): COUNT = #{ i : lo_c <= v_c,i < hi_c for every c }, and SUM =
 * the sum of the aggregate column's values over those rows (exact int64;
 * 0 when agg_words is NULL).  All columns in the transposed layout.
 */
int oracle_scan_conj(const uint32_t *const *words, const uint32_t *b, const uint32_t *base, const int64_t *lo,
                     const int64_t *hi, uint32_t k, uint64_t n, const uint32_t *agg_words, uint32_t agg_b,
                     uint32_t agg_base, int64_t *count, int64_t *sum)
{
    uint64_t i;
    uint32_t c;
    int64_t cnt = 0, sm = 0;
    for (c = 0; c < k; ++c)
        if (!width_ok(b[c], base[c])) return ORACLE_EINVAL;
    if (agg_words && !width_ok(agg_b, agg_base)) return ORACLE_EINVAL;
    for (i = 0; i < n; ++i) {
        int all = 1;
        for (c = 0; c < k && all; ++c) {
            int64_t v = (int64_t)code_at(words[c], i, b[c]) + (int64_t)base[c];
            all = lo[c] <= v && v < hi[c];
        }
        if (!all) continue;
        cnt += 1;
        if (agg_words) sm += (int64_t)code_at(agg_words, i, agg_b) + (int64_t)agg_base;
    }
    *count = cnt;
    *sum = sm;
    return ORACLE_OK;
}

/*
 * Per-block aggregate metadata (an extension of the zone maps, not in the
 * paper): the sum of the block's decoded values over its valid positions.
 * With (min, max, sum) a block whose values all satisfy the predicate
 * (lo <= min and max < hi) contributes (valid count, sum) without reading
 * its data; a block outside it is skipped; only the remaining blocks are
 * scanned.  The result equals the full scan exactly.
 */
int oracle_blocksums(const uint32_t *words, uint64_t n, uint32_t b, uint32_t base, uint64_t *sums)
{
    uint64_t k, i, nb = oracle_n_blocks(n);
    if (!width_ok(b, base)) return ORACLE_EINVAL;
    for (k = 0; k < nb; ++k) {
        uint64_t first = k * BLOCK_VALUES;
        uint64_t last = first + BLOCK_VALUES < n ? first + BLOCK_VALUES : n;
        uint64_t acc = 0;
        for (i = first; i < last; ++i) acc += (uint64_t)code_at(words, i, b) + base;
        sums[k] = acc;
    }
    return ORACLE_OK;
}

int oracle_scan_zoneagg(const uint32_t *words, const uint32_t *zmin, const uint32_t *zmax, const uint64_t *sums,
                        uint64_t n, uint32_t b, uint32_t base, int64_t lo, int64_t hi, int64_t *count,
                        int64_t *sum, uint64_t *blocks_scanned)
{
    uint64_t k, nb = oracle_n_blocks(n), touched = 0;
    int64_t c = 0, s = 0;
    if (!width_ok(b, base)) return ORACLE_EINVAL;
    for (k = 0; k < nb; ++k) {
        uint64_t first = k * BLOCK_VALUES;
        uint64_t last = first + BLOCK_VALUES < n ? first + BLOCK_VALUES : n;
        int64_t bc, bs;
        if ((int64_t)zmax[k] < lo || (int64_t)zmin[k] >= hi) continue;      /* no value can match */
        if (lo <= (int64_t)zmin[k] && (int64_t)zmax[k] < hi) {                /* every value matches */
            c += (int64_t)(last - first);
            s += (int64_t)sums[k];
            continue;
        }
        touched += 1;
        scan_range(words, first, last, b, base, lo, hi, &bc, &bs);
        c += bc;
        s += bs;
    }
    *count = c;
    *sum = s;
    *blocks_scanned = touched;
    return ORACLE_OK;
}

/*
 * Two further layouts of the same codes (paper §3 lists three decode
 * strategies; the transposed one above is strategy (ii)).
 *
 * Row-major bit packing, strategy (i) ("scalar row-major bit-unpacking"):
 * value i's code occupies bits [i*b, i*b + b) of one stream of 32-bit words,
 * least significant bit first; bit p is bit (p mod 32) of word floor(p/32).
 * The stream is zero-padded to whole 1024-value blocks, so it has the same
 * oracle_packed_words(n, b) words as the transposed layout.
 *
 * Byte-aligned widths, strategy (iii): for b in {8, 16, 32} the codes form a
 * plain little-endian array of b-bit integers (the same bytes as row-major
 * packing at those widths), zero-padded the same way.
 */
int oracle_pack_rowmajor(const uint32_t *values, uint64_t n, uint32_t b, uint32_t base, uint32_t *out)
{
    uint64_t i, total = oracle_packed_words(n, b);
    uint32_t k;
    if (!width_ok(b, base)) return ORACLE_EINVAL;
    for (i = 0; i < n; ++i) {
        if (values[i] < base || (uint64_t)(values[i] - base) > ((1ull << b) - 1ull)) return ORACLE_EINVAL;
    }
    memset(out, 0, (size_t)total * sizeof(uint32_t));
    for (i = 0; i < n; ++i) {
        uint32_t u = values[i] - base;
        for (k = 0; k < b; ++k) {
            uint64_t p = i * (uint64_t)b + k;
            if ((u >> k) & 1u) out[p / 32] |= 1u << (p % 32);
        }
    }
    return ORACLE_OK;
}

/* Code of value i of a row-major stream (a 64-bit window over two words). */
static uint32_t rowmajor_code_at(const uint32_t *words, uint64_t i, uint32_t b)
{
    uint64_t p = i * (uint64_t)b;
    uint64_t w = p / 32;
    uint32_t off = (uint32_t)(p % 32);
    uint64_t window = words[w];
    if (off + b > 32) window |= (uint64_t)words[w + 1] << 32;
    return (uint32_t)((window >> off) & ((1ull << b) - 1ull));
}

int oracle_unpack_rowmajor(const uint32_t *words, uint64_t n, uint32_t b, uint32_t base, uint32_t *values)
{
    uint64_t i;
    if (!width_ok(b, base)) return ORACLE_EINVAL;
    for (i = 0; i < n; ++i) values[i] = rowmajor_code_at(words, i, b) + base;
    return ORACLE_OK;
}

int oracle_scan_rowmajor(const uint32_t *words, uint64_t n, uint32_t b, uint32_t base, int64_t lo, int64_t hi,
                         int64_t *count, int64_t *sum)
{
    int64_t c = 0, s = 0;
    uint64_t i;
    if (!width_ok(b, base)) return ORACLE_EINVAL;
    for (i = 0; i < n; ++i) {
        int64_t v = (int64_t)rowmajor_code_at(words, i, b) + (int64_t)base;
        if (lo <= v && v < hi) {
            c += 1;
            s += v;
        }
    }
    *count = c;
    *sum = s;
    return ORACLE_OK;
}

/* Byte-aligned codes: element i of a uint8/uint16/uint32 array. */
static uint32_t bytes_code_at(const void *codes, uint64_t i, uint32_t b)
{
    if (b == 8) return ((const uint8_t *)codes)[i];
    if (b == 16) return ((const uint16_t *)codes)[i];
    return ((const uint32_t *)codes)[i];
}

int oracle_pack_bytes(const uint32_t *values, uint64_t n, uint32_t b, uint32_t base, void *out)
{
    uint64_t i, total = oracle_packed_words(n, b);
    if (b != 8 && b != 16 && b != 32) return ORACLE_EINVAL;
    if (!width_ok(b, base)) return ORACLE_EINVAL;
    for (i = 0; i < n; ++i) {
        if (values[i] < base || (uint64_t)(values[i] - base) > ((1ull << b) - 1ull)) return ORACLE_EINVAL;
    }
    memset(out, 0, (size_t)total * sizeof(uint32_t));
    for (i = 0; i < n; ++i) {
        uint32_t u = values[i] - base;
        if (b == 8) ((uint8_t *)out)[i] = (uint8_t)u;
        else if (b == 16) ((uint16_t *)out)[i] = (uint16_t)u;
        else ((uint32_t *)out)[i] = u;
    }
    return ORACLE_OK;
}

int oracle_scan_bytes(const void *codes, uint64_t n, uint32_t b, uint32_t base, int64_t lo, int64_t hi,
                      int64_t *count, int64_t *sum)
{
    int64_t c = 0, s = 0;
    uint64_t i;
    if (b != 8 && b != 16 && b != 32) return ORACLE_EINVAL;
    if (!width_ok(b, base)) return ORACLE_EINVAL;
    for (i = 0; i < n; ++i) {
        int64_t v = (int64_t)bytes_code_at(codes, i, b) + (int64_t)base;
        if (lo <= v && v < hi) {
            c += 1;
            s += v;
        }
    }
    *count = c;
    *sum = s;
    return ORACLE_OK;
}

/*
 * Materializing select (paper §3 lists "a materializing select" beside the
 * counts; §4 "Branch" measures it): the positions i of the values with
 * lo <= v_i < hi, in increasing order.  The first min(count, capacity)
 * positions go to `pos` (which may be NULL when capacity is 0); the return
 * value is the full count, so a caller can size a second attempt.
 */
uint64_t oracle_select_values(const uint32_t *values, uint64_t n, int64_t lo, int64_t hi,
                              uint32_t *pos, uint64_t capacity)
{
    uint64_t i, k = 0;
    for (i = 0; i < n; ++i) {
        int64_t v = (int64_t)values[i];
        if (lo <= v && v < hi) {
            if (k < capacity) pos[k] = (uint32_t)i;
            k += 1;
        }
    }
    return k;
}

/* The same select over a packed column: decode each value, then test it. */
int oracle_select_packed(const uint32_t *words, uint64_t n, uint32_t b, uint32_t base, int64_t lo,
                         int64_t hi, uint32_t *pos, uint64_t capacity, uint64_t *count)
{
    uint64_t i, k = 0;
    if (!width_ok(b, base)) return ORACLE_EINVAL;
    for (i = 0; i < n; ++i) {
        int64_t v = (int64_t)code_at(words, i, b) + (int64_t)base;
        if (lo <= v && v < hi) {
            if (k < capacity) pos[k] = (uint32_t)i;
            k += 1;
        }
    }
    *count = k;
    return ORACLE_OK;
}

/*
 * The same fused scan split over `threads` disjoint block ranges, one POSIX
 * thread each, with the per-thread (count, sum) added at the end.  Integer
 * addition is associative, so the result equals oracle_scan_packed exactly.
 * Used only to time the oracle on all host cores.
 */
struct range_job {
    const uint32_t *words;
    uint64_t first, last;
    uint32_t b, base;
    int64_t lo, hi, count, sum;
};

static void *range_worker(void *arg)
{
    struct range_job *j = (struct range_job *)arg;
    scan_range(j->words, j->first, j->last, j->b, j->base, j->lo, j->hi, &j->count, &j->sum);
    return NULL;
}

int oracle_scan_packed_threads(const uint32_t *words, uint64_t n, uint32_t b, uint32_t base,
                               int64_t lo, int64_t hi, int threads, int64_t *count, int64_t *sum)
{
    enum { MAX_THREADS = 1024 };
    static struct range_job jobs[MAX_THREADS];
    static pthread_t tids[MAX_THREADS];
    static int running[MAX_THREADS];
    uint64_t nb = oracle_n_blocks(n), per;
    int t;
    int64_t c = 0, s = 0;
    if (!width_ok(b, base) || threads < 1 || threads > MAX_THREADS) return ORACLE_EINVAL;
    per = (nb + (uint64_t)threads - 1) / (uint64_t)threads;
    for (t = 0; t < threads; ++t) {
        uint64_t fb = (uint64_t)t * per, lb = fb + per;
        jobs[t].words = words;
        jobs[t].first = fb * BLOCK_VALUES < n ? fb * BLOCK_VALUES : n;
        jobs[t].last = lb * BLOCK_VALUES < n ? lb * BLOCK_VALUES : n;
        jobs[t].b = b;
        jobs[t].base = base;
        jobs[t].lo = lo;
        jobs[t].hi = hi;
        jobs[t].count = 0;
        jobs[t].sum = 0;
        running[t] = pthread_create(&tids[t], NULL, range_worker, &jobs[t]) == 0;
        if (!running[t]) range_worker(&jobs[t]); /* run inline if a thread cannot start */
    }
    for (t = 0; t < threads; ++t) {
        if (running[t]) pthread_join(tids[t], NULL);
        c += jobs[t].count;
        s += jobs[t].sum;
    }
    *count = c;
    *sum = s;
    return ORACLE_OK;
}
