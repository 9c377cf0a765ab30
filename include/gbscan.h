/*
 * gbscan: fused columnar scan for GB300 (sm_103a) behind a plain C ABI.
 *
 * The operation (paper §2 "Problem and Model"): a column of N unsigned 32-bit
 * values, each stored in b bits (1 <= b <= 32), is decoded, filtered and
 * aggregated in one pass.  Reading the column costs N*b/8 bytes, so the scan
 * can at best run at the memory bandwidth beta; the paper's bandwidth
 * fraction is f = (N*b/8 / T) / beta and its law (Eq. 2) is
 * f = min(1, T_dec*b/(8*beta)) with ridge b* = 8*beta/T_dec.
 *
 * Encoding (paper §3, the FastLanes-style transposed layout):
 *   - frame of reference: code u = v - base, 0 <= u < 2^b, and
 *     base + 2^b - 1 <= 2^32 - 1 (so b = 32 forces base = 0);
 *   - 1024-value blocks over 32 lanes: value j of block k goes to lane
 *     j mod 32, row j / 32; a lane's stream holds its 32 rows' b-bit codes
 *     least-significant bit first; stream bit p is bit p mod 32 of lane word
 *     p / 32; lane word w of block k is 32-bit word 32*b*k + 32*w + lane.
 *     A block is b rows of 32 words, i.e. 128*b contiguous bytes;
 *   - the last block is zero padded; padding never matches.
 *   The packed column occupies scan_packed_words(n, b) 32-bit words.
 *
 * Predicate and aggregate: half-open lo <= v < hi on decoded values (int64
 * bounds; the paper's equality count on c is [c, c+1)); the result is the
 * exact COUNT and the exact int64 SUM of the matching values.  N <= 2^31,
 * so the SUM cannot overflow.
 *
 * Conventions for every entry point:
 *   - the return value is a scan_status; no C++ exception crosses the ABI;
 *     on failure scan_last_error() returns a message (thread local);
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); work is enqueued on it and, unless stated, the call returns
 *     without waiting;
 *   - pointers named dev_* are device memory on the current CUDA device,
 *     host_* are host memory (pinned memory makes copies asynchronous);
 *   - a scan_column owns the device memory it allocates and frees it in
 *     scan_column_destroy; a column made by scan_column_create_packed borrows
 *     the caller's packed buffer, which must outlive the column;
 *   - calls that use the same column must be ordered on one stream (a column
 *     carries its own small device workspace); different columns may run on
 *     different streams concurrently.
 */
#ifndef GBSCAN_H
#define GBSCAN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SCAN_OK = 0,
    SCAN_EINVAL = 1,   /* bad argument: width, range, size, null or misaligned pointer */
    SCAN_ENOMEM = 2,   /* a device or pinned host allocation failed */
    SCAN_ECUDA = 3,    /* a CUDA runtime call failed; see scan_last_error() */
    SCAN_ETIMEOUT = 4, /* a bounded device-side wait gave up; the result is not valid */
    SCAN_EBUSY = 5,    /* resource temporarily unavailable (e.g. a full server queue) */
    SCAN_ENOTSUP = 6   /* the request is valid but this build cannot serve it */
} scan_status;

typedef enum {
    /* Library picks, per call, by the paper's law (§2) and its clustering
     * crossover (§6: skipping pays on clustered data only).  Without a zone
     * map: the branch-free full scan.  With one (lane layout): the exact
     * number of blocks the zone test would keep is counted on the host from
     * sorted copies of the zone map's bounds (no device work, no
     * synchronization), and the branch-free full scan runs when they reach the
     * law's break-even -- a fraction min(0.9, (128b - 8) / (128b + 8)) of the
     * blocks, where the 8 bytes of zone map and id per block cost what the
     * 128b data bytes of the skipped ones save -- else branch-free zone
     * skipping.  The first SCAN_AUTO call after scan_zonemap_build copies the
     * zone map to the host and sorts its bounds, synchronizing `stream` once
     * (make it before any stream capture).  blocks_scanned reports which was
     * run.  Always the same COUNT/SUM. */
    SCAN_AUTO = 0,
    SCAN_BRANCHFREE = 1,   /* full scan, predicated (mask) aggregation */
    SCAN_BRANCHY = 2,      /* full scan, warp-vote early-out per 32-value group */
    SCAN_ZONE_SKIP_BF = 3, /* zone-map block skipping (a persistent walk over the survivors), branch-free */
    SCAN_ZONE_SKIP_BR = 4, /* zone-map block skipping (a persistent walk over the survivors), branchy */
    /* Zone skipping that also answers every block wholly inside [lo, hi)
     * (lo <= min and max < hi) from its metadata -- its valid count and the
     * per-block sum built by scan_zonemap_build -- without reading its data;
     * only blocks that straddle a bound are scanned (an extension of the
     * paper's zone maps; the result is the same).  Lane layout only; not
     * taken by batches or the planner. */
    SCAN_ZONE_AGG_BF = 5,
    SCAN_ZONE_AGG_BR = 6
} scan_strategy;

typedef struct {
    int64_t lo; /* inclusive lower bound on decoded v */
    int64_t hi; /* exclusive upper bound; lo >= hi selects nothing */
} scan_pred;

typedef struct {
    int64_t count;           /* #{ i : lo <= v_i < hi } */
    int64_t sum;             /* sum of those v_i, exact */
    uint64_t blocks_scanned; /* 1024-value blocks whose packed bytes were read */
    uint64_t reserved;
} scan_result;

typedef struct scan_column scan_column; /* opaque */

/* ------------------------------------------------------------ messages */

/* Message for the last failing call on this thread ("" if none). Never NULL. */
const char *scan_last_error(void);

/* Name of a status code, e.g. "SCAN_EINVAL". Never NULL. */
const char *scan_status_string(scan_status s);

/* ------------------------------------------------------ layout (host only) */

/* 32-bit words of a packed column of n values at b bits: ceil(n/1024)*32*b.
 * Returns 0 for b outside 1..32. */
uint64_t scan_packed_words(uint64_t n, uint32_t b);

/* Host encoder (paper §3 transposed layout, with frame of reference).
 * Writes scan_packed_words(n, b) words to host_out (caller owned).  Needs no
 * GPU.  SCAN_EINVAL if b is outside 1..32, base + 2^b - 1 > 2^32 - 1, n > 2^31,
 * a pointer is NULL (n > 0), or any value lies outside [base, base + 2^b). */
scan_status scan_encode_host(const uint32_t *host_values, uint64_t n, uint32_t b, uint32_t base,
                             uint32_t *host_out);

/* Device encoder: the same layout, computed on the GPU from dev_values into
 * dev_out (scan_packed_words(n, b) words, 16-byte aligned).  Synchronises
 * the stream to report out-of-range values as SCAN_EINVAL. */
scan_status scan_encode_device(const uint32_t *dev_values, uint64_t n, uint32_t b, uint32_t base,
                               uint32_t *dev_out, void *stream);

/* ------------------------------------------------------------- layouts */

/* Order of the codes inside each 1024-value block (paper §3, three decode
 * strategies).  Every layout occupies the same scan_packed_words(n, b) words,
 * block k at words [32*b*k, 32*b*(k+1)), the last block zero-padded.
 *   SCAN_LAYOUT_LANES   : lane-interleaved ("FastLanes-style transposed",
 *                         strategy ii; see scan_encode_host).  Default.
 *   SCAN_LAYOUT_ROWMAJOR: value i at bits [i*b, i*b + b) of one LSB-first
 *                         stream of 32-bit words ("scalar row-major",
 *                         strategy i).
 *   SCAN_LAYOUT_BYTES   : b in {8, 16, 32}: the codes as a plain uint8 /
 *                         uint16 / uint32 array ("byte-aligned", strategy
 *                         iii) -- the same bytes as SCAN_LAYOUT_ROWMAJOR at
 *                         those widths, read by a byte-permute decoder.
 * At b = 32 all three are the plain array (and read by the same kernel).
 * Only lane-interleaved columns take zone maps, zone-skip strategies, the
 * select, batches and the server (SCAN_EINVAL otherwise). */
typedef enum {
    SCAN_LAYOUT_LANES = 0,
    SCAN_LAYOUT_ROWMAJOR = 1,
    SCAN_LAYOUT_BYTES = 2
} scan_layout;

/* scan_encode_host / scan_encode_device for any layout (SCAN_EINVAL for
 * SCAN_LAYOUT_BYTES unless b is 8, 16 or 32). */
scan_status scan_encode_host_layout(const uint32_t *host_values, uint64_t n, uint32_t b, uint32_t base,
                                    scan_layout layout, uint32_t *host_out);
scan_status scan_encode_device_layout(const uint32_t *dev_values, uint64_t n, uint32_t b, uint32_t base,
                                      scan_layout layout, uint32_t *dev_out, void *stream);

/* -------------------------------------------------------------- columns */

/* A column in the paper's problem statement (§2: N values stored in b bits
 * each), encoded in §3's transposed layout with a frame of reference: encode
 * host_values (n of them, caller owned, read only) on the host, allocate the
 * column's device memory (owned by the column) and upload.  Returns after the
 * upload is complete.  SCAN_EINVAL as scan_encode_host (bad b or base, n >
 * 2^31, NULL pointers, a value outside [base, base + 2^b)); SCAN_ENOMEM if an
 * allocation fails. */
scan_status scan_column_create(const uint32_t *host_values, uint64_t n, uint32_t b, uint32_t base,
                               void *stream, scan_column **out);

/* As scan_column_create for values already in device memory (dev_values, n
 * of them, caller owned): §3's encoding runs on the GPU into memory the
 * column owns.  Synchronises `stream` to report out-of-range values as
 * SCAN_EINVAL. */
scan_status scan_column_create_device(const uint32_t *dev_values, uint64_t n, uint32_t b,
                                      uint32_t base, void *stream, scan_column **out);

/* Wrap a device buffer already packed in §3's layout (scan_packed_words(n, b)
 * words, 16-byte aligned) without copying; the caller keeps ownership and
 * the buffer must outlive the column.  The column allocates only its small
 * workspace.  SCAN_EINVAL for bad b or base, n > 2^31, a NULL (n > 0) or
 * misaligned buffer. */
scan_status scan_column_create_packed(const uint32_t *dev_packed, uint64_t n, uint32_t b,
                                      uint32_t base, void *stream, scan_column **out);

/* The three creators for a given layout (the ones above use SCAN_LAYOUT_LANES). */
scan_status scan_column_create_layout(const uint32_t *host_values, uint64_t n, uint32_t b, uint32_t base,
                                      scan_layout layout, void *stream, scan_column **out);
scan_status scan_column_create_device_layout(const uint32_t *dev_values, uint64_t n, uint32_t b,
                                             uint32_t base, scan_layout layout, void *stream,
                                             scan_column **out);
scan_status scan_column_create_packed_layout(const uint32_t *dev_packed, uint64_t n, uint32_t b,
                                             uint32_t base, scan_layout layout, void *stream,
                                             scan_column **out);
scan_status scan_column_get_layout(const scan_column *col, scan_layout *layout);

/* Overwrite the column's packed bytes from a host buffer of
 * scan_packed_words(n, b) words (asynchronous if host_packed is pinned).
 * Any zone map built before is marked stale and must be rebuilt. */
scan_status scan_column_upload_packed(scan_column *col, const uint32_t *host_packed, void *stream);

/* Free the column and the device memory it owns (not a borrowed packed
 * buffer).  Synchronises the device first, so no scan of the column is still
 * running.  NULL is accepted and ignored. */
scan_status scan_column_destroy(scan_column *col);

/* Shape and device pointers of a column (any out pointer may be NULL).
 * dev_zonemap is NULL until scan_zonemap_build has run; it holds one
 * (min, max) pair of decoded uint32 values per block, as 2*nblocks words. */
scan_status scan_column_info(const scan_column *col, uint64_t *n, uint32_t *b, uint32_t *base,
                             const uint32_t **dev_packed, const uint32_t **dev_zonemap);

/* ------------------------------------------------------------ zone maps */

/* Build the per-block (min, max) zone map (paper §3, "per-block zone maps
 * (min/max skipping)"; §6 clustering crossover) and, in the same pass, the
 * per-block sum of decoded values (uint64, over valid positions) that the
 * SCAN_ZONE_AGG_* strategies use.  Idempotent; one read of the packed
 * column, 16 bytes written per block.  Lane-interleaved columns only. */
scan_status scan_zonemap_build(scan_column *col, void *stream);

/* Device pointer to the per-block sums (NULL until scan_zonemap_build). */
scan_status scan_column_blocksums(const scan_column *col, const uint64_t **dev_blocksums);

/* ---------------------------------------------------------------- scans */

/* The paper's operation (§2 problem statement; §3 "fused
 * decode->filter->aggregate in one pass"): COUNT and exact int64 SUM of the
 * column's decoded values v with pred.lo <= v < pred.hi.  Enqueues the
 * kernels on `stream`, waits for them and writes the result to host_out
 * (caller owned).  The result is the same, bit for bit, for every strategy;
 * blocks_scanned says how many 1024-value blocks were read.  Zone-skip
 * strategies need a built zone map (SCAN_EINVAL otherwise).  SCAN_ETIMEOUT if
 * a bounded device wait gave up (the result is then not valid; the column's
 * state is reset and it stays usable). */
scan_status scan_run(scan_column *col, scan_pred pred, scan_strategy strategy, void *stream,
                     scan_result *host_out);

/* The same operation as scan_run (§2, §3), asynchronous: writes the 32-byte
 * result to device memory (dev_out, caller-owned, 8-byte aligned; SCAN_EINVAL
 * otherwise, checked before any CUDA call) and returns without waiting.  An
 * empty predicate writes zeros without a kernel.  Check scan_column_status
 * afterwards for device errors. */
scan_status scan_run_async(scan_column *col, scan_pred pred, scan_strategy strategy, void *stream,
                           scan_result *dev_out);

/* Wait for the stream and report (then clear) device-side error flags of the
 * column's kernels: SCAN_OK or SCAN_ETIMEOUT. */
scan_status scan_column_status(scan_column *col, void *stream);

/* ------------------------------------------------- materializing select */

/* Materializing select (paper §3: "a materializing select" beside the count
 * aggregates; §4 "Branch": the branchy and predicated forms of that select).
 * Writes the positions i, in increasing order, of the values with
 * pred.lo <= v_i < pred.hi as uint32 to dev_positions (device memory, at
 * least `capacity` of them; may be NULL when capacity is 0) and the full
 * number of matches to *host_count.  Only the first min(count, capacity)
 * positions are written, so a count above capacity tells the caller how much
 * to allocate for a second call.  strategy: SCAN_BRANCHFREE (every 32-value
 * row runs the predicated store) or SCAN_BRANCHY (a warp vote per row skips
 * rows without a match); SCAN_AUTO means branch-free; the zone-skip
 * strategies are SCAN_EINVAL.  Both give the same positions.  One read of
 * the packed column; calls on one column must be ordered on one stream.
 * Waits for the stream; SCAN_ETIMEOUT if a bounded device wait gave up. */
scan_status scan_select(scan_column *col, scan_pred pred, scan_strategy strategy, uint32_t *dev_positions,
                        uint64_t capacity, void *stream, uint64_t *host_count);

/* As scan_select, but the count goes to device memory (8 bytes) and the call
 * returns without waiting; check scan_column_status afterwards. */
scan_status scan_select_async(scan_column *col, scan_pred pred, scan_strategy strategy,
                              uint32_t *dev_positions, uint64_t capacity, void *stream, uint64_t *dev_count);

/* ---------------------------------------------- conjunctive predicates */

/* Conjunctive scan over k >= 1 columns of one table (the problem of paper §2
 * over rows shared by several columns): COUNT of the rows i with
 * preds[c].lo <= v_c,i < preds[c].hi for every column c, and SUM of the
 * aggregate column's values over those rows (0 when agg is NULL; agg may be
 * one of cols).  All columns lane-interleaved and of equal length.  One pass
 * per predicate column builds a selection vector (a 32-bit row mask per lane
 * and block) in the given order -- later columns skip the decode of blocks
 * whose selection is already empty, so the most selective column first is
 * fastest -- and one pass aggregates over it.  blocks_scanned = blocks of
 * the aggregate column decoded.  strategy: SCAN_AUTO or SCAN_BRANCHFREE.
 * The selection vector (n/8 bytes) is kept with the result column (agg, else
 * cols[0]) for later calls.  Calls sharing a column must be ordered on one
 * stream; waits for the stream. */
scan_status scan_conj(scan_column *const *cols, const scan_pred *preds, uint32_t k, scan_column *agg,
                      scan_strategy strategy, void *stream, scan_result *host_out);

/* As scan_conj, but the 32-byte result goes to device memory and the call
 * returns without waiting; check scan_column_status on the aggregate column
 * (or cols[0] when agg is NULL) afterwards. */
scan_status scan_conj_async(scan_column *const *cols, const scan_pred *preds, uint32_t k, scan_column *agg,
                            scan_strategy strategy, void *stream, scan_result *dev_out);

/* -------------------------------------------------------------- batches */

typedef struct scan_batch scan_batch; /* opaque: a planned batch of column scans */

/* Plan a batch over `ncols` columns (the paper has no batched form; this
 * runs thousands of column scans as one CUDA-graph launch).  Every column's
 * blocks are cut into tiles (by default about 6 KB); columns are grouped by
 * (predicate flavour, width) and each group is served by one width-specialised
 * persistent kernel.  Groups of 16 us or more by the bandwidth law are recorded
 * as two concurrent chains of one graph: the narrow half of their widths
 * ascending, the wide half descending, so that a decode-bound and a
 * bandwidth-bound kernel share every SM (two CTAs per SM); shorter groups run
 * on six more chains, with grids in proportion to their law time.  Warps pop
 * `tiles_per_pop` consecutive tiles per
 * atomic (0 = chosen per group: at least 4, about four pops per warp).
 * strategies[i] picks column i's flavour and whether it skips blocks by zone
 * map (NULL = SCAN_BRANCHFREE for all; SCAN_AUTO counts as branch-free).
 * Zone-skip columns need a built zone map.  The columns must outlive the plan.
 * The first scan_batch_exec records the CUDA graph (copy descriptors, reset
 * results, kernels) that later calls replay. */
scan_status scan_batch_create(scan_column *const *cols, uint32_t ncols,
                              const scan_strategy *strategies, uint32_t tiles_per_pop,
                              void *stream, scan_batch **out);

/* Run the plan with one predicate per column.  host_out (ncols results, may
 * be NULL) is filled after the stream is synchronised; dev_out (ncols results
 * in device memory, may be NULL) is written asynchronously.  Results equal
 * scan_run's bit for bit.  SCAN_ETIMEOUT if a bounded device wait gave up
 * (reported here when host_out is given; a caller that asks for dev_out only
 * checks scan_batch_status). */
scan_status scan_batch_exec(scan_batch *batch, const scan_pred *preds, void *stream,
                            scan_result *host_out, scan_result *dev_out);

/* Autotune the batch's width-group kernels on these predicates (no paper
 * counterpart; the shapes never change a result).  Two phases: every width
 * group's kernel is timed alone (`reps` launches on `stream` after a warm-up)
 * with the rule and every candidate shape of its flavour and width, keeping
 * the three fastest; then, largest group first, each finalist is tried in the
 * whole graph replay (median of 2 * reps + 1) with the other groups' shapes
 * fixed, and kept only if the replay gets faster by more than 0.3% -- the
 * groups overlap on the graph's branches, so a group's time alone does not
 * predict the replay.  The result is kept only if it beats the rule's replay
 * measured again, else every group goes back to the rule.  Installed in the
 * process-wide batch shape table; the batch is laid out again.  Blocking.
 * *groups_tuned gets the number of groups whose shape changed, *rule_us and
 * *tuned_us (may be NULL) the replay times with the rule and the installed
 * shapes.  Results are unaffected. */
scan_status scan_batch_autotune(scan_batch *batch, const scan_pred *preds, uint32_t reps, void *stream,
                                uint32_t *groups_tuned, float *rule_us, float *tuned_us);

/* Status of the plan's last replay on `stream` (no paper counterpart: the
 * error path of a bounded device wait): synchronises the stream and returns
 * SCAN_ETIMEOUT if a device-side wait of that replay gave up, else SCAN_OK.
 * For callers that run scan_batch_exec with dev_out only; the next replay
 * clears the status. */
scan_status scan_batch_status(scan_batch *batch, void *stream);

/* Free the plan (synchronises the device first). */
scan_status scan_batch_destroy(scan_batch *batch);

/* Change the strategy of every column of the plan (re-lays out the tiles;
 * the next scan_batch_exec records a new graph).  Synchronises the device. */
scan_status scan_batch_set_strategies(scan_batch *batch, const scan_strategy *strategies);

/* Planner features of every column for these predicates, computed on the GPU
 * into dev_features (ncols x 4 floats, column order):
 *   f0 = b/32; f1 = log2(max(N,1))/31;
 *   f2 = (log10(max(sigma_hat, 1e-5)) + 5)/5, sigma_hat = matches/values over up
 *        to 32 evenly spaced blocks (an exact sample of the predicate);
 *   f3 = 1 - mean_k (max_k - min_k + 1)/(colmax - colmin + 1) from the zone map
 *        (0 without one): ~0 for shuffled, ~1 for sorted columns.
 * Asynchronous after one stream synchronisation. */
scan_status scan_batch_features(scan_batch *batch, const scan_pred *preds, void *stream,
                                float *dev_features);

/* Law-based plan (paper §2 Eq. 2 per strategy), the fallback when no trained
 * planner is loaded: strategy s costs max(bytes_s/beta, values_s/T_dec[s]),
 * where a zone skip reads the zone map plus a fraction min(1, sigma_hat +
 * (1 - c) + 2/blocks) of the blocks.  t_dec_values_per_s[4] (host) are the
 * fitted T_dec of branch-free, branchy, zone-skip branch-free, zone-skip
 * branchy; dev_choice (ncols int32, device) gets 0..3 in that order. */
scan_status scan_batch_law_choose(scan_batch *batch, const float *dev_features,
                                  float beta_bytes_per_s, const float *t_dec_values_per_s,
                                  void *stream, int32_t *dev_choice);
/* The same law's predicted times, as natural-log milliseconds: dev_log_ms
 * (ncols x 4 float32, device, row = the column's position in the batch) gets
 * log(1e3 * max(bytes_s/beta, values_s/T_dec[s])) per strategy, and 30 for a
 * zone strategy of a column without a zone map.  The prior of
 * scan_planner_choose_prior.  Errors as scan_batch_law_choose. */
scan_status scan_batch_law_times(scan_batch *batch, const float *dev_features,
                                 float beta_bytes_per_s, const float *t_dec_values_per_s,
                                 void *stream, float *dev_log_ms);

/* One-shot batch: plan, run once with host results, free. */
scan_status scan_batch_run(const scan_column *const *cols, const scan_pred *preds, uint32_t ncols,
                           const scan_strategy *strategies, void *stream, scan_result *host_out);

/* ------------------------------------------------------ learned planner */

/* The learned planner (the paper has none; it picks among the paper's
 * strategies, which all return the same result): an FP32
 * network 4 -> 64 -> 64 -> n_strategies with ReLU hidden layers that predicts
 * the log time of each strategy from the four features above; the strategy
 * with the smallest prediction is chosen.  Every strategy returns identical
 * results, so the planner only changes speed.  Forward, backward (mean
 * squared error) and Adam run in this library's CUDA kernels; parameters are
 * one flat float array [W1 (4x64), b1, W2 (64x64), b2, W3 (64xS), b3], each W
 * row-major (fan_in, fan_out); He-uniform initial weights from splitmix64(seed),
 * zero biases. */
typedef struct scan_planner scan_planner;

scan_status scan_planner_create(uint32_t n_strategies, uint64_t seed, scan_planner **out);
scan_status scan_planner_destroy(scan_planner *planner);
uint64_t scan_planner_param_count(const scan_planner *planner);
/* Copy parameters to / from host memory (param_count floats); setting them
 * resets the Adam state. */
scan_status scan_planner_get_params(const scan_planner *planner, float *host_params);
scan_status scan_planner_set_params(scan_planner *planner, const float *host_params);
/* dev_y[rows x S] = network(dev_x[rows x 4]). */
scan_status scan_planner_forward(scan_planner *planner, const float *dev_x, uint32_t rows, float *dev_y,
                                 void *stream);
/* Gradients of mean((y - t)^2) with respect to every parameter into dev_grads
 * (param_count floats, may be NULL); *host_loss (may be NULL) gets the loss
 * after a stream synchronisation. */
scan_status scan_planner_gradients(scan_planner *planner, const float *dev_x, const float *dev_t,
                                   uint32_t rows, float *dev_grads, void *stream, float *host_loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at learning rate lr. */
scan_status scan_planner_train_step(scan_planner *planner, const float *dev_x, const float *dev_t,
                                    uint32_t rows, float lr, void *stream, float *host_loss);
/* dev_choice[rows] = argmin over strategies of the predicted log time. */
scan_status scan_planner_choose(scan_planner *planner, const float *dev_x, uint32_t rows,
                                int32_t *dev_choice, void *stream);
/* As scan_planner_choose, but each row gets the first strategy in index
 * order (branch-free, branchy, zone-skip branch-free, zone-skip branchy)
 * whose predicted log time is within `margin` (>= 0) of the row's minimum --
 * e.g. the network's RMS error in log time, so that the plan leaves a
 * simpler strategy only for a predicted gain larger than the model's own
 * error.  margin 0 is scan_planner_choose. */
scan_status scan_planner_choose_margin(scan_planner *planner, const float *dev_x, uint32_t rows,
                                       float margin, int32_t *dev_choice, void *stream);
/* As scan_planner_choose_margin, on the network's output plus a prior:
 * row n's predicted log time of strategy s is y[n][s] + dev_prior[n*S + s].
 * With the law's log times as the prior (scan_batch_law_times, or an affine
 * calibration of them per strategy) and a network trained on the labels
 * minus that prior, the network learns a correction to the bandwidth law of
 * paper §2 (Eq. 2) instead of the whole time; a network whose output is zero
 * gives the prior's own plan.  dev_prior: rows x S float32, device,
 * row-major.  Errors: SCAN_EINVAL for NULL pointers or a negative margin. */
scan_status scan_planner_choose_prior(scan_planner *planner, const float *dev_x, uint32_t rows,
                                      float margin, const float *dev_prior, int32_t *dev_choice,
                                      void *stream);

/* The law as the fallback and the judge (spec planner; the paper's law,
 * §2 Eq. 2, gives dev_fallback and dev_fallback_log_ms, e.g. from
 * scan_batch_law_choose and scan_batch_law_times): per row, the fallback's
 * strategy, unless (1) the row's features lie inside host_feature_box (8
 * floats: the 4 lower bounds, then the 4 upper bounds of the features the
 * network was trained on; NULL = no box) and (2) the strategy the network
 * predicts fastest among the available ones (fallback log time < 29) is
 * predicted faster than the fallback's by more than `margin` in log time.
 * With margin = the network's RMS error on its labels, noise alone rarely
 * moves a column off the law's plan, and the box keeps the network from
 * extrapolating.  dev_x rows x 4, dev_fallback_log_ms rows x S, int32 out. */
scan_status scan_planner_choose_guarded(scan_planner *planner, const float *dev_x, uint32_t rows, float margin,
                                        const int32_t *dev_fallback, const float *dev_fallback_log_ms,
                                        const float *host_feature_box, int32_t *dev_choice, void *stream);
/* Binary checkpoint: 16-byte header (magic, version 1, S, count) + floats. */
scan_status scan_planner_save(const scan_planner *planner, const char *path);
scan_status scan_planner_load(scan_planner *planner, const char *path);

/* -------------------------------------------------------------- serving */

/* A scan server (the paper has none): continuous
 * batching of COUNT/SUM queries against a device-resident table of columns.
 * A query names n table columns (ids into `cols`), each with its own
 * predicate.  Admission is by device memory: each of `slots` in-flight
 * batches owns device_bytes_per_slot bytes of descriptors and results (112
 * bytes per column scan), and a query waits in the queue until a slot with
 * room for all its scans frees up; a dispatcher thread packs every waiting
 * query that fits into one batched launch on that slot's stream, so batches
 * overlap on the device while new queries keep arriving; a completion thread
 * retires batches in launch order.  Zone maps are used wherever a column has
 * one.  Each result equals the query's result run alone, bit for bit.  The
 * table's columns must outlive the server. */
typedef struct scan_server scan_server;

scan_status scan_server_create(scan_column *const *cols, uint32_t ncols, uint32_t slots,
                               uint64_t device_bytes_per_slot, uint32_t max_queue,
                               scan_server **out);
/* Enqueue a query; SCAN_EBUSY when max_queue queries already wait. */
scan_status scan_server_submit(scan_server *server, const uint32_t *col_ids, const scan_pred *preds,
                               uint32_t n, uint64_t *query_id);
/* Enqueue nqueries queries at once (all or none): query k uses entries
 * offsets[k] .. offsets[k+1]-1 of col_ids/preds; ids go to query_ids[k]. */
scan_status scan_server_submit_many(scan_server *server, uint32_t nqueries, const uint32_t *offsets,
                                    const uint32_t *col_ids, const scan_pred *preds, uint64_t *query_ids);
/* *done = 1 and results copied (n >= the query's column count) once the
 * query has completed; wait != 0 blocks until then.  A collected query id is
 * forgotten.  *latency_us (may be NULL) = completion - submission time. */
scan_status scan_server_poll(scan_server *server, uint64_t query_id, int wait, scan_result *out,
                             uint32_t n, double *latency_us, int *done);
scan_status scan_server_stats(scan_server *server, uint64_t *batches, uint64_t *column_scans,
                              uint64_t *rejected, uint32_t *queued);
/* Stop the threads, wait for batches in flight, free everything. */
scan_status scan_server_destroy(scan_server *server);

/* ------------------------------------------------------ no allocation */

/* The paper has no counterpart to this call; it is an integration aid.
 * The same fused full scan as scan_run_async on a caller-owned packed buffer
 * (scan_packed_words(n, b) words, 16-byte aligned), for callers that cannot
 * allocate device memory when they scan: latency-bound loops that must not
 * take the allocator's implicit synchronisation, engines that manage a fixed
 * memory budget through their own sub-allocator, and plug-ins whose host
 * process owns the device memory.  It calls no cudaMalloc/cudaFree and no
 * allocating library routine.  Its grid-reduction scratch is a statically
 * sized device array of 16 KiB + 64 bytes inside this library (room for 1024
 * CTAs, one per SM), held by every GPU that loads the library until exit; a
 * GPU with more SMs than that is refused with SCAN_EINVAL.
 *   - Outputs: *dev_out gets the 32-byte result, *dev_status gets 0 or error
 *     bits (nonzero means a bounded device wait gave up and the result is not
 *     valid); both are caller-owned device memory, written asynchronously;
 *     dev_out must be 8-byte and dev_status 4-byte aligned (checked, with
 *     the other arguments, before any CUDA call).
 *   - strategy: SCAN_AUTO / SCAN_BRANCHFREE or SCAN_BRANCHY; zone-skip
 *     strategies need a zone map and are refused with SCAN_EINVAL.
 *   - The first call on each device looks up the scratch array's address
 *     (cudaGetSymbolAddress with that device current); make that first call
 *     before any stream capture begins.
 *   - Every call on a device shares the one scratch array and clears its
 *     ticket at the start of the call: calls whose kernels overlap on the GPU
 *     (different streams, no ordering between them) race and give wrong
 *     results.  Order them on one stream or with events.
 * Errors: SCAN_EINVAL for bad width/base, n > 2^31, NULL or misaligned
 * pointers; SCAN_ECUDA if a launch or memset fails. */
scan_status scan_run_packed_noalloc(const uint32_t *dev_packed, uint64_t n, uint32_t b,
                                    uint32_t base, scan_pred pred, scan_strategy strategy,
                                    void *stream, scan_result *dev_out, uint32_t *dev_status);

/* --------------------------------------------------------------- probes */

/* Read-only bandwidth probe (paper §3: beta is the empirical sequential-read
 * maximum): every byte of dev_buf (16-byte aligned, bytes a multiple of 16)
 * is read once and folded into a checksum written to *dev_out (8 bytes). */
scan_status scan_probe_read(const void *dev_buf, uint64_t bytes, void *stream, uint64_t *dev_out);

/* STREAM triad (paper §3 measures beta per machine as STREAM-Triad as well as
 * the read maximum): dev_a[i] = dev_b[i] + s * dev_c[i] for i < n, each
 * element computed as one fused multiply-add.  All three arrays are caller-
 * owned device memory, 16-byte aligned; n is a multiple of 4 (n = 0 does
 * nothing and accepts NULL arrays).  12 bytes move per element.
 * Asynchronous on `stream`.
 * Errors: SCAN_EINVAL for NULL or misaligned arrays or n not a multiple of 4;
 * SCAN_ECUDA if the launch fails. */
scan_status scan_probe_triad(float *dev_a, const float *dev_b, const float *dev_c, float s, uint64_t n,
                             void *stream);

/* Failure-path check: one warp waits, with the same bounded wait every
 * pipeline uses, on a transaction barrier nothing ever completes.  The wait
 * gives up after limit_ns (at most 1 s) and the call returns SCAN_ETIMEOUT;
 * the CUDA context stays usable.  Any other status means the timeout path is
 * broken. */
scan_status scan_selftest_wait_timeout(uint64_t limit_ns, void *stream);

/* Failure-path check of the select's waits on other CTAs (no paper
 * counterpart; a test hook): runs the select over `col` with a wait bound of
 * limit_ns (at most 1 s) while CTA 0 never publishes its totals, so every
 * other CTA's bounded wait must give up, set the status, let its copies land
 * and return.  Returns SCAN_ETIMEOUT when that happened (the status is
 * cleared and the context stays usable); any other status means the path is
 * broken.  Nothing is written. */
scan_status scan_selftest_select_timeout(scan_column *col, uint64_t limit_ns, void *stream);

/* Number of SMs, the persistent grid size and the current shape (tuned or
 * the built-in rule) of the branch-free full scan at width b. */
scan_status scan_launch_shape(uint32_t b, uint32_t *sms, uint32_t *ctas, uint32_t *warps_per_cta,
                              uint32_t *blocks_per_tile, uint32_t *stages);

/* ------------------------------------------------------ launch shapes */

/* Launch shape of a persistent scan kernel (no paper counterpart: the paper's
 * single-thread decoders have no launch geometry; the shapes only change how
 * the fused scan of §3 is spread over the GPU, never its result).  One CTA per
 * SM of `warps` warps; each warp streams tiles of `tile_blocks` 1024-value
 * blocks through `stages` shared-memory slots (the zone-skip kernels pop
 * `tile_blocks` candidate blocks at a time); vote_rows = 1 makes the branchy
 * kernel vote once per row of a thread's lanes instead of once per value, and
 * vote_rows = 2 does the same with each row written as one PTX block (tests
 * OR-ed into one predicate, one vote, one uniform branch), vote_rows = 3 with
 * two rows per block (both rows' tests and votes before either branch);
 * vec_lanes is how many lanes a thread reads as one vector per row: 0 (the
 * width's default: 4 for b <= 16, else 2) or 2 for full scans at b = 9..16,
 * whose smaller warp step lets 16 warps fit.  Legal shapes: full scans 1..16
 * warps, zone-skip scans 1..8; 1..6 stages; tile_blocks a positive multiple of
 * the warp step (vec_lanes blocks), at most 64 (full) or 32 (zone skip);
 * vote_rows only for SCAN_BRANCHY at b <= 21; warps * stages * (tile_blocks
 * * 128 * b + 12) <= 226 KB (the kernels keep up to 1 KB of static shared
 * memory). */
typedef struct {
    uint32_t warps, stages, tile_blocks, vote_rows, vec_lanes;
} scan_shape;

/* Tuning outcome for one (strategy, b): the installed shape and the rule's,
 * their mean times per scan on the tuning column, and the candidates timed. */
typedef struct {
    scan_shape best, rule;
    float best_us, rule_us;
    uint32_t candidates;
} scan_tune_result;

/* Shapes are kept per (kernel, b) for four kernels: SCAN_AUTO/SCAN_BRANCHFREE
 * (branch-free full scan), SCAN_BRANCHY, SCAN_ZONE_SKIP_BF (with
 * SCAN_ZONE_AGG_BF) and SCAN_ZONE_SKIP_BR (with SCAN_ZONE_AGG_BR); every
 * later launch of that kernel at that width uses the installed shape.  The
 * table is process-wide; changing it while scans are being enqueued on other
 * threads is safe, but a scan picks up whichever shape is current when it is
 * enqueued.  Every call below returns SCAN_EINVAL for a bad width, strategy or
 * shape (scan_last_error names the rule). */
scan_status scan_shape_get(uint32_t b, scan_strategy strategy, scan_shape *out);
/* Install `shape` (validated), or the built-in rule again if shape is NULL. */
scan_status scan_shape_set(uint32_t b, scan_strategy strategy, const scan_shape *shape);
/* The tuner's candidate shapes for (strategy, b): *count gets their number,
 * out (may be NULL) the first min(capacity, count) of them. */
scan_status scan_shape_candidates(uint32_t b, scan_strategy strategy, scan_shape *out, uint32_t capacity,
                                  uint32_t *count);
/* Autotune the kernel of `strategy` at col's width: time every candidate on
 * this column and predicate (`reps` back-to-back scans each, on `stream`),
 * re-time the three fastest against the rule three times, interleaved, and
 * install the fastest if it beats the rule (otherwise the rule stays).
 * Blocking.  Tune on a column larger than L2 (at least 2^26 values at small
 * b) so that the copies stream from HBM, with a predicate that selects
 * something; zone-skip strategies need a built zone map.  The column's
 * results are unaffected.  SCAN_ENOMEM / SCAN_ECUDA / SCAN_ETIMEOUT as for
 * scans; on failure the previous shape stays installed. */
scan_status scan_autotune_column(scan_column *col, scan_pred pred, scan_strategy strategy, uint32_t reps,
                                 void *stream, scan_tune_result *out);
/* Write the tuned shapes to `path`, a versioned text file: a "gbscan-shapes 3"
 * line, a "device <name> <SMs>" line, then one "kind b warps stages
 * tile_blocks vote_rows vec_lanes tuned_us rule_us" line per tuned (kernel,
 * b). */
scan_status scan_autotune_save(const char *path);
/* Replace the installed shapes with those of a file written by
 * scan_autotune_save.  All or nothing: a wrong magic or version, a file tuned
 * on another device (name or SM count), an unknown kernel, an illegal shape,
 * a duplicate or a malformed line returns SCAN_EINVAL with the line number in
 * scan_last_error and leaves the installed shapes unchanged. */
scan_status scan_autotune_load(const char *path);
/* Every kernel back to the built-in rule. */
scan_status scan_autotune_reset(void);

/* Shapes of the batched kernels, one per (predicate flavour, b): every width
 * group of a batch launches one kernel with its width's shape (tile_blocks =
 * blocks per batch tile; vote_rows must be 0).  Legal: 1..16 warps, 1..6
 * stages, tile_blocks a multiple of the warp step and at most 64, warps *
 * stages * (tile_blocks * 128 * b + 24) <= 226 KB, vec_lanes = 0.  Shapes
 * above 112 KB of slots leave no room for a second CTA on the SM and lose the
 * overlap of the two chains; the candidates stay below it.  branchy = 0 for the
 * branch-free kernel, 1 for the branchy one.  They are saved and loaded with
 * the others ("batch_bf" / "batch_br" lines).  A batch picks up shape
 * changes when it is created, when its strategies are set, or when it is
 * tuned. */
scan_status scan_batch_shape_get(uint32_t b, int branchy, scan_shape *out);
scan_status scan_batch_shape_set(uint32_t b, int branchy, const scan_shape *shape);
scan_status scan_batch_shape_candidates(uint32_t b, int branchy, scan_shape *out, uint32_t capacity,
                                        uint32_t *count);


#ifdef __cplusplus
}
#endif
#endif /* GBSCAN_H */
