/* A plain C client of the scan library: no Python, no torch.
 *
 * Reads n uint32 values from a binary file, creates a column from host memory
 * (host-side encode and upload), builds its zone map and runs one predicate
 * with every strategy that needs no extra layout.  Prints one line per
 * strategy: "<strategy> <count> <sum> <blocks_scanned>".  Exit status 0 on
 * success; on a library error it prints the status name and message and exits
 * 1.  The test that runs it compares the lines with the oracle.
 *
 * With a seventh argument it also tunes the branch-free kernel's launch
 * shape on this column, saves the shape cache to that path, resets and
 * reloads it, and scans once more, printing "shape <warps> <stages>
 * <tile_blocks> <vote_rows> <vec_lanes>" and "tuned <count> <sum> <blocks>".
 *
 * usage: c_abi_client <values.bin> <n> <b> <base> <lo> <hi> [shape-cache]
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "gbscan.h"

static int fail(const char *what, scan_status s)
{
    fprintf(stderr, "%s: %s: %s\n", what, scan_status_string(s), scan_last_error());
    return 1;
}

int main(int argc, char **argv)
{
    if (argc != 7 && argc != 8) {
        fprintf(stderr, "usage: %s <values.bin> <n> <b> <base> <lo> <hi> [shape-cache]\n", argv[0]);
        return 2;
    }
    const uint64_t n = strtoull(argv[2], NULL, 10);
    const uint32_t b = (uint32_t)strtoul(argv[3], NULL, 10);
    const uint32_t base = (uint32_t)strtoul(argv[4], NULL, 10);
    scan_pred pred;
    pred.lo = strtoll(argv[5], NULL, 10);
    pred.hi = strtoll(argv[6], NULL, 10);

    uint32_t *v = (uint32_t *)malloc(n ? n * sizeof(uint32_t) : 4);
    FILE *f = fopen(argv[1], "rb");
    if (!v || !f || fread(v, sizeof(uint32_t), n, f) != n) {
        fprintf(stderr, "cannot read %llu values from %s\n", (unsigned long long)n, argv[1]);
        return 2;
    }
    fclose(f);

    scan_column *col = NULL;
    scan_status s = scan_column_create(v, n, b, base, NULL, &col);
    if (s != SCAN_OK) return fail("scan_column_create", s);
    s = scan_zonemap_build(col, NULL);
    if (s != SCAN_OK) return fail("scan_zonemap_build", s);

    const scan_strategy strategies[] = {SCAN_BRANCHFREE, SCAN_BRANCHY, SCAN_ZONE_SKIP_BF, SCAN_ZONE_SKIP_BR,
                                        SCAN_ZONE_AGG_BF, SCAN_ZONE_AGG_BR, SCAN_AUTO};
    for (unsigned i = 0; i < sizeof strategies / sizeof strategies[0]; ++i) {
        scan_result r;
        s = scan_run(col, pred, strategies[i], NULL, &r);
        if (s != SCAN_OK) return fail("scan_run", s);
        printf("%d %lld %lld %llu\n", (int)strategies[i], (long long)r.count, (long long)r.sum,
               (unsigned long long)r.blocks_scanned);
    }
    if (argc == 8) {
        scan_tune_result t;
        s = scan_autotune_column(col, pred, SCAN_BRANCHFREE, 1, NULL, &t);
        if (s != SCAN_OK) return fail("scan_autotune_column", s);
        s = scan_autotune_save(argv[7]);
        if (s != SCAN_OK) return fail("scan_autotune_save", s);
        s = scan_autotune_reset();
        if (s != SCAN_OK) return fail("scan_autotune_reset", s);
        s = scan_autotune_load(argv[7]);
        if (s != SCAN_OK) return fail("scan_autotune_load", s);
        scan_shape sh;
        s = scan_shape_get(b, SCAN_BRANCHFREE, &sh);
        if (s != SCAN_OK) return fail("scan_shape_get", s);
        printf("shape %u %u %u %u %u\n", sh.warps, sh.stages, sh.tile_blocks, sh.vote_rows, sh.vec_lanes);
        scan_result r;
        s = scan_run(col, pred, SCAN_BRANCHFREE, NULL, &r);
        if (s != SCAN_OK) return fail("scan_run", s);
        printf("tuned %lld %lld %llu\n", (long long)r.count, (long long)r.sum, (unsigned long long)r.blocks_scanned);
    }
    s = scan_column_destroy(col);
    if (s != SCAN_OK) return fail("scan_column_destroy", s);
    free(v);
    return 0;
}
