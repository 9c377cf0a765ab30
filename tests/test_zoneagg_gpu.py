"""Parity of the metadata-answered zone scan (SCAN_ZONE_AGG_*) with the oracle:
COUNT, SUM and the number of blocks read equal oracle_scan_zoneagg exactly, the
per-block sums equal the oracle's, and on sorted data at most two blocks are
read whatever the selectivity."""
import numpy as np
import pytest

import oracle
import synth
from paper_2606_22423_gb300 import gbscan
from tests._cudart import d2h_u32

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

STRATS = ["zone_agg_bf", "zone_agg_br"]


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.init()
    return gbscan.load()


def _d2h_u64(ptr, count):
    return d2h_u32(ptr, 2 * count).view(np.uint64)


def _check(col, v, b, base, preds):
    n = v.size
    words = oracle.pack(v, b, base)
    col.zonemap_build()
    mn, mx = oracle.zonemap(words, n, b, base)
    sums = oracle.blocksums(words, n, b, base)
    np.testing.assert_array_equal(_d2h_u64(col.dev_blocksums, sums.size), sums)
    for lo, hi in preds:
        c, s, t = oracle.scan_zoneagg(words, mn, mx, sums, n, b, base, lo, hi)
        assert (c, s) == oracle.scan_packed(words, n, b, base, lo, hi)
        for strat in STRATS:
            r = col.run(lo, hi, strat)
            assert r.pair() == (c, s), (b, n, lo, hi, strat)
            if max(lo, base) < min(hi, base + (1 << b)):
                assert r.blocks_scanned == t, (strat, r.blocks_scanned, t)


@pytest.mark.parametrize("b", [3, 8, 12, 16, 21, 24, 29, 32])
@pytest.mark.parametrize("p", [0.0, 0.01, None])
def test_zoneagg_matches_oracle(b, p):
    base = 0 if b == 32 else 40
    n = 200 * 1024 + 313
    seed = synth.seed_for(95, b, 0 if p is None else int(p * 100) + 1)
    v = (synth.uniform_values(seed, n, b, base) if p is None else synth.clustered_values(seed, n, b, p, base))
    col = gbscan.Column.from_host(v, b, base)
    preds = [synth.pick_range(synth.seed_for(96, b, i), b, s, base) for i, s in enumerate([1e-4, 0.01, 0.3, 0.9])]
    preds += [(base, base + (1 << b)), (int(v[n // 2]), int(v[n // 2]) + 1), (int(v[n - 1]), int(v[n - 1]) + 2)]
    _check(col, v, b, base, preds)
    col.close()


def test_zoneagg_tail_and_small_columns():
    b = 10
    for n in (1, 500, 1024, 1025, 3 * 1024 + 1000):
        v = synth.clustered_values(synth.seed_for(97, n), n, b, 0.0)
        col = gbscan.Column.from_host(v, b)
        preds = [(0, 1 << b), (int(v[0]), int(v[-1]) + 1), (int(v[-1]), 1 << b), (int(v[n // 2]), int(v[-1]))]
        _check(col, v, b, 0, preds)
        col.close()


def test_zoneagg_needs_a_zonemap_and_lane_layout():
    v = synth.uniform_values(98, 5000, 9)
    col = gbscan.Column.from_host(v, 9)
    with pytest.raises(gbscan.ScanError):
        col.run(0, 100, "zone_agg_bf")
    col.close()
    col = gbscan.Column.from_host(v, 9, layout="rowmajor")
    with pytest.raises(gbscan.ScanError):
        col.run(0, 100, "zone_agg_bf")
    col.close()
    with pytest.raises(gbscan.ScanError):
        gbscan.Batch([gbscan.Column.from_host(v, 9)], ["zone_agg_bf"])


def test_zoneagg_sorted_n2pow30_b16_reads_at_most_two_blocks():
    """The zone-sweep column (N = 2^30 at b = 16, sorted): every predicate is
    answered from metadata plus at most two boundary blocks, with the full
    scan's result."""
    n, b = 1 << 30, 16
    v = synth.clustered_values_device(synth.seed_for(3, 0), n, b, 0.0)
    col = gbscan.Column.from_device(v, n, b)
    del v
    col.zonemap_build()
    for i, sigma in enumerate([1e-4, 0.1, 0.5, 1.0]):
        lo, hi = synth.pick_range(synth.seed_for(99, i), b, sigma)
        full = col.run(lo, hi, "branchfree")
        for strat in STRATS:
            r = col.run(lo, hi, strat)
            assert r.pair() == full.pair()
            assert r.blocks_scanned <= 2
    col.close()
    torch.cuda.empty_cache()
