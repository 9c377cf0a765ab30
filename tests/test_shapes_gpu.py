"""Every launch shape the autotuner may install gives the oracle's result
(bit-exact COUNT/SUM, and the blocks read of zone skipping), at every width,
for all four tunable kernels; the tuner itself installs one of its candidates
(or keeps the rule) and leaves results exact; its cache round-trips on the
device it was tuned on."""
import numpy as np
import pytest

import oracle
import synth
from paper_2606_22423_gb300 import gbscan

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KINDS = {"branchfree": ["branchfree"], "branchy": ["branchy"], "zone_bf": ["zone_bf", "zone_agg_bf"],
         "zone_br": ["zone_br", "zone_agg_br"]}


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.init()
    gbscan.load()
    gbscan.autotune_reset()
    yield
    gbscan.autotune_reset()


@pytest.mark.parametrize("b", range(1, 33))
def test_every_candidate_shape_matches_the_oracle(b):
    base = min(77, (1 << 32) - (1 << b))
    n = 300 * 1024 + 555                      # several tiles at every candidate shape, ragged tail
    uni = synth.uniform_values(synth.seed_for(90, b), n, b, base)
    clu = synth.clustered_values(synth.seed_for(90, b, 1), n, b, 0.01, base)
    cols = {"uniform": gbscan.Column.from_host(uni, b, base), "clustered": gbscan.Column.from_host(clu, b, base)}
    vals = {"uniform": uni, "clustered": clu}
    for c in cols.values():
        c.zonemap_build()
    preds = [synth.pick_range(synth.seed_for(90, b, 2 + i), b, s, base) for i, s in enumerate([0.01, 0.6])]
    want, touched = {}, {}
    for name, v in vals.items():
        words = oracle.pack(v, b, base)
        zmin, zmax = oracle.zonemap(words, n, b, base)
        for lo, hi in preds:
            want[(name, lo, hi)] = oracle.scan_values(v, lo, hi)
            touched[(name, lo, hi)] = oracle.scan_zoneskip(words, zmin, zmax, n, b, base, lo, hi)[2]
    for kind, strategies in KINDS.items():
        name = "uniform" if kind in ("branchfree", "branchy") else "clustered"
        for shape in gbscan.shape_candidates(b, kind):
            gbscan.shape_set(b, kind, shape)
            for lo, hi in preds:
                for st in strategies:
                    r = cols[name].run(lo, hi, st)
                    assert r.pair() == want[(name, lo, hi)], (b, kind, shape, st, lo, hi)
                    if st in ("zone_bf", "zone_br"):
                        assert r.blocks_scanned == touched[(name, lo, hi)], (b, kind, shape)
                    elif st in ("branchfree", "branchy"):
                        assert r.blocks_scanned == (n + 1023) // 1024
        gbscan.shape_set(b, kind, None)
    for c in cols.values():
        c.close()


@pytest.mark.parametrize("b,strategy", [(6, "branchy"), (13, "branchfree"), (24, "branchy"), (16, "zone_bf")])
def test_autotune_installs_a_candidate_and_stays_exact(b, strategy, tmp_path):
    gbscan.autotune_reset()
    n = (1 << 24) + 321
    v = (synth.clustered_values(synth.seed_for(91, b), n, b, 0.01) if strategy.startswith("zone")
         else synth.uniform_values(synth.seed_for(91, b), n, b))
    col = gbscan.Column.from_host(v, b)
    col.zonemap_build()
    lo, hi = synth.pick_range(synth.seed_for(91, b, 1), b, 0.3)
    res = col.autotune(lo, hi, strategy, reps=2)
    cands = gbscan.shape_candidates(b, strategy)
    assert res["candidates"] == len(cands)
    assert res["best"] in cands or res["best"] == res["rule"]
    assert res["best_us"] <= res["rule_us"] and res["best_us"] > 0
    assert gbscan.shape_get(b, strategy) == res["best"]
    for s in (0.001, 0.3, 1.0):
        plo, phi = synth.pick_range(synth.seed_for(91, b, 7), b, s)
        assert col.run(plo, phi, strategy).pair() == oracle.scan_values(v, plo, phi)
    path = str(tmp_path / "shapes.txt")
    gbscan.autotune_save(path)
    text = open(path).read()
    assert "device " in text and "none 0" not in text          # tied to this GPU
    gbscan.autotune_reset()
    gbscan.autotune_load(path)
    assert gbscan.shape_get(b, strategy) == res["best"]
    gbscan.autotune_reset()
    col.close()


def test_autotune_rejects_an_empty_predicate_and_keeps_the_old_shape():
    gbscan.autotune_reset()
    v = synth.uniform_values(5, 1 << 16, 10)
    col = gbscan.Column.from_host(v, 10)
    keep = dict(warps=12, stages=2, tile_blocks=4, vote_rows=0, vec_lanes=0)
    gbscan.shape_set(10, "branchfree", keep)
    with pytest.raises(gbscan.ScanError) as e:
        col.autotune(500, 500, "branchfree")
    assert e.value.status == gbscan.SCAN_EINVAL
    assert gbscan.shape_get(10, "branchfree") == keep
    assert col.run(3, 900).pair() == oracle.scan_values(v, 3, 900)
    gbscan.autotune_reset()
    col.close()
    assert np.all(v < 1024)


@pytest.mark.parametrize("b", [1, 4, 8, 13, 16, 24, 32])
def test_single_slot_shapes_match_the_oracle(b):
    """Single-slot rings (stages = 1, legal for any full scan) at several tile sizes and
    warp counts, on a column of several tile rounds with a ragged tail: the oracle's
    COUNT/SUM, every block read, both flavours."""
    gbscan.autotune_reset()
    step = 4 if b <= 16 else 2
    base = min(77, (1 << 32) - (1 << b))
    n = 200 * 1024 + 71
    v = synth.uniform_values(synth.seed_for(92, b), n, b, base)
    col = gbscan.Column.from_host(v, b, base)
    preds = [synth.pick_range(synth.seed_for(92, b, i), b, s, base) for i, s in enumerate([0.001, 0.1, 1.0])]
    for warps, tiles in ((8, step), (12, 2 * step), (16, 4 * step)):
        if warps * (tiles * 128 * b + 12) > 226 * 1024:
            continue
        for st in ("branchfree", "branchy"):
            gbscan.shape_set(b, st, dict(warps=warps, stages=1, tile_blocks=tiles, vote_rows=0, vec_lanes=0))
            for lo, hi in preds:
                r = col.run(lo, hi, st)
                assert r.pair() == oracle.scan_values(v, lo, hi), (b, st, warps, tiles, lo, hi)
                assert r.blocks_scanned == (n + 1023) // 1024
            gbscan.shape_set(b, st, None)
    col.close()
