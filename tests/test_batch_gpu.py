"""Batched scan parity: one persistent launch over many columns of mixed
width, length, order and strategy must give, column by column, exactly the
oracle's COUNT/SUM (and the single-column scan's blocks-read count)."""
import numpy as np
import pytest

import oracle
import synth
from paper_2606_22423_gb300 import gbscan

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ALL = ["branchfree", "branchy", "zone_bf", "zone_br"]


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.init()
    return gbscan.load()


def _make_columns(ncols, seed, max_len=40_000):
    rng = np.random.default_rng(seed)
    cols, vals, meta = [], [], []
    for i in range(ncols):
        b = int(rng.integers(1, 33))
        n = int(rng.integers(0, max_len)) if i % 7 else int(rng.integers(1, 3000))
        base = 0 if b == 32 else int(rng.integers(0, min(1 << 20, (1 << 32) - (1 << b)) + 1))
        s = synth.seed_for(60, i, seed)
        v = (synth.uniform_values(s, n, b, base) if i % 2 else
             synth.clustered_values(s, n, b, [0.0, 0.01, 0.1][i % 3], base))
        c = gbscan.Column.from_host(v, b, base)
        c.zonemap_build()
        cols.append(c)
        vals.append(v)
        meta.append((b, base))
    return cols, vals, meta


def _preds(meta, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i, (b, base) in enumerate(meta):
        if i % 11 == 3:
            out.append((base + 5, base + 5))                       # empty
        elif i % 13 == 4:
            out.append((base - 1, base + (1 << b) + 1))            # full domain
        else:
            sigma = float(synth.log_uniform(rng, 1e-4, 1.0))
            out.append(synth.pick_range(int(rng.integers(1 << 30)), b, sigma, base))
    return out


@pytest.mark.parametrize("mix", ["branchfree", "mixed"])
def test_batch_equals_oracle_and_single_column(mix):
    cols, vals, meta = _make_columns(96, 1)
    strategies = ["branchfree"] * len(cols) if mix == "branchfree" else [ALL[i % 4] for i in range(len(cols))]
    bt = gbscan.Batch(cols, strategies)
    for rep in range(3):                                   # graph replays with new predicates
        preds = _preds(meta, 10 + rep)
        got = bt.run(preds)
        for i, ((lo, hi), v) in enumerate(zip(preds, vals)):
            assert got[i].pair() == oracle.scan_values(v, lo, hi), (i, meta[i], strategies[i])
            single = cols[i].run(lo, hi, strategies[i])
            assert got[i].blocks_scanned == single.blocks_scanned, (i, strategies[i])
    bt.close()
    for c in cols:
        c.close()


def test_batch_pop_sizes_and_one_shot():
    cols, vals, meta = _make_columns(40, 2, max_len=300_000)
    preds = _preds(meta, 5)
    want = [oracle.scan_values(v, lo, hi) for v, (lo, hi) in zip(vals, preds)]
    for pop in [1, 3, 64]:
        bt = gbscan.Batch(cols, None, tiles_per_pop=pop)
        assert [r.pair() for r in bt.run(preds)] == want
        bt.close()
    assert [r.pair() for r in gbscan.scan_batch_run(cols, preds)] == want
    for c in cols:
        c.close()


def test_batch_device_results_and_zone_requirement():
    cols, vals, meta = _make_columns(10, 3)
    preds = _preds(meta, 6)
    bt = gbscan.Batch(cols, ["zone_bf"] * 10)
    out = torch.zeros((10, 4), dtype=torch.int64, device="cuda")
    for _ in range(2):                      # device results only: nothing is copied to the host
        bt.run(preds, dev_out=out, host=False)
        bt.status()                         # syncs; no device wait gave up
        got = out.cpu().numpy()
        for i, (v, (lo, hi)) in enumerate(zip(vals, preds)):
            assert (int(got[i, 0]), int(got[i, 1])) == oracle.scan_values(v, lo, hi)
    # host results after device-only replays come from this replay
    host = bt.run(_preds(meta, 7))
    for i, (v, (lo, hi)) in enumerate(zip(vals, _preds(meta, 7))):
        assert host[i].pair() == oracle.scan_values(v, lo, hi)
    bt.close()
    plain = gbscan.Column.from_host(vals[0], meta[0][0], meta[0][1])
    with pytest.raises(gbscan.ScanError):
        gbscan.Batch([plain], ["zone_bf"])
    plain.close()
    for c in cols:
        c.close()


def test_full_size_batch_4096_columns_against_the_oracle():
    """The batched workload at full size (4096 columns, lengths log-uniform in
    [2^10, 2^26] scaled to 2^31 values in total, b uniform in 1..32, half
    uniform / half sorted with displacement, sigma log-uniform in [1e-4, 1]),
    drawn on the device as the benchmark does: every column's COUNT/SUM under
    every plan equals brute force over the generator's raw values (all 4096
    columns, no sampling)."""
    from concurrent.futures import ThreadPoolExecutor

    spec = synth.batch_spec(synth.seed_for(4))
    cols, raws, preds = [], [], []
    for i, (n, b, p, sigma) in enumerate(spec):
        seed = synth.seed_for(4, i)
        v = (synth.uniform_values_device(seed, n, b) if p is None
             else synth.clustered_values_device(seed, n, b, p))
        c = gbscan.Column.from_device(v, n, b)
        c.zonemap_build()
        cols.append(c)
        raws.append(v.cpu().numpy().view(np.uint32))
        preds.append(synth.pick_range(synth.seed_for(4, i, 1), b, sigma))
        del v
    assert sum(x[0] for x in spec) <= 1 << 31 and len(cols) == 4096
    with ThreadPoolExecutor(16) as ex:
        want = list(ex.map(lambda i: oracle.scan_values(raws[i], *preds[i]), range(len(cols))))
    del raws
    plans = {s: [s] * len(cols) for s in ALL}
    plans["mixed"] = [ALL[i % 4] for i in range(len(cols))]
    for name, strategies in plans.items():
        bt = gbscan.Batch(cols, strategies)
        for _ in range(2):                                  # the graph replayed
            got = bt.run(preds)
            bad = [i for i in range(len(cols)) if got[i].pair() != want[i]]
            assert not bad, (name, bad[:5])
        bt.close()
    for c in cols:
        c.close()
    torch.cuda.empty_cache()


def _width_columns(seed, n):
    """Two columns per width b = 1..32 (uniform; sorted with 1% displaced), n values each."""
    cols, vals = [], []
    for b in range(1, 33):
        for k, v in enumerate([synth.uniform_values(synth.seed_for(61, b, seed), n, b),
                               synth.clustered_values(synth.seed_for(61, b, seed + 1), n, b, 0.01)]):
            c = gbscan.Column.from_host(v, b)
            c.zonemap_build()
            cols.append(c)
            vals.append(v)
    return cols, vals


def test_every_batch_candidate_shape_matches_the_oracle():
    """Every shape the batch tuner may install, for both flavours, with and
    without zone skipping: results equal the oracle's (all candidates of every
    width are run, the i-th candidate of every width in the same batch)."""
    gbscan.autotune_reset()
    n = 150_000 + 77                      # more than two 64-block tiles, ragged tail
    cols, vals = _width_columns(1, n)
    rng = np.random.default_rng(7)
    preds = [synth.pick_range(int(rng.integers(1 << 30)), c.b, float(synth.log_uniform(rng, 1e-3, 1.0)))
             for c in cols]
    want = [oracle.scan_values(v, lo, hi) for v, (lo, hi) in zip(vals, preds)]
    for branchy in (False, True):
        cands = {b: gbscan.batch_shape_candidates(b, branchy) for b in range(1, 33)}
        strategies = [("branchy" if branchy else "branchfree") if i % 2 == 0 else ("zone_br" if branchy else "zone_bf")
                      for i in range(len(cols))]
        for ci in range(max(len(c) for c in cands.values())):
            for b in range(1, 33):
                gbscan.batch_shape_set(b, branchy, cands[b][ci % len(cands[b])])
            bt = gbscan.Batch(cols, strategies)
            got = bt.run(preds)
            bad = [i for i in range(len(cols)) if got[i].pair() != want[i]]
            assert not bad, (branchy, ci, [(cols[i].b, strategies[i]) for i in bad[:4]])
            bt.close()
    gbscan.autotune_reset()
    for c in cols:
        c.close()


def test_batch_autotune_installs_group_shapes_and_stays_exact():
    gbscan.autotune_reset()
    cols, vals = _width_columns(3, 1 << 18)
    strategies = ["branchfree" if i % 2 == 0 else "zone_br" for i in range(len(cols))]
    rng = np.random.default_rng(8)
    preds = [synth.pick_range(int(rng.integers(1 << 30)), c.b, float(synth.log_uniform(rng, 1e-4, 1.0)))
             for c in cols]
    bt = gbscan.Batch(cols, strategies)
    res = bt.autotune(preds, reps=2)
    assert 0 <= res["groups"] <= 64 and 0 < res["tuned_us"] <= res["rule_us"]
    for b in (1, 16, 32):
        assert gbscan.batch_shape_get(b, False) in gbscan.batch_shape_candidates(b, False) + \
            [dict(warps=8, stages=2, tile_blocks=gbscan.batch_shape_get(b, False)["tile_blocks"], vote_rows=0,
                  vec_lanes=0)]
    for rep in range(2):
        got = bt.run(preds)
        assert [r.pair() for r in got] == [oracle.scan_values(v, lo, hi) for v, (lo, hi) in zip(vals, preds)]
    bt.close()
    gbscan.autotune_reset()
    for c in cols:
        c.close()
