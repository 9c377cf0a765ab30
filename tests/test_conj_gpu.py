"""Parity of the conjunctive multi-column scan with the oracle, through the C ABI:
COUNT and SUM equal oracle_scan_conj exactly; blocks_scanned equals the number
of blocks holding a selected row (computed with numpy from the raw values)."""
import numpy as np
import pytest

import oracle
import synth
from paper_2606_22423_gb300 import gbscan
from tests._cudart import d2h_u32

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.init()
    return gbscan.load()


def _table(n, specs, salt, orders=None):
    vals, cols = [], []
    for i, (b, base) in enumerate(specs):
        seed = synth.seed_for(100, salt, i)
        p = None if orders is None else orders[i]
        v = synth.uniform_values(seed, n, b, base) if p is None else synth.clustered_values(seed, n, b, p, base)
        vals.append(v)
        cols.append(gbscan.Column.from_host(v, b, base))
    return vals, cols


def _expect(vals, specs, preds, agg_i, n):
    m = np.ones(n, bool)
    for v, (lo, hi) in zip(vals, preds):
        m &= (v.astype(np.int64) >= lo) & (v.astype(np.int64) < hi)
    s = int(vals[agg_i][m].astype(np.int64).sum()) if agg_i is not None else 0
    blocks = int(np.any(np.pad(m, (0, (-n) % 1024)).reshape(-1, 1024), axis=1).sum())
    return int(m.sum()), s, blocks


@pytest.mark.parametrize("n", [1, 1000, 1024, 5 * 1024 + 1, 300 * 1024 + 777])
def test_conjunction_matches_oracle(n):
    specs = [(7, 10), (16, 0), (21, 1000), (32, 0), (12, 5)]
    vals, cols = _table(n, specs, n)
    words = [oracle.pack(v, b, base) for v, (b, base) in zip(vals, specs)]
    rng = np.random.default_rng(n)
    for trial in range(4):
        k = 1 + trial % 4
        idx = list(rng.permutation(len(specs))[:k])
        preds = [synth.pick_range(int(rng.integers(1 << 30)), specs[i][0], [0.9, 0.5, 0.3, 0.05][trial], specs[i][1])
                 for i in idx]
        for agg_i in (None, idx[0], 4):
            want = oracle.scan_conj([(words[i], specs[i][0], specs[i][1], lo, hi) for i, (lo, hi) in zip(idx, preds)],
                                    n, None if agg_i is None else (words[agg_i], *specs[agg_i]))
            c, s, blocks = _expect([vals[i] for i in idx], specs, preds, None, n)
            assert want[0] == c
            r = gbscan.scan_conj([cols[i] for i in idx], preds, cols[agg_i] if agg_i is not None else None)
            assert (r.count, r.sum) == want, (n, idx, preds, agg_i)
            if agg_i is not None and n:
                assert r.blocks_scanned == blocks
    for c in cols:
        c.close()


def test_conjunction_edge_cases():
    n = 20 * 1024 + 3
    specs = [(9, 0), (14, 100)]
    vals, cols = _table(n, specs, 1, orders=[0.0, None])
    full = [(0, 1 << 9), (100, 100 + (1 << 14))]
    r = gbscan.scan_conj(cols, full, cols[1])
    assert (r.count, r.sum) == (n, int(vals[1].astype(np.int64).sum()))
    assert gbscan.scan_conj(cols, [(0, 1 << 9), (5, 5)], cols[0]).count == 0          # one empty range
    assert gbscan.scan_conj(cols, [(1 << 9, 1 << 12), (0, 1 << 20)]).count == 0       # outside the domain
    # a selective sorted first column leaves later columns little to decode
    lo = int(vals[0][n // 2])
    r = gbscan.scan_conj(cols, [(lo, lo + 1), (100, 100 + (1 << 13))], cols[1])
    c, s, blocks = _expect(vals, specs, [(lo, lo + 1), (100, 100 + (1 << 13))], 1, n)
    assert (r.count, r.sum, r.blocks_scanned) == (c, s, blocks)
    assert blocks <= 3
    # the asynchronous form writes the same result to device memory
    dres = torch.zeros(4, dtype=torch.int64, device="cuda")
    s_ = torch.cuda.Stream()
    q = gbscan.Conj(cols, [(lo, lo + 1), (100, 100 + (1 << 13))], cols[1])
    q.run_async(dres, s_)
    cols[1].status(s_)
    assert dres.cpu().tolist()[:3] == [c, s, blocks]
    gbscan.Conj(cols, [(0, 1 << 9), (5, 5)], cols[0]).run_async(dres, s_)     # empty: zeros
    torch.cuda.synchronize()
    assert dres.cpu().tolist() == [0, 0, 0, 0]
    for c_ in cols:
        c_.close()


def test_conjunction_rejects_bad_tables():
    a = gbscan.Column.from_host(synth.uniform_values(1, 4096, 8), 8)
    b = gbscan.Column.from_host(synth.uniform_values(2, 4095, 8), 8)
    r = gbscan.Column.from_host(synth.uniform_values(3, 4096, 8), 8, layout="rowmajor")
    for cols in ([a, b], [a, r]):
        with pytest.raises(gbscan.ScanError):
            gbscan.scan_conj(cols, [(0, 10), (0, 10)])
    with pytest.raises(gbscan.ScanError):
        gbscan.scan_conj([], [])
    for c in (a, b, r):
        c.close()


def test_conjunction_serving_table_size():
    """Three columns of the serving table's size (2^27 rows; b = 8, 16, 24) with an
    aggregate column, exact against the oracle on the device-encoded words."""
    n = 1 << 27
    specs = [(8, 0), (16, 0), (24, 0)]
    cols, words = [], []
    for i, (b, _) in enumerate(specs):
        v = synth.uniform_values_device(synth.seed_for(101, i), n, b)
        c = gbscan.Column.from_device(v, n, b)
        del v
        cols.append(c)
        words.append(d2h_u32(c.dev_packed, gbscan.scan_packed_words(n, b)))
    preds = [synth.pick_range(synth.seed_for(102, i), b, s) for i, ((b, _), s) in enumerate(zip(specs, [0.5, 0.3, 0.7]))]
    want = oracle.scan_conj([(w, b, 0, lo, hi) for w, (b, _), (lo, hi) in zip(words, specs, preds)], n,
                            (words[2], 24, 0))
    r = gbscan.scan_conj(cols, preds, cols[2])
    assert (r.count, r.sum) == want
    for c in cols:
        c.close()
    torch.cuda.empty_cache()
