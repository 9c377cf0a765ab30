"""The branchy PTX row votes (vote_rows 2: one row per block, 3: two rows per
block) give the oracle's COUNT and SUM at every width they serve (b <= 21), in
both geometries, at the predicates where a vote decides the most: a full domain
(every vote taken), a single value, a value the column lacks (no vote taken)
and a sparse range, on a column with a ragged tail."""
import numpy as np
import pytest

import oracle
import synth
from paper_2606_22423_gb300 import gbscan

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.init()
    gbscan.load()
    gbscan.autotune_reset()
    yield
    gbscan.autotune_reset()


@pytest.mark.parametrize("b", range(1, 22))
def test_ptx_vote_forms_match_the_oracle(b):
    base = 1000 + b
    n = 97 * 1024 + 333                       # several tiles at every shape, ragged tail
    v = synth.uniform_values(synth.seed_for(95, b), n, b, base)
    col = gbscan.Column.from_host(v, b, base)
    top = base + (1 << b)
    preds = [(base - 5, top + 5),             # full domain: every vote taken
             (int(v[n // 2]), int(v[n // 2]) + 1),   # one value
             synth.pick_range(synth.seed_for(95, b, 1), b, 1e-4, base)]
    present = np.unique(v)
    if present.size < (1 << b):               # a code in the domain that no value has: no vote taken
        absent = int(np.setdiff1d(np.arange(base, top, dtype=np.int64), present.astype(np.int64))[0])
        preds.append((absent, absent + 1))
    want = [oracle.scan_values(v, lo, hi) for lo, hi in preds]
    geos = [0, 2] if 9 <= b <= 16 else [0]
    for vote in (2, 3):
        for lanes in geos:
            step = lanes or (4 if b <= 16 else 2)
            for warps, tiles in ((16, step), (12, step), (8, 2 * step)):
                if warps * 2 * (tiles * 128 * b + 12) > 226 * 1024:    # the shared-memory budget
                    continue
                shape = dict(warps=warps, stages=2, tile_blocks=tiles, vote_rows=vote, vec_lanes=lanes)
                gbscan.shape_set(b, "branchy", shape)
                for (lo, hi), w in zip(preds, want):
                    r = col.run(lo, hi, "branchy")
                    assert r.pair() == w, (b, shape, lo, hi)
                    assert r.blocks_scanned == (n + 1023) // 1024
    gbscan.shape_set(b, "branchy", None)
    col.close()
