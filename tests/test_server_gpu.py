"""Serving: queries that arrive while others run are batched together and
overlap on the device, yet every query's result equals the query run alone."""
import threading
import time

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
    return gbscan.load()


@pytest.fixture(scope="module")
def table():
    cols, vals = [], []
    widths = [4, 8, 12, 16, 24, 32]
    for i in range(12):
        b, n = widths[i % 6], (1 << 18) + 77 * i
        v = synth.clustered_values(700 + i, n, b, 0.0) if i % 2 == 0 else synth.uniform_values(700 + i, n, b)
        c = gbscan.Column.from_host(v, b)
        c.zonemap_build()
        cols.append(c)
        vals.append(v)
    yield cols, vals
    for c in cols:
        c.close()


def _queries(cols, count, seed):
    rng = np.random.default_rng(seed)
    qs = []
    for _ in range(count):
        k = int(rng.integers(1, 9))
        ids = [int(x) for x in rng.choice(len(cols), size=k, replace=True)]
        preds = [synth.pick_range(int(rng.integers(1 << 30)), cols[c].b,
                                  float(synth.log_uniform(rng, 1e-4, 1.0))) for c in ids]
        qs.append((ids, preds))
    return qs


def test_results_in_the_mix_equal_results_alone(table):
    cols, vals = table
    qs = _queries(cols, 300, 1)
    alone = [[cols[c].run(lo, hi).pair() for c, (lo, hi) in zip(ids, preds)] for ids, preds in qs]
    for ids, preds in qs[:10]:                       # alone is itself the oracle's answer
        for c, (lo, hi) in zip(ids, preds):
            assert cols[c].run(lo, hi).pair() == oracle.scan_values(vals[c], lo, hi)
    srv = gbscan.Server(cols, slots=3, device_bytes_per_slot=112 * 64)
    got = [None] * len(qs)

    def submitter(lo_i, hi_i, delay):
        for i in range(lo_i, hi_i):
            qid = srv.submit(*qs[i])
            got[i] = qid
            time.sleep(delay)

    # two producers with different pacing so queries arrive while batches run ...
    t1 = threading.Thread(target=submitter, args=(0, 100, 0.0))
    t2 = threading.Thread(target=submitter, args=(100, 200, 0.0002))
    t1.start(); t2.start()
    # ... and bursts that must be packed several queries to a launch
    for k in range(200, 300, 25):
        got[k:k + 25] = srv.submit_many(qs[k:k + 25])
    t1.join(); t2.join()
    lat = []
    for i, (ids, _) in enumerate(qs):
        done, res, us = srv.poll(got[i], len(ids), wait=True)
        assert done
        assert [r.pair() for r in res] == alone[i], i
        lat.append(us)
    st = srv.stats()
    assert st["column_scans"] == sum(len(ids) for ids, _ in qs)
    assert st["batches"] < len(qs)                   # queries were batched together
    assert min(lat) > 0
    srv.close()


def test_admission_queue_limit_and_small_slots(table):
    cols, _ = table
    srv = gbscan.Server(cols, slots=1, device_bytes_per_slot=112 * 8, max_queue=4)
    qs = _queries(cols, 64, 2)
    ids, busy = [], 0
    for q in qs:
        try:
            ids.append((srv.submit(*q), q))
        except gbscan.ScanError as e:
            assert e.status == gbscan.SCAN_EBUSY
            busy += 1
    for qid, (cids, preds) in ids:
        done, res, _ = srv.poll(qid, len(cids), wait=True)
        assert done and [r.pair() for r in res] == [cols[c].run(lo, hi).pair() for c, (lo, hi) in zip(cids, preds)]
    assert srv.stats()["rejected"] == busy
    with pytest.raises(gbscan.ScanError):            # more scans than one slot holds
        srv.submit(list(range(9)), [(0, 5)] * 9)
    srv.close()


def test_served_query_at_the_serving_table_size_against_the_oracle():
    """Columns of the serving table's size (2^27 values; b in {4, 8, 12, 16, 24,
    32}; sorted and shuffled), drawn on the device: an 8-column query and a
    burst of smaller ones served together give brute force over the raw values."""
    from concurrent.futures import ThreadPoolExecutor

    widths = [4, 8, 12, 16, 24, 32]
    n = 1 << 27
    cols, raws = [], []
    for c in range(8):
        b = widths[c % 6]
        seed = synth.seed_for(5, c)
        v = (synth.clustered_values_device(seed, n, b, 0.0) if c % 2 == 0
             else synth.uniform_values_device(seed, n, b))
        col = gbscan.Column.from_device(v, n, b)
        col.zonemap_build()
        cols.append(col)
        raws.append(v.cpu().numpy().view(np.uint32))
        del v
    rng = np.random.default_rng(synth.seed_for(5, 0, 7))
    queries = [(list(range(8)), [synth.pick_range(int(rng.integers(1 << 30)), cols[c].b,
                                                  float(synth.log_uniform(rng, 1e-4, 1.0))) for c in range(8)])]
    queries += [q for q in _queries(cols, 12, 3)]
    srv = gbscan.Server(cols, slots=4, device_bytes_per_slot=112 * 512)
    ids = [srv.submit(ids_, preds) for ids_, preds in queries]          # submitted back to back
    jobs = [(c, lo, hi) for ids_, preds in queries for c, (lo, hi) in zip(ids_, preds)]
    with ThreadPoolExecutor(16) as ex:
        flat = list(ex.map(lambda j: oracle.scan_values(raws[j[0]], j[1], j[2]), jobs))
    k = 0
    for qid, (ids_, preds) in zip(ids, queries):
        done, res, _ = srv.poll(qid, len(ids_), wait=True)
        assert done
        assert [r.pair() for r in res] == flat[k:k + len(ids_)]
        k += len(ids_)
    srv.close()
    for c in cols:
        c.close()
    torch.cuda.empty_cache()
