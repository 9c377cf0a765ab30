"""Parity of the CUDA path with the oracle, through the C ABI.

Integer work, so the bar is bit-exact: COUNT, SUM and (for zone skipping)
the number of blocks read must equal the oracle's.  Small cases span several
tiles of every width plus a ragged tail; the large cases use the sizes and
launch shapes the benchmark times."""
import math

import numpy as np
import pytest

import oracle
import synth
from paper_2606_22423_gb300 import gbscan
from tests._cudart import d2h_u32

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

STRATS = ["branchfree", "branchy", "zone_bf", "zone_br", "auto"]


def auto_dense_min(nblocks, b):
    """SCAN_AUTO's break-even survivor count (header: a fraction
    min(0.9, (128b - 8) / (128b + 8)) of the blocks)."""
    return math.ceil(min(0.9, (128.0 * b - 8.0) / (128.0 * b + 8.0)) * nblocks)
SIGMAS = [1e-3, 0.1, 0.5, 1.0]


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.init()
    return gbscan.load()


def _dev(a: np.ndarray):
    return torch.from_numpy(a.view(np.int32).copy()).cuda()


def _check_column(col, v, b, base, preds, zmin=None, zmax=None, words=None):
    n = v.size
    words = oracle.pack(v, b, base) if words is None else words
    if zmin is None:
        zmin, zmax = oracle.zonemap(words, n, b, base)
    col.zonemap_build()
    nblocks = (n + 1023) // 1024
    for lo, hi in preds:
        want = oracle.scan_packed(words, n, b, base, lo, hi)
        zc, zs, touched = oracle.scan_zoneskip(words, zmin, zmax, n, b, base, lo, hi)
        assert (zc, zs) == want
        for strat in STRATS:
            r = col.run(lo, hi, strat)
            assert r.pair() == want, f"b={b} n={n} [{lo},{hi}) {strat}: {r.pair()} != {want}"
            if lo < hi and want is not None and n:
                empty = max(lo, base) >= min(hi, base + (1 << b))
                if not empty:
                    expect_blocks = touched if strat.startswith("zone") else nblocks
                    if strat == "auto":
                        # the zone test's survivors against the break-even: all blocks, or the survivors
                        expect_blocks = nblocks if touched >= auto_dense_min(nblocks, b) else touched
                    assert r.blocks_scanned == expect_blocks, (strat, r.blocks_scanned, expect_blocks)


def _preds(b, base, salt):
    out = []
    for i, s in enumerate(SIGMAS):
        out.append(synth.pick_range(synth.seed_for(70, b, salt * 16 + i), b, s, base))
    d = 1 << b
    out += [(base, base + d), (base - 5, base + d + 5), (base + d - 1, base + d), (base, base + 1),
            (base + 3, base + 3), (base + 9, base + 2), (-(1 << 40), base), (base + d, 1 << 40)]
    return out


@pytest.mark.parametrize("b", range(1, 33))
def test_all_widths_strategies_orders_and_tails(b):
    max_base = (1 << 32) - (1 << b)
    base = min(4321, max_base)
    n = 300 * 1024 + 555            # several tiles at every width, ragged tail
    for oi, (order, p) in enumerate([("uniform", None), ("sorted", 0.0), ("swapped", 0.01)]):
        seed = synth.seed_for(71, b, oi)
        v = (synth.uniform_values(seed, n, b, base) if p is None
             else synth.clustered_values(seed, n, b, p, base))
        col = gbscan.Column.from_host(v, b, base)
        _check_column(col, v, b, base, _preds(b, base, len(order)))
        col.close()


@pytest.mark.parametrize("b", [1, 3, 8, 13, 16, 21, 22, 27, 28, 32])
def test_device_encoder_matches_oracle(b):
    max_base = (1 << 32) - (1 << b)
    for n, base in [(1, 0), (1000, min(5, max_base)), (1024, max_base), (70 * 1024 + 999, 0)]:
        v = synth.uniform_values(synth.seed_for(72, b, n), n, b, base)
        words = gbscan.scan_packed_words(n, b)
        out = torch.zeros(words, dtype=torch.int32, device="cuda")
        gbscan.scan_encode_device(_dev(v), n, b, base, out)
        np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), oracle.pack(v, b, base))
        col = gbscan.Column.from_device(_dev(v), n, b, base)
        _check_column(col, v, b, base, _preds(b, base, 3)[:4])
        col.close()


def test_device_encoder_rejects_out_of_range_values():
    v = np.array([0, 5, 300, 7], dtype=np.uint32)
    with pytest.raises(gbscan.ScanError) as e:
        gbscan.Column.from_device(_dev(v), 4, 8, 0)
    assert e.value.status == gbscan.SCAN_EINVAL


@pytest.mark.parametrize("b", [1, 6, 16, 25, 32])
def test_zonemap_matches_oracle(b):
    n = 100 * 1024 + 17
    v = synth.clustered_values(synth.seed_for(73, b), n, b, 0.1)
    col = gbscan.Column.from_host(v, b)
    col.zonemap_build()
    nb = (n + 1023) // 1024
    torch.cuda.synchronize()
    zptr = col.zonemap_ptr()
    assert zptr
    host = d2h_u32(zptr, 2 * nb)
    zmin, zmax = oracle.zonemap(oracle.pack(v, b), n, b)
    np.testing.assert_array_equal(host[0::2], zmin)
    np.testing.assert_array_equal(host[1::2], zmax)
    col.close()


def test_edge_sizes_and_packed_borrowing():
    for n in [0, 1, 31, 1023, 1024, 1025, 2048, 5000]:
        for b in [1, 9, 32]:
            v = synth.uniform_values(synth.seed_for(74, b, n), n, b)
            words = oracle.pack(v, b)
            dev = _dev(words) if words.size else torch.zeros(4, dtype=torch.int32, device="cuda")
            col = gbscan.Column.from_packed(dev, n, b)
            _check_column(col, v, b, 0, _preds(b, 0, 5), words=words)
            col.close()


def test_misaligned_packed_buffer_is_rejected():
    buf = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(gbscan.ScanError) as e:
        gbscan.Column.from_packed(buf.data_ptr() + 4, 1024, 1)
    assert e.value.status == gbscan.SCAN_EINVAL


def test_zone_skip_without_zonemap_is_rejected():
    v = synth.uniform_values(1, 5000, 8)
    col = gbscan.Column.from_host(v, 8)
    with pytest.raises(gbscan.ScanError) as e:
        col.run(0, 10, "zone_bf")
    assert e.value.status == gbscan.SCAN_EINVAL
    col.close()


def test_async_result_in_device_memory():
    b, n = 12, 50 * 1024 + 3
    v = synth.uniform_values(synth.seed_for(75), n, b)
    col = gbscan.Column.from_host(v, b)
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    for lo, hi in [(100, 2000), (7, 7), (0, 1 << 12)]:
        col.run_async(lo, hi, out, "branchfree", stream=s)
        col.status(stream=s)
        got = tuple(int(x) for x in out.cpu()[:2])
        assert got == oracle.scan_values(v, lo, hi)
    col.close()


def test_maximum_size_and_largest_sum():
    # n = 2^31 values: b = 1 with every code 1, and b = 32 with every value
    # 2^32 - 1, whose SUM (2^63 - 2^31) is the largest the ABI can return.
    n = 1 << 31
    for b, word, v in [(1, -1, 1), (32, -1, (1 << 32) - 1)]:
        words = gbscan.scan_packed_words(n, b)
        dev = torch.full((words,), word, dtype=torch.int32, device="cuda")
        col = gbscan.Column.from_packed(dev, n, b)
        col.zonemap_build()
        for strat in STRATS:
            assert col.run(v, v + 1, strat).pair() == (n, n * v)
            assert col.run(0, v, strat).pair() == (0, 0)
        col.close()
        del dev
        torch.cuda.empty_cache()


def _device_column(b, n, seed, p=None):
    """A column drawn and encoded on the device (the benchmark's path), with host
    copies of the generator's raw values and of the library's packed words."""
    v = (synth.uniform_values_device(seed, n, b) if p is None
         else synth.clustered_values_device(seed, n, b, p))
    col = gbscan.Column.from_device(v, n, b)
    raw = v.cpu().numpy().view(np.uint32)
    host = d2h_u32(col.dev_packed, gbscan.scan_packed_words(n, b))
    del v
    return col, raw, host


def _brute_force(raw, preds):
    """oracle.scan_values over the raw values for every predicate, in threads
    (the C loop releases the interpreter lock)."""
    from concurrent.futures import ThreadPoolExecutor

    with ThreadPoolExecutor(len(preds)) as ex:
        return list(ex.map(lambda pr: oracle.scan_values(raw, *pr), preds))


def test_plain_scan_n2pow24_b8():
    # plain single-column scan: 2^24 uniform values in [0, 2^8), sigma = 0.1
    n, b = 1 << 24, 8
    col, raw, words = _device_column(b, n, synth.seed_for(1))
    np.testing.assert_array_equal(words, oracle.pack(raw, b))
    lo, hi = synth.pick_range(synth.seed_for(1, 0, 1), b, 0.1)
    want = oracle.scan_values(raw, lo, hi)
    assert want == oracle.scan_packed_threads(words, n, b, 0, lo, hi, 8)
    for strat in ["branchfree", "branchy"]:
        assert col.run(lo, hi, strat).pair() == want
    col.close()


@pytest.mark.parametrize("b", [1, 7, 16, 23, 32])
def test_sweep_size_n2pow28_from_raw_values(b):
    """The sweep's column size, drawn and encoded on the device as the benchmark
    does: the library's words equal oracle.pack of the generator's raw values,
    and every strategy's COUNT/SUM equals brute force over those raw values."""
    n = 1 << 28
    col, raw, words = _device_column(b, n, synth.seed_for(2, b))
    np.testing.assert_array_equal(words, oracle.pack(raw, b))
    col.zonemap_build()
    preds = [synth.pick_range(synth.seed_for(2, b, int(s * 1000)), b, s) for s in [1e-3, 0.5]]
    for (lo, hi), want in zip(preds, _brute_force(raw, preds)):
        for strat in ["branchfree", "branchy", "zone_bf", "zone_br", "zone_agg_bf"]:
            r = col.run(lo, hi, strat)
            assert r.pair() == want, (b, lo, hi, strat)
            if not strat.startswith("zone"):
                assert r.blocks_scanned == n // 1024
    col.close()


def test_zone_size_n2pow30_b16_from_raw_values():
    """The zone sweep's column (2^30 values at b = 16, 1% displaced): encoder
    bytes, zone maps, every strategy and the blocks read against the oracle."""
    n, b = 1 << 30, 16
    col, raw, words = _device_column(b, n, synth.seed_for(3, 0, 1), p=0.01)
    np.testing.assert_array_equal(words, oracle.pack(raw, b))
    col.zonemap_build()
    zmin, zmax = oracle.zonemap(words, n, b)
    preds = [synth.pick_range(synth.seed_for(3, 0, 2 + i), b, s) for i, s in enumerate([1e-4, 1e-3, 0.1])]
    for (lo, hi), want in zip(preds, _brute_force(raw, preds)):
        zc, zs, touched = oracle.scan_zoneskip(words, zmin, zmax, n, b, 0, lo, hi)
        assert (zc, zs) == want
        full = col.run(lo, hi, "branchfree")
        assert full.pair() == want and full.blocks_scanned == n // 1024
        for strat in ["branchy", "zone_bf", "zone_br", "zone_agg_bf"]:
            r = col.run(lo, hi, strat)
            assert r.pair() == want, (lo, hi, strat)
            if strat in ("zone_bf", "zone_br"):
                assert r.blocks_scanned == touched
    col.close()


def test_auto_edges_layouts_stale_and_rebuilt_zone_maps():
    """SCAN_AUTO without a zone map (or on a non-lane layout) runs the full scan;
    after scan_column_upload_packed the zone map is stale, AUTO falls back to the
    full scan on the new data, and once the map is rebuilt its survivor count
    (sorted bounds taken again) follows the new data."""
    b, n = 12, 200 * 1024 + 99
    sorted_v = synth.clustered_values(synth.seed_for(76, 1), n, b, 0.0)
    shuffled_v = synth.clustered_values(synth.seed_for(76, 2), n, b, 1.0)
    nblocks = (n + 1023) // 1024
    lo, hi = synth.pick_range(synth.seed_for(76, 3), b, 0.02)
    col = gbscan.Column.from_host(sorted_v, b)
    r = col.run(lo, hi, "auto")                          # no zone map yet: full scan
    assert r.pair() == oracle.scan_values(sorted_v, lo, hi) and r.blocks_scanned == nblocks
    col.zonemap_build()
    r = col.run(lo, hi, "auto")                          # sorted and selective: zone skipping
    assert r.pair() == oracle.scan_values(sorted_v, lo, hi) and r.blocks_scanned < nblocks // 10
    for plo, phi in [(5, 5), (0, 1 << b), (-(1 << 40), 0), (1 << b, 1 << 40)]:   # empty, full, outside
        assert col.run(plo, phi, "auto").pair() == oracle.scan_values(sorted_v, plo, phi)
    # new data through the packed upload: the zone map is stale and AUTO scans everything
    col.upload_packed(oracle.pack(shuffled_v, b))
    torch.cuda.synchronize()
    r = col.run(lo, hi, "auto")
    assert r.pair() == oracle.scan_values(shuffled_v, lo, hi) and r.blocks_scanned == nblocks
    col.zonemap_build()                                  # shuffled: every block survives -> full scan
    r = col.run(lo, hi, "auto")
    assert r.pair() == oracle.scan_values(shuffled_v, lo, hi) and r.blocks_scanned == nblocks
    col.upload_packed(oracle.pack(sorted_v, b))          # and back: selective again once rebuilt
    torch.cuda.synchronize()
    col.zonemap_build()
    r = col.run(lo, hi, "auto")
    assert r.pair() == oracle.scan_values(sorted_v, lo, hi) and r.blocks_scanned < nblocks // 10
    col.close()
    for layout in ("rowmajor", "bytes"):
        lb = 16 if layout == "bytes" else 13
        v = synth.clustered_values(synth.seed_for(76, 4), n, lb, 0.0)
        c = gbscan.Column.from_host(v, lb, layout=layout)
        plo, phi = synth.pick_range(synth.seed_for(76, 5), lb, 0.01)
        r = c.run(plo, phi, "auto")
        assert r.pair() == oracle.scan_values(v, plo, phi) and r.blocks_scanned == nblocks
        c.close()
