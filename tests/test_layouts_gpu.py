"""Parity of the row-major and byte-aligned layouts (paper §3 strategies i and
iii) with the oracle, through the C ABI: the device encoder's words and every
scan's COUNT/SUM must equal the oracle's exactly, for every width, both
predicate flavours, ragged sizes and the benchmark's column size."""
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


def _dev(a: np.ndarray):
    return torch.from_numpy(a.view(np.int32).copy()).cuda()


def _preds(b, base, salt):
    out = [synth.pick_range(synth.seed_for(85, b, salt * 8 + i), b, s, base)
           for i, s in enumerate([1e-3, 0.1, 0.5, 1.0])]
    return out + [(base - 3, base + (1 << b) + 5), (base + 7, base + 7)]


def _oracle_scan(layout, words, n, b, base, lo, hi):
    if layout == "bytes":
        return oracle.scan_bytes(words, n, b, base, lo, hi)
    return oracle.scan_rowmajor(words, n, b, base, lo, hi)


@pytest.mark.parametrize("b", range(1, 33))
def test_rowmajor_all_widths(b):
    base = 0 if b == 32 else 500
    n = 300 * 1024 + 555
    v = synth.uniform_values(synth.seed_for(86, b), n, b, base)
    words = oracle.pack_rowmajor(v, b, base)
    col = gbscan.Column.from_device(_dev(v), n, b, base, layout="rowmajor")
    assert col.layout == "rowmajor"
    np.testing.assert_array_equal(d2h_u32(col.dev_packed, words.size), words)
    for lo, hi in _preds(b, base, 1):
        want = oracle.scan_rowmajor(words, n, b, base, lo, hi)
        for strat in ("branchfree", "branchy"):
            assert col.run(lo, hi, strat).pair() == want, (b, lo, hi, strat)
    col.close()


@pytest.mark.parametrize("b", [8, 16, 32])
def test_bytes_layout(b):
    base = 0 if b == 32 else 11
    for n in (1, 1023, 1025, 200 * 1024 + 77):
        v = synth.uniform_values(synth.seed_for(87, b, n), n, b, base)
        words = oracle.pack_bytes(v, b, base)
        for make in ("host", "device"):
            col = (gbscan.Column.from_host(v, b, base, layout="bytes") if make == "host"
                   else gbscan.Column.from_device(_dev(v), n, b, base, layout="bytes"))
            np.testing.assert_array_equal(d2h_u32(col.dev_packed, words.size), words)
            for lo, hi in _preds(b, base, n % 7):
                want = oracle.scan_bytes(words, n, b, base, lo, hi)
                for strat in ("branchfree", "branchy"):
                    assert col.run(lo, hi, strat).pair() == want, (b, n, lo, hi, strat, make)
            col.close()


def test_rowmajor_edge_sizes_and_sorted_data():
    for b in (5, 13, 27):
        for n in (1, 31, 1024, 1025, 2 * 1024 + 1):
            v = synth.clustered_values(synth.seed_for(88, b, n), n, b, 0.0)
            words = oracle.pack_rowmajor(v, b)
            col = gbscan.Column.from_host(v, b, layout="rowmajor")
            for lo, hi in [(0, 1 << b), (int(v[n // 2]), int(v[n // 2]) + 3), (1, 1)]:
                want = oracle.scan_rowmajor(words, n, b, 0, lo, hi)
                for strat in ("branchfree", "branchy"):
                    assert col.run(lo, hi, strat).pair() == want
            col.close()


def test_other_layouts_are_rejected_where_lanes_are_needed():
    v = synth.uniform_values(89, 5000, 9)
    col = gbscan.Column.from_host(v, 9, layout="rowmajor")
    with pytest.raises(gbscan.ScanError):
        col.zonemap_build()
    with pytest.raises(gbscan.ScanError):
        col.run(0, 10, "zone_bf")
    with pytest.raises(gbscan.ScanError):
        col.select(0, 10, None, "branchfree", capacity=0)
    with pytest.raises(gbscan.ScanError):
        gbscan.Batch([col])
    with pytest.raises(gbscan.ScanError):
        gbscan.Column.from_host(v, 9, layout="bytes")            # bytes needs b in {8, 16, 32}
    col.close()


@pytest.mark.parametrize("layout,b", [("rowmajor", 5), ("rowmajor", 16), ("bytes", 8), ("bytes", 16)])
def test_full_size_n2pow28(layout, b):
    """The benchmark's layout workload: N = 2^28 uniform values, exact against
    the oracle on the device-encoded words."""
    n = 1 << 28
    v = synth.uniform_values_device(synth.seed_for(90, b), n, b)
    col = gbscan.Column.from_device(v, n, b, layout=layout)
    del v
    words = d2h_u32(col.dev_packed, gbscan.scan_packed_words(n, b))
    for s in (1e-3, 0.5):
        lo, hi = synth.pick_range(synth.seed_for(91, b, int(s * 1000)), b, s)
        want = _oracle_scan(layout, words, n, b, 0, lo, hi)
        for strat in ("branchfree", "branchy"):
            assert col.run(lo, hi, strat).pair() == want, (layout, b, s, strat)
    col.close()
    torch.cuda.empty_cache()
