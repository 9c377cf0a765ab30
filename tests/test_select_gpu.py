"""Parity of the materializing select with the oracle, through the C ABI.

Positions are integers, so the bar is bit-exact: the full position list (in
order) and the count must equal the oracle's.  Small cases span several tiles
and several grid iterations of every tested width plus a ragged tail; the
large cases use the benchmark's sizes (N = 2^28) and compare the whole list."""
import numpy as np
import pytest

import oracle
import synth
from paper_2606_22423_gb300 import gbscan
from tests._cudart import d2h_u32

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FLAVOURS = ["branchfree", "branchy"]


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.init()
    return gbscan.load()


def _positions(col, lo, hi, strat, capacity, fill=-1):
    out = torch.full((max(capacity, 1),), fill, dtype=torch.int32, device="cuda")
    k = col.select(lo, hi, out if capacity else None, strat, capacity=capacity)
    got = out.cpu().numpy().view(np.uint32)
    return got, k


def _check(col, words, n, b, base, lo, hi):
    want, k = oracle.select_packed(words, n, b, base, lo, hi)
    for strat in FLAVOURS:
        got, kk = _positions(col, lo, hi, strat, max(k, 1))
        assert kk == k, (b, n, lo, hi, strat, kk, k)
        np.testing.assert_array_equal(got[:k], want, err_msg=f"b={b} n={n} [{lo},{hi}) {strat}")
    return k


# n values chosen to span several tiles and, for the wider widths, several
# grid iterations (152 CTAs x 8 warps x tile blocks per iteration)
@pytest.mark.parametrize("b,n", [(1, 70_001), (3, 400_003), (8, 1_000_000), (13, 2_500_017),
                                 (16, 5_000_111), (24, 3_000_001), (31, 6_000_007), (32, 7_500_123)])
def test_select_matches_oracle(b, n):
    base = 0 if b == 32 else 1000
    v = synth.uniform_values(synth.seed_for(90, b), n, b, base)
    words = oracle.pack(v, b, base)
    col = gbscan.Column.from_host(v, b, base)
    for i, s in enumerate([1e-4, 0.1, 0.5, 1.0]):
        lo, hi = synth.pick_range(synth.seed_for(91, b, i), b, s, base)
        _check(col, words, n, b, base, lo, hi)
    # a predicate reaching past both ends of the domain selects everything
    assert _check(col, words, n, b, base, -5, 1 << 40) == n
    col.close()


def test_select_sorted_column_and_edge_sizes():
    b = 12
    for n in [1, 31, 1023, 1024, 1025, 4096 + 5]:
        v = synth.clustered_values(synth.seed_for(92, n), n, b, 0.01)
        words = oracle.pack(v, b)
        col = gbscan.Column.from_host(v, b)
        for lo, hi in [(0, 1 << b), (100, 2000), (int(v[n // 2]), int(v[n // 2]) + 1), (3000, 3000)]:
            _check(col, words, n, b, 0, lo, hi)
        col.close()


def test_select_capacity_and_empty():
    b, n = 9, 300_000
    v = synth.uniform_values(93, n, b)
    words = oracle.pack(v, b)
    col = gbscan.Column.from_host(v, b)
    lo, hi = 100, 300
    want, k = oracle.select_packed(words, n, b, 0, lo, hi)
    for strat in FLAVOURS:
        for cap in [1, 7, k // 3, k - 1]:
            # with capacity cap the call writes exactly the first cap positions
            out = torch.full((cap + 16,), -1, dtype=torch.int32, device="cuda")
            assert col.select(lo, hi, out, strat, capacity=cap) == k
            h = out.cpu().numpy().view(np.uint32)
            np.testing.assert_array_equal(h[:cap], want[:cap])
            assert np.all(h[cap:] == 0xFFFFFFFF)
        assert col.select(lo, hi, None, strat, capacity=0) == k        # count only
        assert col.select(300, 100, None, strat) == 0                  # inverted range
        assert col.select(1 << b, 1 << 20, None, strat) == 0           # above the domain
    col.close()


def test_select_async_count_in_device_memory():
    b, n = 20, 2_000_000
    v = synth.uniform_values(94, n, b)
    words = oracle.pack(v, b)
    col = gbscan.Column.from_host(v, b)
    lo, hi = synth.pick_range(95, b, 0.3)
    want, k = oracle.select_packed(words, n, b, 0, lo, hi)
    pos = torch.zeros(k, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    for strat in FLAVOURS:
        pos.zero_()
        col.select_async(lo, hi, pos, cnt, strat, stream=s)
        col.status(s)
        assert int(cnt.item()) == k
        np.testing.assert_array_equal(pos.cpu().numpy().view(np.uint32), want)
    col.close()


def test_select_rejects_zone_strategies_and_null_output():
    v = synth.uniform_values(96, 5000, 8)
    col = gbscan.Column.from_host(v, 8)
    with pytest.raises(gbscan.ScanError):
        col.select(0, 10, None, "zone_bf", capacity=0)
    with pytest.raises(gbscan.ScanError):
        col.select(0, 10, None, "branchfree", capacity=10)   # no buffer for 10 positions
    col.close()


@pytest.mark.parametrize("b", [16, 32])
def test_select_full_size_n2pow28(b):
    """The benchmark's select workload: N = 2^28 uniform values; the whole
    position list is compared with the oracle's."""
    n = 1 << 28
    v = (synth.uniform_values_device(synth.seed_for(97, b), n, b))
    col = gbscan.Column.from_device(v, n, b)
    words = d2h_u32(col.dev_packed, gbscan.scan_packed_words(n, b))
    del v
    for s in [0.01, 0.5]:
        lo, hi = synth.pick_range(synth.seed_for(98, b, int(s * 100)), b, s)
        want, k = oracle.select_packed(words, n, b, 0, lo, hi)
        out = torch.empty(k, dtype=torch.int32, device="cuda")
        for strat in FLAVOURS:
            out.fill_(-1)
            assert col.select(lo, hi, out, strat) == k
            np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), want)
        del out
    col.close()
    torch.cuda.empty_cache()
