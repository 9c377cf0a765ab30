"""Pins for the CPU oracle against facts that do not come from the oracle.

Each test names what fixes the expected value:
  * the layout definition written at bit level with numpy bit arrays (an
    independent construction from the oracle's shift/mask arithmetic);
  * reductions of special widths to plain numpy reshapes (b = 8, 16, 32);
  * histogram brute force (np.bincount) for COUNT/SUM, exhaustive on tiny
    domains;
  * closed forms (a permutation of 0..N-1 sums to N(N-1)/2);
  * invariants (range additivity, frame-of-reference shift, zone-skip
    exactness, multiset invariance under displacement);
  * the probability of a zone-map skip on i.i.d. uniform data;
  * np.flatnonzero over the raw values for the materializing select.
A plausible mistake in the oracle (swapped lane/row, MSB-first streams, a
dropped carry word, an inclusive upper bound, base not added back, a tail
block counted) fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
import synth

SIZES = [0, 1, 31, 32, 33, 1023, 1024, 1025, 4096 + 7]


def layout_by_bits(values: np.ndarray, b: int, base: int) -> np.ndarray:
    """Lane-interleaved image built from bit arrays (no shifts or masks).

    Value j of a 1024-value block sits at lane j % 32, row j // 32; a lane's
    stream is the concatenation of its rows' b-bit codes, least significant
    bit first; stream bit p is bit p % 32 of lane word p // 32; word w of lane
    l of block k is stored at 32*b*k + 32*w + l.
    """
    n = values.size
    nb = (n + 1023) // 1024
    codes = np.zeros(nb * 1024, dtype=np.uint32)
    codes[:n] = values - np.uint32(base)
    bits = np.unpackbits(codes.astype("<u4").view(np.uint8), bitorder="little")
    bits = bits.reshape(nb * 1024, 32)[:, :b]              # code bits, LSB first
    bits = bits.reshape(nb, 32, 32, b)                       # (block, row, lane, bit)
    streams = bits.transpose(0, 2, 1, 3).reshape(nb, 32, 32 * b)   # (block, lane, stream bit)
    words = np.packbits(streams.reshape(nb, 32, b, 32), axis=-1, bitorder="little")
    words = words.reshape(nb, 32, b, 4).copy().view("<u4").reshape(nb, 32, b)  # (block, lane, word)
    return words.transpose(0, 2, 1).reshape(-1).astype(np.uint32)


def hist_count_sum(values: np.ndarray, lo: int, hi: int):
    """COUNT/SUM from a value histogram (small domains only)."""
    if values.size == 0:
        return 0, 0
    h = np.bincount(values.astype(np.int64))
    lo_c, hi_c = max(lo, 0), min(hi, h.size)
    if lo_c >= hi_c:
        return 0, 0
    v = np.arange(lo_c, hi_c, dtype=np.int64)
    return int(h[lo_c:hi_c].sum()), int((h[lo_c:hi_c] * v).sum())


@pytest.mark.parametrize("b", range(1, 33))
def test_pack_matches_bit_level_layout(b):
    base = 0 if b == 32 else 7 * b
    for n in SIZES:
        v = synth.uniform_values(synth.seed_for(90, b, n), n, b, base)
        got = oracle.pack(v, b, base)
        assert got.size == oracle.packed_words(n, b) == ((n + 1023) // 1024) * 32 * b
        if n:
            np.testing.assert_array_equal(got, layout_by_bits(v, b, base))


@pytest.mark.parametrize("b", range(1, 33))
def test_round_trip_all_widths_and_tails(b):
    max_base = (1 << 32) - (1 << b)          # largest base that keeps codes in 32 bits
    base = max_base if b % 3 == 0 else min(12345, max_base)
    for n in SIZES:
        v = synth.uniform_values(synth.seed_for(91, b, n), n, b, base)
        np.testing.assert_array_equal(oracle.unpack(oracle.pack(v, b, base), n, b, base), v)


def test_b32_is_the_plain_array():
    # negative control (i) at b = 32: the transposed layout is the identity
    v = synth.uniform_values(5, 4096, 32)
    np.testing.assert_array_equal(oracle.pack(v, 32), v)
    # tail: zero padded to whole blocks
    w = oracle.pack(v[:1500], 32)
    np.testing.assert_array_equal(w[:1500], v[:1500])
    assert not w[1500:].any()


def test_b16_and_b8_are_plain_transposes():
    # b = 16: lane word w holds rows 2w (low half) and 2w+1 (high half)
    v = synth.uniform_values(6, 3 * 1024, 16)
    halves = oracle.pack(v, 16).view("<u2").reshape(3, 16, 32, 2)   # block, word, lane, half
    np.testing.assert_array_equal(halves.transpose(0, 1, 3, 2).reshape(-1), v)
    # b = 8: lane word w holds rows 4w .. 4w+3, one byte each
    v = synth.uniform_values(7, 2 * 1024, 8)
    q = oracle.pack(v, 8).view(np.uint8).reshape(2, 8, 32, 4)       # block, word, lane, byte
    np.testing.assert_array_equal(q.transpose(0, 1, 3, 2).reshape(-1), v)


def test_b3_repeating_pattern_closed_form():
    # v_j = j mod 8 puts the constant code l mod 8 in every row of lane l;
    # for lane 1 the 96-bit stream has ones exactly at positions = 0 (mod 3)
    v = (np.arange(1024) % 8).astype(np.uint32)
    w = oracle.pack(v, 3).reshape(3, 32)
    expect = [sum(1 << p for p in range(32) if (32 * i + p) % 3 == 0) for i in range(3)]
    assert [int(x) for x in w[:, 1]] == expect == [0x49249249, 0x92492492, 0x24924924]
    assert not w[:, 0].any() and not w[:, 8].any()


@pytest.mark.parametrize("b", [1, 2, 3, 4])
def test_scan_exhaustive_small_domains(b):
    d = 1 << b
    for n in [1, 33, 1025, 2100]:
        v = synth.uniform_values(synth.seed_for(92, b, n), n, b)
        w = oracle.pack(v, b)
        for lo in range(-1, d + 2):
            for hi in range(-1, d + 2):
                want = hist_count_sum(v, lo, hi)
                assert oracle.scan_values(v, lo, hi) == want
                assert oracle.scan_packed(w, n, b, 0, lo, hi) == want


@pytest.mark.parametrize("b", [5, 8, 11, 13, 16, 21, 27, 31, 32])
def test_scan_packed_matches_histogram(b):
    n = 5000
    v = synth.uniform_values(synth.seed_for(93, b), n, b)
    w = oracle.pack(v, b)
    rng = np.random.default_rng(b)
    d = 1 << b
    for _ in range(20):
        lo, hi = sorted(int(x) for x in rng.integers(0, d + 1, size=2))
        # histogram over the sorted unique values keeps memory small at large b
        uniq, cnt = np.unique(v, return_counts=True)
        m = (uniq >= lo) & (uniq < hi)
        want = (int(cnt[m].sum()), int((uniq[m].astype(np.int64) * cnt[m]).sum()))
        assert oracle.scan_packed(w, n, b, 0, lo, hi) == want


def test_full_domain_closed_form():
    n = 3 * 1024 + 77
    b = math.ceil(math.log2(n))
    v = np.random.default_rng(1).permutation(n).astype(np.uint32)
    w = oracle.pack(v, b)
    assert oracle.scan_packed(w, n, b, 0, 0, 1 << b) == (n, n * (n - 1) // 2)
    assert oracle.scan_packed(w, n, b, 0, -(1 << 40), 1 << 40) == (n, n * (n - 1) // 2)
    # equality predicate [c, c+1) hits exactly one value of a permutation
    for c in (0, 1, n // 2, n - 1):
        assert oracle.scan_packed(w, n, b, 0, c, c + 1) == (1, c)
    assert oracle.scan_packed(w, n, b, 0, n, 1 << b) == (0, 0)


def test_empty_and_inverted_ranges():
    v = synth.uniform_values(3, 3000, 10)
    w = oracle.pack(v, 10)
    for lo, hi in [(5, 5), (9, 3), (1 << 10, 1 << 11), (-10, 0)]:
        assert oracle.scan_packed(w, 3000, 10, 0, lo, hi) == (0, 0)


def test_range_additivity_and_for_shift():
    b, base, n = 12, 100_000, 7000
    v = synth.uniform_values(4, n, b, base)
    w = oracle.pack(v, b, base)
    rng = np.random.default_rng(9)
    for _ in range(30):
        a, m, c = sorted(int(x) for x in rng.integers(base, base + (1 << b) + 1, size=3))
        ac = oracle.scan_packed(w, n, b, base, a, c)
        am = oracle.scan_packed(w, n, b, base, a, m)
        mc = oracle.scan_packed(w, n, b, base, m, c)
        assert ac == (am[0] + mc[0], am[1] + mc[1])
        # frame of reference: the same codes read with base 0 see every value shifted
        cu, su = oracle.scan_packed(w, n, b, 0, a - base, c - base)
        assert ac == (cu, su + base * cu)


def test_threaded_scan_equals_single_thread():
    b, n = 9, 50_000
    v = synth.uniform_values(8, n, b)
    w = oracle.pack(v, b)
    for lo, hi in [(0, 512), (13, 300), (511, 512)]:
        ref = oracle.scan_packed(w, n, b, 0, lo, hi)
        for t in (1, 3, 8):
            assert oracle.scan_packed_threads(w, n, b, 0, lo, hi, t) == ref


@pytest.mark.parametrize("b", [1, 7, 16, 32])
def test_zonemap_matches_numpy_block_reductions(b):
    base = 0 if b == 32 else 3
    for n in [1, 1024, 5000]:
        v = synth.clustered_values(synth.seed_for(94, b, n), n, b, 0.01, base)
        zmin, zmax = oracle.zonemap(oracle.pack(v, b, base), n, b, base)
        nb = (n + 1023) // 1024
        pad_lo = np.full(nb * 1024, np.iinfo(np.uint32).max, np.uint32)
        pad_hi = np.zeros(nb * 1024, np.uint32)
        pad_lo[:n] = v
        pad_hi[:n] = v
        np.testing.assert_array_equal(zmin, pad_lo.reshape(nb, 1024).min(axis=1))
        np.testing.assert_array_equal(zmax, pad_hi.reshape(nb, 1024).max(axis=1))


@pytest.mark.parametrize("p", [0.0, 0.01, 0.1, 1.0])
def test_zoneskip_is_exact_and_sorted_touches_few_blocks(p):
    b, n = 16, 64 * 1024 + 100
    v = synth.clustered_values(synth.seed_for(95, 0, int(p * 100)), n, b, p)
    w = oracle.pack(v, b)
    zmin, zmax = oracle.zonemap(w, n, b)
    for sigma in [1e-4, 1e-3, 1e-2, 0.1, 0.5]:
        lo, hi = synth.pick_range(synth.seed_for(95, 1, int(sigma * 1e4)), b, sigma)
        c, s, touched = oracle.scan_zoneskip(w, zmin, zmax, n, b, 0, lo, hi)
        assert (c, s) == oracle.scan_packed(w, n, b, 0, lo, hi) == oracle.scan_values(v, lo, hi)
        if p == 0.0:
            # sorted: the matches are one contiguous run of positions
            assert touched <= math.ceil(c / 1024) + 1


def test_zoneskip_on_uniform_data_follows_the_skip_probability():
    # i.i.d. uniform codes: a block is skipped iff all 1024 values miss on one
    # side, probability (lo/D)^1024 + (1 - hi/D)^1024.  The range [D-1, D)
    # keeps only blocks that hold the maximum code: P(skip) = (1-1/D)^1024.
    b, n = 16, 2048 * 1024
    d = 1 << b
    v = synth.uniform_values(11, n, b)
    w = oracle.pack(v, b)
    zmin, zmax = oracle.zonemap(w, n, b)
    nb = n // 1024
    _, _, touched = oracle.scan_zoneskip(w, zmin, zmax, n, b, 0, d - 1, d)
    p_skip = (1 - 1 / d) ** 1024
    skipped = nb - touched
    sd = math.sqrt(nb * p_skip * (1 - p_skip))
    assert abs(skipped - nb * p_skip) < 5 * sd
    # an interior range of selectivity 0.1 skips nothing
    lo, hi = d // 2, d // 2 + d // 10
    _, _, touched = oracle.scan_zoneskip(w, zmin, zmax, n, b, 0, lo, hi)
    assert touched == nb


def test_displacement_keeps_the_multiset():
    b, n = 16, 30_000
    ref = np.sort(synth.uniform_values(21, n, b))
    for p in [0.0, 0.01, 0.1, 1.0]:
        v = synth.clustered_values(21, n, b, p)
        np.testing.assert_array_equal(np.sort(v), ref)
        w = oracle.pack(v, b)
        assert oracle.scan_packed(w, n, b, 0, 1000, 40000) == oracle.scan_values(ref, 1000, 40000)


def test_invalid_inputs_are_rejected():
    v = np.array([0, 1, 2, 300], dtype=np.uint32)
    with pytest.raises(ValueError):
        oracle.pack(v, 8)            # 300 needs 9 bits
    with pytest.raises(ValueError):
        oracle.pack(v, 0)
    with pytest.raises(ValueError):
        oracle.pack(v, 33)
    with pytest.raises(ValueError):
        oracle.pack(v + 5, 9, base=6)  # value below the base
    with pytest.raises(ValueError):
        oracle.pack(v, 32, base=1)     # base + 2^32 - 1 overflows 32 bits


def test_pick_range_hits_target_selectivity():
    for b in [4, 8, 16]:
        for sigma in [1e-3, 0.1, 0.5, 1.0]:
            lo, hi = synth.pick_range(1, b, sigma)
            assert 0 <= lo < hi <= (1 << b)
            assert hi - lo == max(1, round(sigma * (1 << b)))


# ------------------------------------------------------- materializing select
@pytest.mark.parametrize("b", [1, 5, 8, 13, 24, 32])
def test_select_matches_flatnonzero(b):
    """Paper §3 "a materializing select": positions of the matches, in order,
    fixed by numpy's flatnonzero over the generator's raw values."""
    base = 0 if b == 32 else 17
    for n in (1, 1023, 1024, 5 * 1024 + 77):
        v = synth.uniform_values(synth.seed_for(31, b, n), n, b, base)
        w = oracle.pack(v, b, base)
        for sigma in (1e-3, 0.1, 0.5, 1.0):
            lo, hi = synth.pick_range(synth.seed_for(32, b, n), b, sigma, base)
            want = np.flatnonzero((v.astype(np.int64) >= lo) & (v.astype(np.int64) < hi))
            got, k = oracle.select_packed(w, n, b, base, lo, hi)
            assert k == want.size
            np.testing.assert_array_equal(got, want.astype(np.uint32))
            raw, k2 = oracle.select_values(v, lo, hi)
            assert k2 == k
            np.testing.assert_array_equal(raw, got)


def test_select_agrees_with_count_and_sum():
    """The selected positions carry exactly COUNT values whose sum is SUM."""
    b, n, base = 11, 20_000, 5
    v = synth.uniform_values(41, n, b, base)
    w = oracle.pack(v, b, base)
    for lo, hi in [(base, base + 100), (base + 700, base + 1500), (0, 1 << 40)]:
        pos, k = oracle.select_packed(w, n, b, base, lo, hi)
        c, sm = hist_count_sum(v, lo, hi)
        assert k == c
        assert int(v[pos].astype(np.int64).sum()) == sm
        assert np.all(np.diff(pos.astype(np.int64)) > 0)


def test_select_capacity_truncates_but_counts_everything():
    b, n = 6, 3000
    v = synth.uniform_values(42, n, b)
    w = oracle.pack(v, b)
    full, k = oracle.select_packed(w, n, b, 0, 10, 40)
    for cap in (0, 1, 7, k - 1, k, k + 5):
        got, kk = oracle.select_packed(w, n, b, 0, 10, 40, capacity=cap)
        assert kk == k
        np.testing.assert_array_equal(got, full[:min(cap, k)])


def test_select_empty_and_degenerate():
    v = synth.uniform_values(43, 4096, 9)
    w = oracle.pack(v, 9)
    assert oracle.select_packed(w, 4096, 9, 0, 50, 50)[1] == 0      # empty range
    assert oracle.select_packed(w, 4096, 9, 0, 60, 50)[1] == 0      # inverted range
    assert oracle.select_packed(w, 0, 9, 0, 0, 512)[1] == 0         # no values
    pos, k = oracle.select_packed(w, 4096, 9, 0, 0, 512)            # full domain
    assert k == 4096
    np.testing.assert_array_equal(pos, np.arange(4096, dtype=np.uint32))


# ------------------------------------------- row-major and byte-aligned layouts
def rowmajor_by_bits(values: np.ndarray, b: int, base: int) -> np.ndarray:
    """Paper §3 strategy (i) written at bit level: code i's bit k is stream bit
    i*b + k; stream bit p is bit p mod 32 of word p // 32; padded to whole blocks."""
    n = values.size
    u = (values.astype(np.uint64) - base)
    bits = ((u[:, None] >> np.arange(b, dtype=np.uint64)) & 1).astype(np.uint8).reshape(-1)
    nblocks = (n + 1023) // 1024
    stream = np.zeros(nblocks * 1024 * b, dtype=np.uint8)
    stream[:bits.size] = bits
    words = stream.reshape(-1, 32).astype(np.uint64)
    return (words << np.arange(32, dtype=np.uint64)).sum(axis=1).astype(np.uint32)


@pytest.mark.parametrize("b", [1, 3, 7, 8, 13, 16, 21, 31, 32])
def test_rowmajor_pack_matches_bit_level_stream(b):
    base = 0 if b == 32 else 9
    for n in (1, 33, 1024, 3 * 1024 + 17):
        v = synth.uniform_values(synth.seed_for(61, b, n), n, b, base)
        w = oracle.pack_rowmajor(v, b, base)
        np.testing.assert_array_equal(w, rowmajor_by_bits(v, b, base))
        np.testing.assert_array_equal(oracle.unpack_rowmajor(w, n, b, base), v)


def test_rowmajor_at_byte_widths_is_the_plain_array():
    for b, dt in [(8, np.uint8), (16, np.uint16), (32, np.uint32)]:
        n = 5000
        v = synth.uniform_values(62, n, b)
        w = oracle.pack_rowmajor(v, b)
        np.testing.assert_array_equal(w.view(dt)[:n], v.astype(dt))
        np.testing.assert_array_equal(oracle.pack_bytes(v, b), w)
        assert not w.view(dt)[n:].any()                      # zero padding to whole blocks


@pytest.mark.parametrize("b", [2, 5, 8, 12, 16, 19, 27, 32])
def test_rowmajor_and_bytes_scans_match_histogram(b):
    base = 0 if b == 32 else 100
    n = 7000
    v = synth.uniform_values(synth.seed_for(63, b), n, b, base)
    w = oracle.pack_rowmajor(v, b, base)
    for i, sigma in enumerate([1e-3, 0.1, 0.5, 1.0]):
        lo, hi = synth.pick_range(synth.seed_for(64, b, i), b, sigma, base)
        m = (v.astype(np.int64) >= lo) & (v.astype(np.int64) < hi)
        want = (int(m.sum()), int(v[m].astype(np.int64).sum()))
        assert oracle.scan_rowmajor(w, n, b, base, lo, hi) == want
        if b in (8, 16, 32):
            assert oracle.scan_bytes(oracle.pack_bytes(v, b, base), n, b, base, lo, hi) == want


def test_byte_layout_rejects_other_widths():
    with pytest.raises(ValueError):
        oracle.pack_bytes(np.arange(10, dtype=np.uint32), 12)


# ----------------------------------------------- per-block aggregate metadata
@pytest.mark.parametrize("b", [1, 9, 16, 32])
def test_blocksums_match_numpy_block_reductions(b):
    n = 5 * 1024 + 300
    base = 0 if b == 32 else 7
    v = synth.uniform_values(synth.seed_for(71, b), n, b, base)
    w = oracle.pack(v, b, base)
    pad = np.concatenate([v.astype(np.uint64), np.zeros(6 * 1024 - n, np.uint64)]).reshape(6, 1024)
    np.testing.assert_array_equal(oracle.blocksums(w, n, b, base), pad.sum(axis=1))


@pytest.mark.parametrize("p", [0.0, 0.01, 1.0])
def test_zoneagg_is_exact_and_sorted_data_scans_at_most_two_blocks(p):
    """Answering wholly-inside blocks from metadata never changes the result;
    on sorted data only the (at most two) blocks holding a range end are scanned."""
    n, b = 40 * 1024 + 77, 14
    v = synth.clustered_values(synth.seed_for(72, int(p * 100)), n, b, p)
    w = oracle.pack(v, b)
    mn, mx = oracle.zonemap(w, n, b)
    sm = oracle.blocksums(w, n, b)
    for lo, hi in [(0, 1 << b), (100, 9000), (int(v[n // 3]), int(v[n // 3]) + 1), (5000, 5000), (16000, 1 << 20)]:
        m = (v.astype(np.int64) >= lo) & (v.astype(np.int64) < hi)
        c, s, t = oracle.scan_zoneagg(w, mn, mx, sm, n, b, 0, lo, hi)
        assert (c, s) == (int(m.sum()), int(v[m].astype(np.int64).sum()))
        # the scanned blocks are exactly those neither outside nor wholly inside
        inside = (mn.astype(np.int64) >= lo) & (mx.astype(np.int64) < hi)
        outside = (mx.astype(np.int64) < lo) | (mn.astype(np.int64) >= hi)
        assert t == int(np.sum(~inside & ~outside))
        if p == 0.0:
            assert t <= 2


# ------------------------------------------------ conjunctive predicates
def test_conjunction_matches_numpy_masks():
    """COUNT of rows meeting every predicate and SUM of the aggregate column over
    them, fixed by numpy boolean masks over the raw values."""
    n = 9 * 1024 + 77
    specs = [(5, 0), (12, 300), (23, 7), (32, 0)]
    vals, cols = [], []
    for i, (b, base) in enumerate(specs):
        v = synth.uniform_values(synth.seed_for(73, i), n, b, base)
        vals.append(v)
        lo, hi = synth.pick_range(synth.seed_for(74, i), b, 0.6, base)
        cols.append((oracle.pack(v, b, base), b, base, lo, hi))
    agg_v = synth.uniform_values(75, n, 20, 9)
    agg = (oracle.pack(agg_v, 20, 9), 20, 9)
    for k in (1, 2, 4):
        m = np.ones(n, bool)
        for v, (_, b, base, lo, hi) in zip(vals[:k], cols[:k]):
            m &= (v.astype(np.int64) >= lo) & (v.astype(np.int64) < hi)
        assert oracle.scan_conj(cols[:k], n, agg) == (int(m.sum()), int(agg_v[m].astype(np.int64).sum()))
        assert oracle.scan_conj(cols[:k], n, None) == (int(m.sum()), 0)
    # one column with itself as the aggregate is the plain scan
    w, b, base, lo, hi = cols[1]
    assert oracle.scan_conj([cols[1]], n, (w, b, base)) == oracle.scan_packed(w, n, b, base, lo, hi)

