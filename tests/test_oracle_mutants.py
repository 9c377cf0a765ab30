"""The oracle's pins catch plausible mistakes: each mutant below is the oracle
source with one planted error, compiled on the CPU; the pin checks must fail
on every mutant and pass on the unmodified source."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import synth
from tests.test_oracle import hist_count_sum, layout_by_bits, rowmajor_by_bits

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "gbscan_oracle.c")

MUTANTS = {
    "inclusive upper bound": [("(int64_t)code_at(words, i, b) + (int64_t)base;\n        if (lo <= v && v < hi) {\n"
                               "            c += 1;",
                               "(int64_t)code_at(words, i, b) + (int64_t)base;\n        if (lo <= v && v <= hi) {\n"
                               "            c += 1;")],
    "base not added back": [("int64_t v = (int64_t)code_at(words, i, b) + (int64_t)base;\n        if (lo <= v && v < hi) {\n"
                             "            c += 1;",
                             "int64_t v = (int64_t)code_at(words, i, b);\n        if (lo <= v && v < hi) {\n"
                             "            c += 1;")],
    "row-major stream written MSB first": [("if ((u >> k) & 1u) out[p / 32] |= 1u << (p % 32);",
                                            "if ((u >> k) & 1u) out[p / 32] |= 1u << (31 - p % 32);")],
    "row-major straddling high word dropped": [("    if (off + b > 32) window |= (uint64_t)words[w + 1] << 32;\n"
                                                "    return (uint32_t)((window >> off) & ((1ull << b) - 1ull));\n}\n\n"
                                                "int oracle_unpack_rowmajor",
                                                "    return (uint32_t)((window >> off) & ((1ull << b) - 1ull));\n}\n\n"
                                                "int oracle_unpack_rowmajor")],
    "wholly-inside test includes hi": [("if (lo <= (int64_t)zmin[k] && (int64_t)zmax[k] < hi) {",
                                        "if (lo <= (int64_t)zmin[k] && (int64_t)zmax[k] <= hi) {")],
    "inside tail block counted whole": [("            c += (int64_t)(last - first);\n            s += (int64_t)sums[k];",
                                         "            c += (int64_t)BLOCK_VALUES;\n            s += (int64_t)sums[k];")],
    "conjunction checks only the first column": [("for (c = 0; c < k && all; ++c) {",
                                                  "for (c = 0; c < 1 && all; ++c) {")],
    "select inclusive upper bound": [("(int64_t)base;\n        if (lo <= v && v < hi) {\n            if (k < capacity)",
                                      "(int64_t)base;\n        if (lo <= v && v <= hi) {\n            if (k < capacity)")],
    "select position off by one": [("if (k < capacity) pos[k] = (uint32_t)i;\n            k += 1;\n        }\n    }\n"
                                    "    *count = k;",
                                    "if (k < capacity) pos[k] = (uint32_t)(i + 1);\n            k += 1;\n        }\n    }\n"
                                    "    *count = k;")],
    "select count stops at capacity": [("if (k < capacity) pos[k] = (uint32_t)i;\n            k += 1;\n        }\n    }\n"
                                        "    *count = k;",
                                        "if (k < capacity) { pos[k] = (uint32_t)i; k += 1; }\n        }\n    }\n"
                                        "    *count = k;")],
    "zone skip off by one": [("if ((int64_t)zmax[k] < lo || (int64_t)zmin[k] >= hi) continue;\n        touched += 1;",
                              "if ((int64_t)zmax[k] <= lo || (int64_t)zmin[k] >= hi) continue;\n        touched += 1;")],
    "tail padding in zone map": [("        uint64_t last = first + BLOCK_VALUES < n ? first + BLOCK_VALUES : n;\n"
                                  "        uint32_t mn = 0xFFFFFFFFu, mx = 0;",
                                  "        uint64_t last = first + BLOCK_VALUES;\n"
                                  "        uint32_t mn = 0xFFFFFFFFu, mx = 0;")],
    "top bit of each code dropped": [("lane)] << 32;\n    return (uint32_t)((window >> off) & ((1ull << b) - 1ull));",
                                      "lane)] << 32;\n    return (uint32_t)((window >> off) & ((1ull << (b - 1)) - 1ull));")],
    "lane and row swapped": [("uint32_t lane = (uint32_t)(j % LANES);\n        uint64_t row = j / LANES;",
                              "uint32_t lane = (uint32_t)(j / LANES);\n        uint64_t row = j % LANES;"),
                             ("uint32_t lane = (uint32_t)(j % LANES);\n    uint64_t row = j / LANES;",
                              "uint32_t lane = (uint32_t)(j / LANES);\n    uint64_t row = j % LANES;")],
    "rows in reverse order": [("uint64_t p = row * b;            /* first stream bit of this value */",
                               "uint64_t p = (31 - row) * b;     /* first stream bit of this value */"),
                              ("    uint64_t p = row * b;\n    uint64_t w = p / 32;",
                               "    uint64_t p = (31 - row) * b;\n    uint64_t w = p / 32;")],
}


class Lib:
    """ctypes view of one compiled oracle variant."""

    def __init__(self, path):
        self.l = ctypes.CDLL(path)
        u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
        i64, u64, u32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32
        self.l.oracle_pack.argtypes = [u32p, u64, u32, u32, u32p]
        self.l.oracle_unpack.argtypes = [u32p, u64, u32, u32, u32p]
        self.l.oracle_scan_packed.argtypes = [u32p, u64, u32, u32, i64, i64, ctypes.POINTER(i64),
                                              ctypes.POINTER(i64)]
        self.l.oracle_zonemap.argtypes = [u32p, u64, u32, u32, u32p, u32p]
        self.l.oracle_scan_zoneskip.argtypes = [u32p, u32p, u32p, u64, u32, u32, i64, i64, ctypes.POINTER(i64),
                                                ctypes.POINTER(i64), ctypes.POINTER(u64)]
        self.l.oracle_select_packed.argtypes = [u32p, u64, u32, u32, i64, i64, u32p, u64, ctypes.POINTER(u64)]
        u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
        self.l.oracle_blocksums.argtypes = [u32p, u64, u32, u32, u64p]
        self.l.oracle_scan_zoneagg.argtypes = [u32p, u32p, u32p, u64p, u64, u32, u32, i64, i64,
                                               ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(u64)]
        self.l.oracle_scan_conj.argtypes = [ctypes.POINTER(ctypes.c_void_p), u32p, u32p, ctypes.POINTER(i64),
                                            ctypes.POINTER(i64), u32, u64, ctypes.c_void_p, u32, u32,
                                            ctypes.POINTER(i64), ctypes.POINTER(i64)]
        self.l.oracle_pack_rowmajor.argtypes = [u32p, u64, u32, u32, u32p]
        self.l.oracle_scan_rowmajor.argtypes = [u32p, u64, u32, u32, i64, i64, ctypes.POINTER(i64),
                                                ctypes.POINTER(i64)]

    def pack(self, v, b, base=0):
        out = np.zeros(((v.size + 1023) // 1024) * 32 * b, np.uint32)
        assert self.l.oracle_pack(v, v.size, b, base, out) == 0
        return out

    def unpack(self, w, n, b, base=0):
        out = np.zeros(n, np.uint32)
        self.l.oracle_unpack(w, n, b, base, out)
        return out

    def scan(self, w, n, b, base, lo, hi):
        c, s = ctypes.c_int64(), ctypes.c_int64()
        self.l.oracle_scan_packed(w, n, b, base, lo, hi, ctypes.byref(c), ctypes.byref(s))
        return c.value, s.value

    def zonemap(self, w, n, b, base=0):
        nb = (n + 1023) // 1024
        mn, mx = np.zeros(nb, np.uint32), np.zeros(nb, np.uint32)
        self.l.oracle_zonemap(w, n, b, base, mn, mx)
        return mn, mx

    def zoneagg(self, w, mn, mx, n, b, base, lo, hi):
        sums = np.zeros((n + 1023) // 1024, np.uint64)
        self.l.oracle_blocksums(w, n, b, base, sums)
        c, s, t = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_uint64()
        self.l.oracle_scan_zoneagg(w, mn, mx, sums, n, b, base, lo, hi, ctypes.byref(c), ctypes.byref(s),
                                   ctypes.byref(t))
        return c.value, s.value, t.value

    def conj(self, cols, n):
        k = len(cols)
        ptrs = (ctypes.c_void_p * k)(*[c[0].ctypes.data for c in cols])
        bs = np.array([c[1] for c in cols], np.uint32)
        bases = np.array([c[2] for c in cols], np.uint32)
        los = (ctypes.c_int64 * k)(*[c[3] for c in cols])
        his = (ctypes.c_int64 * k)(*[c[4] for c in cols])
        c_, s_ = ctypes.c_int64(), ctypes.c_int64()
        self.l.oracle_scan_conj(ptrs, bs, bases, los, his, k, n, None, 0, 0, ctypes.byref(c_), ctypes.byref(s_))
        return c_.value

    def pack_rowmajor(self, v, b, base=0):
        out = np.zeros(((v.size + 1023) // 1024) * 32 * b, np.uint32)
        assert self.l.oracle_pack_rowmajor(v, v.size, b, base, out) == 0
        return out

    def scan_rowmajor(self, w, n, b, base, lo, hi):
        c, s = ctypes.c_int64(), ctypes.c_int64()
        self.l.oracle_scan_rowmajor(w, n, b, base, lo, hi, ctypes.byref(c), ctypes.byref(s))
        return c.value, s.value

    def select(self, w, n, b, base, lo, hi, cap):
        out, k = np.zeros(max(cap, 1), np.uint32), ctypes.c_uint64()
        self.l.oracle_select_packed(w, n, b, base, lo, hi, out, cap, ctypes.byref(k))
        return out[:min(cap, k.value)], k.value

    def zoneskip(self, w, mn, mx, n, b, base, lo, hi):
        c, s, t = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_uint64()
        self.l.oracle_scan_zoneskip(w, mn, mx, n, b, base, lo, hi, ctypes.byref(c), ctypes.byref(s), ctypes.byref(t))
        return c.value, s.value, t.value


def pins(o):
    """A compact copy of the independent pins (layout bits, round trip, brute force,
    frame of reference, zone maps, zone-skip exactness and skip rule, row-major streams,
    select positions)."""
    for b in (3, 8, 13, 32):
        for n in (1025, 4096 + 7):
            v = synth.uniform_values(synth.seed_for(77, b, n), n, b)
            w = o.pack(v, b)
            np.testing.assert_array_equal(w, layout_by_bits(v, b, 0))
            np.testing.assert_array_equal(o.unpack(w, n, b), v)
    v = synth.uniform_values(5, 1025, 3)
    w = o.pack(v, 3)
    for lo in range(-1, 10):
        for hi in range(-1, 10):
            assert o.scan(w, 1025, 3, 0, lo, hi) == hist_count_sum(v, lo, hi)
    base, b = 1000, 6
    v = synth.uniform_values(6, 3000, b, base)
    w = o.pack(v, b, base)
    for lo, hi in [(base, base + 64), (base + 5, base + 40)]:
        m = (v >= lo) & (v < hi)
        assert o.scan(w, 3000, b, base, lo, hi) == (int(m.sum()), int(v[m].astype(np.int64).sum()))
    n, b = 5000, 12
    v = synth.clustered_values(7, n, b, 0.0, 3)
    w = o.pack(v, b, 3)
    mn, mx = o.zonemap(w, n, b, 3)
    pad = np.concatenate([v, np.full(5 * 1024 - n, v[-1], np.uint32)]).reshape(5, 1024)
    np.testing.assert_array_equal(mn, pad.min(axis=1))
    np.testing.assert_array_equal(mx, pad.max(axis=1))
    for lo, hi in [(int(v[1500]), int(v[1500]) + 1), (int(v[2047]), int(v[3100])), (int(mx[0]), int(mx[0]) + 9)]:
        c, s, t = o.zoneskip(w, mn, mx, n, b, 3, lo, hi)
        m = (v >= lo) & (v < hi)
        assert (c, s) == (int(m.sum()), int(v[m].astype(np.int64).sum()))
        assert t == int(np.sum(~((mx < lo) | (mn >= hi))))
    # block aggregates: exact on sorted data with a wholly-inside run and a partial tail block
    n, b = 6 * 1024 + 500, 12
    v = synth.clustered_values(9, n, b, 0.0)
    w = o.pack(v, b)
    mn, mx = o.zonemap(w, n, b)
    for lo, hi in [(0, 1 << b), (int(v[2000]), int(mx[-1]) + 1), (int(mn[2]), int(mx[4]) + 1),
                   (int(mn[2]), int(mx[4]))]:
        m = (v.astype(np.int64) >= lo) & (v.astype(np.int64) < hi)
        c, s_, t = o.zoneagg(w, mn, mx, n, b, 0, lo, hi)
        assert (c, s_) == (int(m.sum()), int(v[m].astype(np.int64).sum()))
    # conjunction of two columns: COUNT fixed by numpy masks
    n = 3000
    va, vb = synth.uniform_values(10, n, 6), synth.uniform_values(11, n, 9)
    ca = (o.pack(va, 6), 6, 0, 10, 50)
    cb = (o.pack(vb, 9), 9, 0, 100, 400)
    m = (va >= 10) & (va < 50) & (vb >= 100) & (vb < 400)
    assert o.conj([ca, cb], n) == int(m.sum())
    # row-major layout: bit-level stream and brute-force scans
    for b in (3, 13, 24):
        v = synth.uniform_values(synth.seed_for(78, b), 2100, b)
        w = o.pack_rowmajor(v, b)
        np.testing.assert_array_equal(w, rowmajor_by_bits(v, b, 0))
        lo, hi = int(v[7]), int(v[7]) + (1 << (b - 1))
        m = (v.astype(np.int64) >= lo) & (v.astype(np.int64) < hi)
        assert o.scan_rowmajor(w, 2100, b, 0, lo, hi) == (int(m.sum()), int(v[m].astype(np.int64).sum()))
    # materializing select: positions fixed by flatnonzero; capacity keeps the full count
    n, b, base = 3000, 7, 40
    v = synth.uniform_values(8, n, b, base)
    w = o.pack(v, b, base)
    for lo, hi in [(base + 3, base + 20), (base + 100, base + 128)]:
        want = np.flatnonzero((v >= lo) & (v < hi)).astype(np.uint32)
        got, k = o.select(w, n, b, base, lo, hi, n)
        assert k == want.size
        np.testing.assert_array_equal(got, want)
        got, k = o.select(w, n, b, base, lo, hi, 5)
        assert k == want.size
        np.testing.assert_array_equal(got, want[:5])


def _compile(tmpdir, name, text):
    src = os.path.join(tmpdir, f"{name}.c")
    lib = os.path.join(tmpdir, f"{name}.so")
    with open(src, "w") as f:
        f.write(text)
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-fPIC", "-shared", "-pthread", "-o", lib, src])
    return Lib(lib)


def test_pins_pass_on_the_oracle(tmp_path):
    pins(_compile(str(tmp_path), "original", open(SRC).read()))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_the_mutant(tmp_path, name):
    text = open(SRC).read()
    for old, new in MUTANTS[name]:
        assert text.count(old) == 1, f"mutation anchor not found once: {old!r}"
        text = text.replace(old, new)
    o = _compile(str(tmp_path), "mutant", text)
    with pytest.raises(AssertionError):
        pins(o)
