"""CPU oracle for the fused columnar scan (paper §2-§3).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / reference leg are the only callers.  The
product library never imports this package and this package never imports
the product library; the two share only the seeded generators in ``synth``.

The arithmetic lives in plain C (``gbscan_oracle.c``), built with gcc into
``oracle/_build/liboracle.so``.  This module only marshals numpy arrays.
Every function is pinned in ``tests/test_oracle.py`` against facts that do
not come from the oracle itself (bit-level layout definition, reductions to
numpy reshapes at b = 8/16/32, histogram brute force, closed forms).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gbscan_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
EINVAL = 1

_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (portable flags only; it also runs on Arm)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_n_blocks.restype = _u64
            lib.oracle_n_blocks.argtypes = [_u64]
            lib.oracle_packed_words.restype = _u64
            lib.oracle_packed_words.argtypes = [_u64, _u32]
            lib.oracle_pack.restype = ctypes.c_int
            lib.oracle_pack.argtypes = [_u32p, _u64, _u32, _u32, _u32p]
            lib.oracle_unpack.restype = ctypes.c_int
            lib.oracle_unpack.argtypes = [_u32p, _u64, _u32, _u32, _u32p]
            lib.oracle_scan_values.restype = None
            lib.oracle_scan_values.argtypes = [
                _u32p, _u64, _i64, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
            lib.oracle_scan_packed.restype = ctypes.c_int
            lib.oracle_scan_packed.argtypes = [
                _u32p, _u64, _u32, _u32, _i64, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
            lib.oracle_zonemap.restype = ctypes.c_int
            lib.oracle_zonemap.argtypes = [_u32p, _u64, _u32, _u32, _u32p, _u32p]
            lib.oracle_scan_zoneskip.restype = ctypes.c_int
            lib.oracle_scan_zoneskip.argtypes = [
                _u32p, _u32p, _u32p, _u64, _u32, _u32, _i64, _i64,
                ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_u64)]
            lib.oracle_scan_conj.restype = ctypes.c_int
            lib.oracle_scan_conj.argtypes = [
                ctypes.POINTER(ctypes.c_void_p), _u32p, _u32p, ctypes.POINTER(_i64), ctypes.POINTER(_i64), _u32,
                _u64, ctypes.c_void_p, _u32, _u32, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
            lib.oracle_blocksums.restype = ctypes.c_int
            lib.oracle_blocksums.argtypes = [_u32p, _u64, _u32, _u32, _u64p]
            lib.oracle_scan_zoneagg.restype = ctypes.c_int
            lib.oracle_scan_zoneagg.argtypes = [
                _u32p, _u32p, _u32p, _u64p, _u64, _u32, _u32, _i64, _i64, ctypes.POINTER(_i64),
                ctypes.POINTER(_i64), ctypes.POINTER(_u64)]
            lib.oracle_pack_rowmajor.restype = ctypes.c_int
            lib.oracle_pack_rowmajor.argtypes = [_u32p, _u64, _u32, _u32, _u32p]
            lib.oracle_unpack_rowmajor.restype = ctypes.c_int
            lib.oracle_unpack_rowmajor.argtypes = [_u32p, _u64, _u32, _u32, _u32p]
            lib.oracle_scan_rowmajor.restype = ctypes.c_int
            lib.oracle_scan_rowmajor.argtypes = [
                _u32p, _u64, _u32, _u32, _i64, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
            lib.oracle_pack_bytes.restype = ctypes.c_int
            lib.oracle_pack_bytes.argtypes = [_u32p, _u64, _u32, _u32, _u32p]
            lib.oracle_scan_bytes.restype = ctypes.c_int
            lib.oracle_scan_bytes.argtypes = [
                _u32p, _u64, _u32, _u32, _i64, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
            lib.oracle_select_values.restype = _u64
            lib.oracle_select_values.argtypes = [_u32p, _u64, _i64, _i64, _u32p, _u64]
            lib.oracle_select_packed.restype = ctypes.c_int
            lib.oracle_select_packed.argtypes = [
                _u32p, _u64, _u32, _u32, _i64, _i64, _u32p, _u64, ctypes.POINTER(_u64)]
            lib.oracle_scan_packed_threads.restype = ctypes.c_int
            lib.oracle_scan_packed_threads.argtypes = [
                _u32p, _u64, _u32, _u32, _i64, _i64, ctypes.c_int,
                ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
            _lib = lib
    return _lib


def _u32arr(a) -> np.ndarray:
    a = np.ascontiguousarray(a)
    if a.dtype != np.uint32:
        raise TypeError(f"expected uint32 array, got {a.dtype}")
    return a


def n_blocks(n: int) -> int:
    return int(_load().oracle_n_blocks(n))


def packed_words(n: int, b: int) -> int:
    return int(_load().oracle_packed_words(n, b))


def pack(values, b: int, base: int = 0) -> np.ndarray:
    """Lane-interleaved FOR encoding of ``values`` (uint32) at ``b`` bits."""
    v = _u32arr(values)
    n = v.size
    out = np.zeros(max(packed_words(n, b), 1), dtype=np.uint32)
    rc = _load().oracle_pack(v if n else np.zeros(1, np.uint32), n, b, base, out)
    if rc != OK:
        raise ValueError(f"oracle_pack rejected the input (b={b}, base={base})")
    return out[: packed_words(n, b)]


def unpack(words, n: int, b: int, base: int = 0) -> np.ndarray:
    w = _u32arr(words)
    out = np.zeros(max(n, 1), dtype=np.uint32)
    rc = _load().oracle_unpack(w if w.size else np.zeros(1, np.uint32), n, b, base, out)
    if rc != OK:
        raise ValueError("oracle_unpack rejected the input")
    return out[:n]


def scan_values(values, lo: int, hi: int) -> tuple[int, int]:
    """Brute force COUNT and SUM of lo <= v < hi over raw values."""
    v = _u32arr(values)
    c, s = _i64(), _i64()
    _load().oracle_scan_values(v if v.size else np.zeros(1, np.uint32), v.size, lo, hi,
                               ctypes.byref(c), ctypes.byref(s))
    return c.value, s.value


def scan_packed(words, n: int, b: int, base: int, lo: int, hi: int) -> tuple[int, int]:
    """Fused decode -> filter -> aggregate over a packed column."""
    w = _u32arr(words)
    c, s = _i64(), _i64()
    rc = _load().oracle_scan_packed(w if w.size else np.zeros(1, np.uint32), n, b, base, lo, hi,
                                    ctypes.byref(c), ctypes.byref(s))
    if rc != OK:
        raise ValueError("oracle_scan_packed rejected the input")
    return c.value, s.value


def scan_packed_threads(words, n: int, b: int, base: int, lo: int, hi: int,
                        threads: int) -> tuple[int, int]:
    w = _u32arr(words)
    c, s = _i64(), _i64()
    rc = _load().oracle_scan_packed_threads(w if w.size else np.zeros(1, np.uint32), n, b, base,
                                            lo, hi, threads, ctypes.byref(c), ctypes.byref(s))
    if rc != OK:
        raise ValueError("oracle_scan_packed_threads rejected the input")
    return c.value, s.value


def zonemap(words, n: int, b: int, base: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Per-block (min, max) of decoded values."""
    w = _u32arr(words)
    nb = n_blocks(n)
    zmin = np.zeros(max(nb, 1), dtype=np.uint32)
    zmax = np.zeros(max(nb, 1), dtype=np.uint32)
    rc = _load().oracle_zonemap(w if w.size else np.zeros(1, np.uint32), n, b, base, zmin, zmax)
    if rc != OK:
        raise ValueError("oracle_zonemap rejected the input")
    return zmin[:nb], zmax[:nb]


def scan_zoneskip(words, zmin, zmax, n: int, b: int, base: int, lo: int, hi: int):
    """Zone-map skipping scan; returns (count, sum, blocks_scanned)."""
    w = _u32arr(words)
    zmn, zmx = _u32arr(zmin), _u32arr(zmax)
    c, s, t = _i64(), _i64(), _u64()
    one = np.zeros(1, np.uint32)
    rc = _load().oracle_scan_zoneskip(w if w.size else one, zmn if zmn.size else one,
                                      zmx if zmx.size else one, n, b, base, lo, hi,
                                      ctypes.byref(c), ctypes.byref(s), ctypes.byref(t))
    if rc != OK:
        raise ValueError("oracle_scan_zoneskip rejected the input")
    return c.value, s.value, t.value


def select_values(values, lo: int, hi: int, capacity: int | None = None):
    """Positions (uint32, increasing) of raw values in [lo, hi), and the full count."""
    v = _u32arr(values)
    cap = v.size if capacity is None else capacity
    out = np.zeros(max(cap, 1), np.uint32)
    k = int(_load().oracle_select_values(v if v.size else np.zeros(1, np.uint32), v.size, lo, hi, out, cap))
    return out[:min(k, cap)], k


def select_packed(words, n: int, b: int, base: int, lo: int, hi: int, capacity: int | None = None):
    """Materializing select over a packed column: (positions, full count)."""
    w = _u32arr(words)
    cap = n if capacity is None else capacity
    out = np.zeros(max(cap, 1), np.uint32)
    k = _u64()
    rc = _load().oracle_select_packed(w if w.size else np.zeros(1, np.uint32), n, b, base, lo, hi, out, cap,
                                      ctypes.byref(k))
    if rc != OK:
        raise ValueError("oracle_select_packed rejected the input")
    return out[:min(k.value, cap)], int(k.value)


def pack_rowmajor(values, b: int, base: int = 0) -> np.ndarray:
    """Row-major bit stream (paper §3 strategy (i)) of ``values``, padded to whole blocks."""
    v = _u32arr(values)
    out = np.zeros(max(packed_words(v.size, b), 1), np.uint32)
    if _load().oracle_pack_rowmajor(v if v.size else np.zeros(1, np.uint32), v.size, b, base, out) != OK:
        raise ValueError("oracle_pack_rowmajor rejected the input")
    return out[:packed_words(v.size, b)]


def unpack_rowmajor(words, n: int, b: int, base: int = 0) -> np.ndarray:
    w = _u32arr(words)
    out = np.zeros(max(n, 1), np.uint32)
    if _load().oracle_unpack_rowmajor(w if w.size else np.zeros(2, np.uint32), n, b, base, out) != OK:
        raise ValueError("oracle_unpack_rowmajor rejected the input")
    return out[:n]


def scan_rowmajor(words, n: int, b: int, base: int, lo: int, hi: int):
    w = _u32arr(words)
    c, s = _i64(), _i64()
    if _load().oracle_scan_rowmajor(w if w.size else np.zeros(2, np.uint32), n, b, base, lo, hi,
                                    ctypes.byref(c), ctypes.byref(s)) != OK:
        raise ValueError("oracle_scan_rowmajor rejected the input")
    return c.value, s.value


def pack_bytes(values, b: int, base: int = 0) -> np.ndarray:
    """Byte-aligned codes (paper §3 strategy (iii), b in {8, 16, 32}) as 32-bit words, padded to whole blocks."""
    v = _u32arr(values)
    out = np.zeros(max(packed_words(v.size, b), 1), np.uint32)
    if _load().oracle_pack_bytes(v if v.size else np.zeros(1, np.uint32), v.size, b, base, out) != OK:
        raise ValueError("oracle_pack_bytes rejected the input")
    return out[:packed_words(v.size, b)]


def scan_bytes(words, n: int, b: int, base: int, lo: int, hi: int):
    w = _u32arr(words)
    c, s = _i64(), _i64()
    if _load().oracle_scan_bytes(w if w.size else np.zeros(1, np.uint32), n, b, base, lo, hi,
                                 ctypes.byref(c), ctypes.byref(s)) != OK:
        raise ValueError("oracle_scan_bytes rejected the input")
    return c.value, s.value


def blocksums(words, n: int, b: int, base: int = 0) -> np.ndarray:
    """Per-block sum of decoded values over valid positions (uint64)."""
    w = _u32arr(words)
    nb = n_blocks(n)
    out = np.zeros(max(nb, 1), np.uint64)
    if _load().oracle_blocksums(w if w.size else np.zeros(1, np.uint32), n, b, base, out) != OK:
        raise ValueError("oracle_blocksums rejected the input")
    return out[:nb]


def scan_zoneagg(words, zmin, zmax, sums, n: int, b: int, base: int, lo: int, hi: int):
    """Scan answering blocks wholly inside [lo, hi) from (min, max, sum); returns
    (count, sum, blocks_scanned)."""
    w = _u32arr(words)
    zmn, zmx = _u32arr(zmin), _u32arr(zmax)
    sm = np.ascontiguousarray(sums, dtype=np.uint64)
    c, s, t = _i64(), _i64(), _u64()
    one, one64 = np.zeros(1, np.uint32), np.zeros(1, np.uint64)
    rc = _load().oracle_scan_zoneagg(w if w.size else one, zmn if zmn.size else one, zmx if zmx.size else one,
                                     sm if sm.size else one64, n, b, base, lo, hi,
                                     ctypes.byref(c), ctypes.byref(s), ctypes.byref(t))
    if rc != OK:
        raise ValueError("oracle_scan_zoneagg rejected the input")
    return c.value, s.value, t.value


def scan_conj(columns, n: int, agg=None):
    """Conjunctive scan: columns = [(words, b, base, lo, hi), ...] of n rows each;
    agg = (words, b, base) or None.  Returns (count, sum of agg over matching rows)."""
    k = len(columns)
    ws = [_u32arr(c[0]) for c in columns]
    ptrs = (ctypes.c_void_p * max(k, 1))(*[w.ctypes.data for w in ws])
    bs = np.array([c[1] for c in columns] or [1], np.uint32)
    bases = np.array([c[2] for c in columns] or [0], np.uint32)
    los = (_i64 * max(k, 1))(*[c[3] for c in columns])
    his = (_i64 * max(k, 1))(*[c[4] for c in columns])
    aw = _u32arr(agg[0]) if agg is not None else None
    cnt, sm = _i64(), _i64()
    rc = _load().oracle_scan_conj(ptrs, bs, bases, los, his, k, n, aw.ctypes.data if aw is not None else None,
                                  agg[1] if agg else 0, agg[2] if agg else 0, ctypes.byref(cnt), ctypes.byref(sm))
    if rc != OK:
        raise ValueError("oracle_scan_conj rejected the input")
    return cnt.value, sm.value
