"""The C ABI without a GPU: the library loads, exports every function that
include/gbscan.h declares, and its host-side logic (layout sizes, the host
encoder, argument checks) agrees with the oracle."""
import os
import re

import numpy as np
import pytest

import oracle
import synth
from paper_2606_22423_gb300 import gbscan

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(scan_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    return gbscan.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), f"{name} declared but not exported"
        assert name in gbscan.SIGNATURES, f"{name} has no binding"


def test_packed_words(lib):
    for n in [0, 1, 1023, 1024, 1025, 1 << 31]:
        for b in [1, 7, 32]:
            assert gbscan.scan_packed_words(n, b) == oracle.packed_words(n, b)
    assert gbscan.scan_packed_words(5, 0) == 0 and gbscan.scan_packed_words(5, 33) == 0


@pytest.mark.parametrize("b", range(1, 33))
def test_host_encoder_is_byte_identical_to_the_oracle(lib, b):
    max_base = (1 << 32) - (1 << b)
    for n, base in [(1, 0), (1000, min(77, max_base)), (1024, max_base), (3 * 1024 + 5, 0),
                    (70 * 1024 + 999, min(12345, max_base))]:
        v = synth.uniform_values(synth.seed_for(80, b, n), n, b, base)
        got = gbscan.scan_encode_host(v, b, base)
        np.testing.assert_array_equal(got, oracle.pack(v, b, base))


@pytest.mark.parametrize("b", [1, 3, 8, 11, 16, 24, 31, 32])
def test_host_rowmajor_and_byte_encoders_match_the_oracle(lib, b):
    """Paper §3 strategies (i) and (iii): the host encoder writes the oracle's
    row-major stream; the byte layout is that stream at b = 8/16/32."""
    for n, base in [(1, 0), (1500, 0 if b == 32 else 3), (5 * 1024 + 7, 0)]:
        v = synth.uniform_values(synth.seed_for(81, b, n), n, b, base)
        got = gbscan.scan_encode_host(v, b, base, layout="rowmajor")
        np.testing.assert_array_equal(got, oracle.pack_rowmajor(v, b, base))
        if b in (8, 16, 32):
            np.testing.assert_array_equal(gbscan.scan_encode_host(v, b, base, layout="bytes"),
                                          oracle.pack_bytes(v, b, base))
    with pytest.raises(gbscan.ScanError):
        gbscan.scan_encode_host(np.arange(10, dtype=np.uint32), 12, 0, layout="bytes")


def test_host_encoder_rejects_bad_input(lib):
    v = np.array([1, 2, 3, 400], dtype=np.uint32)
    for b, base, why in [(8, 0, "outside"), (0, 0, "width"), (33, 0, "width"), (9, 2, "outside"),
                         (32, 1, "width")]:
        with pytest.raises(gbscan.ScanError) as e:
            gbscan.scan_encode_host(v, b, base)
        assert e.value.status == gbscan.SCAN_EINVAL
        assert why in str(e.value)


def test_status_strings(lib):
    assert gbscan._status_name(gbscan.SCAN_ETIMEOUT) == "SCAN_ETIMEOUT"
    assert gbscan._status_name(99) == "SCAN_UNKNOWN"


def test_launch_shapes_fit_shared_memory(lib):
    for b in range(1, 33):
        # shape queries need no device for the per-width part
        st = gbscan.load().scan_launch_shape
        import ctypes

        vals = [ctypes.c_uint32() for _ in range(5)]
        assert st(b, None, None, *[ctypes.byref(v) for v in vals[2:]]) == gbscan.SCAN_OK
        warps, tb, stages = (int(v.value) for v in vals[2:])
        step = 4 if b <= 16 else 2          # blocks per warp step (lanes per thread)
        assert tb % step == 0 and tb >= step
        assert tb * 128 * b <= 8 * 1024      # a tile fits one 8 KB slot
        assert warps * stages * tb * 128 * b <= 227 * 1024


def test_triad_probe_rejects_bad_arguments(lib):
    """Argument checks run before any CUDA call: misaligned arrays, n not a
    multiple of 4 and NULL arrays are refused (the pointers are never touched)."""
    for a, b, c, n, why in [(0x1000, 0x2000, 0x3000, 6, "multiple of 4"), (0x1004, 0x2000, 0x3000, 8, "aligned"),
                            (0x1000, 0x2008, 0x3000, 8, "aligned"), (None, 0x2000, 0x3000, 8, "null")]:
        with pytest.raises(gbscan.ScanError) as e:
            gbscan.scan_probe_triad(a, b, c, 3.0, n)
        assert e.value.status == gbscan.SCAN_EINVAL
        assert why in str(e.value)


def test_device_result_pointers_must_be_aligned(lib):
    """The kernels store 64-bit words to the result and a 32-bit status word: a
    misaligned caller pointer is refused with SCAN_EINVAL before any CUDA call
    (the pointers below are never touched)."""
    import ctypes

    for out, status, why in [(0x2004, 0x3000, "dev_out must be 8-byte aligned"),
                             (0x2000, 0x3002, "dev_status must be 4-byte aligned")]:
        with pytest.raises(gbscan.ScanError) as e:
            gbscan.scan_run_packed_noalloc(0x1000, 4096, 9, 0, 0, 10, out, status)
        assert e.value.status == gbscan.SCAN_EINVAL and why in str(e.value)
    # scan_run_async checks its result pointer before it reads the column handle
    rc = lib.scan_run_async(ctypes.c_void_p(0x10), gbscan.scan_pred(0, 10), gbscan.SCAN_BRANCHFREE, None,
                            ctypes.c_void_p(0x2001))
    assert rc == gbscan.SCAN_EINVAL
    assert "8-byte aligned" in lib.scan_last_error().decode()
