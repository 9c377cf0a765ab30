"""ctypes binding of libgbscan.so (the C ABI declared in include/gbscan.h).

Argument marshalling only: every step of the scan runs in the library's
CUDA kernels.  There is no CPU fallback; if the library is missing or fails
to load, importing this module raises.  Device buffers are passed as torch
tensors (their data_ptr()) or raw integers, streams as torch.cuda.Stream or
raw cudaStream_t integers.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbscan.so")

SCAN_OK, SCAN_EINVAL, SCAN_ENOMEM, SCAN_ECUDA, SCAN_ETIMEOUT, SCAN_EBUSY, SCAN_ENOTSUP = range(7)
SCAN_AUTO, SCAN_BRANCHFREE, SCAN_BRANCHY, SCAN_ZONE_SKIP_BF, SCAN_ZONE_SKIP_BR, SCAN_ZONE_AGG_BF, SCAN_ZONE_AGG_BR = range(7)
SCAN_LAYOUT_LANES, SCAN_LAYOUT_ROWMAJOR, SCAN_LAYOUT_BYTES = range(3)
LAYOUTS = {"lanes": SCAN_LAYOUT_LANES, "rowmajor": SCAN_LAYOUT_ROWMAJOR, "bytes": SCAN_LAYOUT_BYTES}
STRATEGIES = {
    "auto": SCAN_AUTO,
    "branchfree": SCAN_BRANCHFREE,
    "branchy": SCAN_BRANCHY,
    "zone_bf": SCAN_ZONE_SKIP_BF,
    "zone_br": SCAN_ZONE_SKIP_BR,
    "zone_agg_bf": SCAN_ZONE_AGG_BF,
    "zone_agg_br": SCAN_ZONE_AGG_BR,
}


class ScanError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


class scan_pred(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int64), ("hi", ctypes.c_int64)]


class scan_shape(ctypes.Structure):
    _fields_ = [("warps", ctypes.c_uint32), ("stages", ctypes.c_uint32), ("tile_blocks", ctypes.c_uint32),
                ("vote_rows", ctypes.c_uint32), ("vec_lanes", ctypes.c_uint32)]

    def as_dict(self):
        return {"warps": int(self.warps), "stages": int(self.stages), "tile_blocks": int(self.tile_blocks),
                "vote_rows": int(self.vote_rows), "vec_lanes": int(self.vec_lanes)}


def _shape(shape) -> "scan_shape":
    if isinstance(shape, scan_shape):
        return shape
    return scan_shape(shape["warps"], shape["stages"], shape["tile_blocks"], shape.get("vote_rows", 0),
                      shape.get("vec_lanes", 0))


class scan_tune_result(ctypes.Structure):
    _fields_ = [("best", scan_shape), ("rule", scan_shape), ("best_us", ctypes.c_float),
                ("rule_us", ctypes.c_float), ("candidates", ctypes.c_uint32)]


class scan_result(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int64), ("sum", ctypes.c_int64),
                ("blocks_scanned", ctypes.c_uint64), ("reserved", ctypes.c_uint64)]

    def pair(self):
        return int(self.count), int(self.sum)


_u32p = ctypes.POINTER(ctypes.c_uint32)
_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_st = ctypes.c_int

# name -> (restype, argtypes); every function declared in include/gbscan.h
SIGNATURES = {
    "scan_last_error": (ctypes.c_char_p, []),
    "scan_status_string": (ctypes.c_char_p, [_st]),
    "scan_packed_words": (_u64, [_u64, _u32]),
    "scan_encode_host": (_st, [_vp, _u64, _u32, _u32, _vp]),
    "scan_encode_device": (_st, [_vp, _u64, _u32, _u32, _vp, _vp]),
    "scan_column_create": (_st, [_vp, _u64, _u32, _u32, _vp, ctypes.POINTER(_vp)]),
    "scan_column_create_device": (_st, [_vp, _u64, _u32, _u32, _vp, ctypes.POINTER(_vp)]),
    "scan_column_create_packed": (_st, [_vp, _u64, _u32, _u32, _vp, ctypes.POINTER(_vp)]),
    "scan_column_upload_packed": (_st, [_vp, _vp, _vp]),
    "scan_column_destroy": (_st, [_vp]),
    "scan_column_info": (_st, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u32), ctypes.POINTER(_u32),
                               ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
    "scan_zonemap_build": (_st, [_vp, _vp]),
    "scan_run": (_st, [_vp, scan_pred, _st, _vp, ctypes.POINTER(scan_result)]),
    "scan_run_async": (_st, [_vp, scan_pred, _st, _vp, _vp]),
    "scan_column_status": (_st, [_vp, _vp]),
    "scan_encode_host_layout": (_st, [_vp, _u64, _u32, _u32, ctypes.c_int, _vp]),
    "scan_encode_device_layout": (_st, [_vp, _u64, _u32, _u32, ctypes.c_int, _vp, _vp]),
    "scan_column_create_layout": (_st, [_vp, _u64, _u32, _u32, ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    "scan_column_create_device_layout": (_st, [_vp, _u64, _u32, _u32, ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    "scan_column_create_packed_layout": (_st, [_vp, _u64, _u32, _u32, ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    "scan_column_get_layout": (_st, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "scan_column_blocksums": (_st, [_vp, ctypes.POINTER(_vp)]),
    "scan_select": (_st, [_vp, scan_pred, _st, _vp, _u64, _vp, ctypes.POINTER(_u64)]),
    "scan_conj": (_st, [_vp, _vp, _u32, _vp, _st, _vp, ctypes.POINTER(scan_result)]),
    "scan_selftest_select_timeout": (_st, [_vp, _u64, _vp]),
    "scan_conj_async": (_st, [_vp, _vp, _u32, _vp, _st, _vp, _vp]),
    "scan_select_async": (_st, [_vp, scan_pred, _st, _vp, _u64, _vp, _vp]),
    "scan_probe_read": (_st, [_vp, _u64, _vp, _vp]),
    "scan_probe_triad": (_st, [_vp, _vp, _vp, ctypes.c_float, _u64, _vp]),
    "scan_launch_shape": (_st, [_u32] + [ctypes.POINTER(_u32)] * 5),
    "scan_shape_get": (_st, [_u32, _st, ctypes.POINTER(scan_shape)]),
    "scan_shape_set": (_st, [_u32, _st, ctypes.POINTER(scan_shape)]),
    "scan_shape_candidates": (_st, [_u32, _st, _vp, _u32, ctypes.POINTER(_u32)]),
    "scan_autotune_column": (_st, [_vp, scan_pred, _st, _u32, _vp, ctypes.POINTER(scan_tune_result)]),
    "scan_autotune_save": (_st, [ctypes.c_char_p]),
    "scan_autotune_load": (_st, [ctypes.c_char_p]),
    "scan_autotune_reset": (_st, []),
    "scan_batch_shape_get": (_st, [_u32, ctypes.c_int, ctypes.POINTER(scan_shape)]),
    "scan_batch_shape_set": (_st, [_u32, ctypes.c_int, ctypes.POINTER(scan_shape)]),
    "scan_batch_shape_candidates": (_st, [_u32, ctypes.c_int, _vp, _u32, ctypes.POINTER(_u32)]),
    "scan_batch_autotune": (_st, [_vp, _vp, _u32, _vp, ctypes.POINTER(_u32), ctypes.POINTER(ctypes.c_float),
                                  ctypes.POINTER(ctypes.c_float)]),
    "scan_selftest_wait_timeout": (_st, [_u64, _vp]),
    "scan_run_packed_noalloc": (_st, [_vp, _u64, _u32, _u32, scan_pred, _st, _vp, _vp, _vp]),
    "scan_batch_create": (_st, [_vp, _u32, _vp, _u32, _vp, ctypes.POINTER(_vp)]),
    "scan_batch_exec": (_st, [_vp, _vp, _vp, _vp, _vp]),
    "scan_batch_destroy": (_st, [_vp]),
    "scan_batch_status": (_st, [_vp, _vp]),
    "scan_batch_run": (_st, [_vp, _vp, _u32, _vp, _vp, _vp]),
    "scan_batch_set_strategies": (_st, [_vp, _vp]),
    "scan_batch_features": (_st, [_vp, _vp, _vp, _vp]),
    "scan_batch_law_choose": (_st, [_vp, _vp, ctypes.c_float, _vp, _vp, _vp]),
    "scan_batch_law_times": (_st, [_vp, _vp, ctypes.c_float, _vp, _vp, _vp]),
    "scan_planner_create": (_st, [_u32, _u64, ctypes.POINTER(_vp)]),
    "scan_planner_destroy": (_st, [_vp]),
    "scan_planner_param_count": (_u64, [_vp]),
    "scan_planner_get_params": (_st, [_vp, _vp]),
    "scan_planner_set_params": (_st, [_vp, _vp]),
    "scan_planner_forward": (_st, [_vp, _vp, _u32, _vp, _vp]),
    "scan_planner_gradients": (_st, [_vp, _vp, _vp, _u32, _vp, _vp, _vp]),
    "scan_planner_train_step": (_st, [_vp, _vp, _vp, _u32, ctypes.c_float, _vp, _vp]),
    "scan_planner_choose": (_st, [_vp, _vp, _u32, _vp, _vp]),
    "scan_planner_choose_margin": (_st, [_vp, _vp, _u32, ctypes.c_float, _vp, _vp]),
    "scan_planner_choose_prior": (_st, [_vp, _vp, _u32, ctypes.c_float, _vp, _vp, _vp]),
    "scan_planner_choose_guarded": (_st, [_vp, _vp, _u32, ctypes.c_float, _vp, _vp, _vp, _vp, _vp]),
    "scan_planner_save": (_st, [_vp, ctypes.c_char_p]),
    "scan_planner_load": (_st, [_vp, ctypes.c_char_p]),
    "scan_server_create": (_st, [_vp, _u32, _u32, _u64, _u32, ctypes.POINTER(_vp)]),
    "scan_server_submit": (_st, [_vp, _vp, _vp, _u32, ctypes.POINTER(_u64)]),
    "scan_server_submit_many": (_st, [_vp, _u32, _vp, _vp, _vp, _vp]),
    "scan_server_poll": (_st, [_vp, _u64, ctypes.c_int, _vp, _u32, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_int)]),
    "scan_server_stats": (_st, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u64),
                                ctypes.POINTER(_u32)]),
    "scan_server_destroy": (_st, [_vp]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the library (build it first with paper_2606_22423_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"libgbscan.so not built at {path}; run paper_2606_22423_gb300.build")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _status_name(s: int) -> str:
    return load().scan_status_string(s).decode()


def _check(status: int):
    if status != SCAN_OK:
        raise ScanError(status, load().scan_last_error().decode())


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):          # numpy array
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ------------------------------------------------------------------ thin API
def scan_packed_words(n: int, b: int) -> int:
    return int(load().scan_packed_words(n, b))


def scan_encode_host(values, b: int, base: int = 0, out=None, layout="lanes"):
    """Encode a uint32 numpy array on the host; returns the packed uint32 array."""
    import numpy as np

    v = np.ascontiguousarray(values, dtype=np.uint32)
    words = scan_packed_words(v.size, b)
    if out is None:
        out = np.zeros(max(words, 1), dtype=np.uint32)
    if layout == "lanes":
        _check(load().scan_encode_host(_ptr(v), v.size, b, base, _ptr(out)))
    else:
        _check(load().scan_encode_host_layout(_ptr(v), v.size, b, base, LAYOUTS[layout], _ptr(out)))
    return out[:words]


def scan_encode_device(dev_values, n: int, b: int, base: int, dev_out, stream=None):
    _check(load().scan_encode_device(_ptr(dev_values), n, b, base, _ptr(dev_out), _stream(stream)))


def scan_probe_read(dev_buf, nbytes: int, dev_out, stream=None):
    _check(load().scan_probe_read(_ptr(dev_buf), nbytes, _stream(stream), _ptr(dev_out)))


def scan_probe_triad(dev_a, dev_b, dev_c, s: float, n: int, stream=None):
    """STREAM triad a = b + s*c over n float32 elements (device arrays)."""
    _check(load().scan_probe_triad(_ptr(dev_a), _ptr(dev_b), _ptr(dev_c), float(s), n, _stream(stream)))


def scan_run_packed_noalloc(dev_packed, n: int, b: int, base: int, lo: int, hi: int, dev_out,
                            dev_status, strategy="branchfree", stream=None):
    """Full scan without any device allocation (static scratch inside the library)."""
    st = STRATEGIES[strategy] if isinstance(strategy, str) else int(strategy)
    _check(load().scan_run_packed_noalloc(_ptr(dev_packed), n, b, base, scan_pred(lo, hi), st,
                                          _stream(stream), _ptr(dev_out), _ptr(dev_status)))


def scan_launch_shape(b: int) -> dict:
    vals = [ctypes.c_uint32() for _ in range(5)]
    _check(load().scan_launch_shape(b, *[ctypes.byref(v) for v in vals]))
    keys = ["sms", "ctas", "warps_per_cta", "blocks_per_tile", "stages"]
    return {k: int(v.value) for k, v in zip(keys, vals)}


def _strategy(strategy) -> int:
    return STRATEGIES[strategy] if isinstance(strategy, str) else int(strategy)


def shape_get(b: int, strategy="branchfree") -> dict:
    """The launch shape the kernel of `strategy` uses at width b now."""
    out = scan_shape()
    _check(load().scan_shape_get(b, _strategy(strategy), ctypes.byref(out)))
    return out.as_dict()


def shape_set(b: int, strategy="branchfree", shape=None):
    """Install a shape (dict or scan_shape), or the built-in rule with None."""
    if shape is None:
        _check(load().scan_shape_set(b, _strategy(strategy), None))
        return
    _check(load().scan_shape_set(b, _strategy(strategy), ctypes.byref(_shape(shape))))


def shape_candidates(b: int, strategy="branchfree") -> list:
    """The autotuner's candidate shapes for (strategy, b)."""
    count = _u32()
    _check(load().scan_shape_candidates(b, _strategy(strategy), None, 0, ctypes.byref(count)))
    arr = (scan_shape * max(count.value, 1))()
    _check(load().scan_shape_candidates(b, _strategy(strategy), arr, count.value, ctypes.byref(count)))
    return [arr[i].as_dict() for i in range(count.value)]


def batch_shape_get(b: int, branchy: bool = False) -> dict:
    """The shape the batched kernel of this flavour uses for width-b groups."""
    out = scan_shape()
    _check(load().scan_batch_shape_get(b, int(bool(branchy)), ctypes.byref(out)))
    return out.as_dict()


def batch_shape_set(b: int, branchy: bool = False, shape=None):
    if shape is None:
        _check(load().scan_batch_shape_set(b, int(bool(branchy)), None))
        return
    _check(load().scan_batch_shape_set(b, int(bool(branchy)), ctypes.byref(_shape(shape))))


def batch_shape_candidates(b: int, branchy: bool = False) -> list:
    count = _u32()
    _check(load().scan_batch_shape_candidates(b, int(bool(branchy)), None, 0, ctypes.byref(count)))
    arr = (scan_shape * max(count.value, 1))()
    _check(load().scan_batch_shape_candidates(b, int(bool(branchy)), arr, count.value, ctypes.byref(count)))
    return [arr[i].as_dict() for i in range(count.value)]


def autotune_save(path: str):
    _check(load().scan_autotune_save(os.fsencode(path)))


def autotune_load(path: str):
    _check(load().scan_autotune_load(os.fsencode(path)))


def autotune_reset():
    _check(load().scan_autotune_reset())


class Column:
    """Owning handle of a scan_column."""

    def __init__(self, handle: int, keepalive=None):
        self._h = ctypes.c_void_p(handle)
        self._keep = keepalive
        n, b, base = _u64(), _u32(), _u32()
        dp, dz = _vp(), _vp()
        _check(load().scan_column_info(self._h, ctypes.byref(n), ctypes.byref(b), ctypes.byref(base),
                                       ctypes.byref(dp), ctypes.byref(dz)))
        self.n, self.b, self.base = int(n.value), int(b.value), int(base.value)
        self.dev_packed = dp.value or 0
        lay = ctypes.c_int()
        _check(load().scan_column_get_layout(self._h, ctypes.byref(lay)))
        self.layout = {v: k for k, v in LAYOUTS.items()}[lay.value]

    # constructors mirror scan_column_create{,_device,_packed}{,_layout}
    @classmethod
    def from_host(cls, values, b: int, base: int = 0, stream=None, layout="lanes") -> "Column":
        import numpy as np

        v = np.ascontiguousarray(values, dtype=np.uint32)
        h = _vp()
        _check(load().scan_column_create_layout(_ptr(v) if v.size else None, v.size, b, base, LAYOUTS[layout],
                                                _stream(stream), ctypes.byref(h)))
        return cls(h.value)

    @classmethod
    def from_device(cls, dev_values, n: int, b: int, base: int = 0, stream=None, layout="lanes") -> "Column":
        h = _vp()
        _check(load().scan_column_create_device_layout(_ptr(dev_values), n, b, base, LAYOUTS[layout],
                                                       _stream(stream), ctypes.byref(h)))
        return cls(h.value)

    @classmethod
    def from_packed(cls, dev_packed, n: int, b: int, base: int = 0, stream=None, layout="lanes") -> "Column":
        h = _vp()
        _check(load().scan_column_create_packed_layout(_ptr(dev_packed), n, b, base, LAYOUTS[layout],
                                                       _stream(stream), ctypes.byref(h)))
        return cls(h.value, keepalive=dev_packed)

    @property
    def handle(self):
        return self._h

    def upload_packed(self, host_packed, stream=None):
        _check(load().scan_column_upload_packed(self._h, _ptr(host_packed), _stream(stream)))

    def zonemap_build(self, stream=None):
        _check(load().scan_zonemap_build(self._h, _stream(stream)))

    def zonemap_ptr(self) -> int:
        dz = _vp()
        _check(load().scan_column_info(self._h, None, None, None, None, ctypes.byref(dz)))
        return dz.value or 0

    def autotune(self, lo: int, hi: int, strategy="branchfree", reps: int = 3, stream=None) -> dict:
        """Tune the kernel of `strategy` at this column's width (scan_autotune_column)."""
        out = scan_tune_result()
        _check(load().scan_autotune_column(self._h, scan_pred(lo, hi), _strategy(strategy), reps, _stream(stream),
                                           ctypes.byref(out)))
        return {"best": out.best.as_dict(), "rule": out.rule.as_dict(), "best_us": float(out.best_us),
                "rule_us": float(out.rule_us), "candidates": int(out.candidates)}

    def run(self, lo: int, hi: int, strategy="branchfree", stream=None) -> scan_result:
        st = STRATEGIES[strategy] if isinstance(strategy, str) else int(strategy)
        out = scan_result()
        _check(load().scan_run(self._h, scan_pred(lo, hi), st, _stream(stream), ctypes.byref(out)))
        return out

    def run_async(self, lo: int, hi: int, dev_out, strategy="branchfree", stream=None):
        st = STRATEGIES[strategy] if isinstance(strategy, str) else int(strategy)
        _check(load().scan_run_async(self._h, scan_pred(lo, hi), st, _stream(stream), _ptr(dev_out)))

    def select(self, lo: int, hi: int, positions=None, strategy="branchfree", stream=None,
               capacity=None) -> int:
        """Materializing select: positions (uint32 bits in a device int32 tensor, in
        increasing order) of the values in [lo, hi); returns the full match count.
        Only the first min(count, capacity) positions are written."""
        st = STRATEGIES[strategy] if isinstance(strategy, str) else int(strategy)
        cap = (0 if positions is None else positions.numel()) if capacity is None else int(capacity)
        count = _u64()
        _check(load().scan_select(self._h, scan_pred(lo, hi), st, _ptr(positions), cap, _stream(stream),
                                  ctypes.byref(count)))
        return int(count.value)

    def select_async(self, lo: int, hi: int, positions, dev_count, strategy="branchfree", stream=None,
                     capacity=None):
        """As select, with the count written to device memory (one int64)."""
        st = STRATEGIES[strategy] if isinstance(strategy, str) else int(strategy)
        cap = (0 if positions is None else positions.numel()) if capacity is None else int(capacity)
        _check(load().scan_select_async(self._h, scan_pred(lo, hi), st, _ptr(positions), cap, _stream(stream),
                                        _ptr(dev_count)))

    @property
    def dev_blocksums(self) -> int:
        """Device address of the per-block sums (0 before zonemap_build)."""
        p = _vp()
        _check(load().scan_column_blocksums(self._h, ctypes.byref(p)))
        return p.value or 0

    def status(self, stream=None):
        _check(load().scan_column_status(self._h, _stream(stream)))

    def close(self):
        if self._h is not None and self._h.value:
            _check(load().scan_column_destroy(self._h))
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _strategy_array(strategies, n):
    if strategies is None:
        return None
    arr = (ctypes.c_int * n)(*[STRATEGIES[x] if isinstance(x, str) else int(x) for x in strategies])
    return arr


class Batch:
    """A planned batch over many columns (scan_batch_create / _exec / _destroy)."""

    def __init__(self, columns, strategies=None, tiles_per_pop: int = 0, stream=None):
        self.columns = list(columns)
        n = len(self.columns)
        self._cols = (_vp * max(n, 1))(*[c.handle.value for c in self.columns])
        self._strats = _strategy_array(strategies, n)
        h = _vp()
        _check(load().scan_batch_create(self._cols, n, self._strats, tiles_per_pop, _stream(stream),
                                        ctypes.byref(h)))
        self._h = h

    def set_strategies(self, strategies):
        n = len(self.columns)
        self._strats = _strategy_array(strategies, n)
        _check(load().scan_batch_set_strategies(self._h, self._strats))

    def features(self, preds, dev_features, stream=None):
        """Planner features (ncols x 4 float32, device) for these predicates."""
        n = len(self.columns)
        pr = (scan_pred * max(n, 1))(*[scan_pred(int(lo), int(hi)) for lo, hi in preds])
        _check(load().scan_batch_features(self._h, pr, _stream(stream), _ptr(dev_features)))

    def law_choose(self, dev_features, beta_bytes_per_s, t_dec_values_per_s, dev_choice, stream=None):
        """Strategy per column (int32, device) from the bandwidth law with fitted T_dec."""
        td = (ctypes.c_float * 4)(*[float(x) for x in t_dec_values_per_s])
        _check(load().scan_batch_law_choose(self._h, _ptr(dev_features), float(beta_bytes_per_s), td,
                                            _stream(stream), _ptr(dev_choice)))

    def law_times(self, dev_features, beta_bytes_per_s, t_dec_values_per_s, dev_log_ms, stream=None):
        """The law's predicted log milliseconds per (column, strategy) (float32, device, ncols x 4)."""
        td = (ctypes.c_float * 4)(*[float(x) for x in t_dec_values_per_s])
        _check(load().scan_batch_law_times(self._h, _ptr(dev_features), float(beta_bytes_per_s), td,
                                           _stream(stream), _ptr(dev_log_ms)))

    @staticmethod
    def pred_array(preds):
        """Marshal predicates once (reusable across runs)."""
        return (scan_pred * max(len(preds), 1))(*[scan_pred(int(lo), int(hi)) for lo, hi in preds])

    def run(self, preds, stream=None, dev_out=None, host=True):
        n = len(self.columns)
        pr = preds if isinstance(preds, ctypes.Array) else self.pred_array(preds)
        out = (scan_result * max(n, 1))() if host else None
        _check(load().scan_batch_exec(self._h, pr, _stream(stream), out if host else None, _ptr(dev_out)))
        return [out[i] for i in range(n)] if host else None

    def status(self, stream=None):
        """Raise ScanError (SCAN_ETIMEOUT) if the last replay's device waits gave up."""
        _check(load().scan_batch_status(self._h, _stream(stream)))

    def autotune(self, preds, reps: int = 3, stream=None) -> dict:
        """Tune the width groups' kernels on these predicates (scan_batch_autotune): groups
        changed, and the graph replay's time with the rule and the installed shapes."""
        pr = preds if isinstance(preds, ctypes.Array) else self.pred_array(preds)
        groups, rule, tuned = _u32(), ctypes.c_float(), ctypes.c_float()
        _check(load().scan_batch_autotune(self._h, pr, reps, _stream(stream), ctypes.byref(groups),
                                          ctypes.byref(rule), ctypes.byref(tuned)))
        return {"groups": int(groups.value), "rule_us": float(rule.value), "tuned_us": float(tuned.value)}

    def close(self):
        if self._h is not None and self._h.value:
            _check(load().scan_batch_destroy(self._h))
            self._h = _vp(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def scan_conj(columns, preds, agg=None, stream=None) -> scan_result:
    """Conjunctive scan: COUNT of rows meeting every (lo, hi) of `preds` on the
    matching `columns`, and SUM of `agg` (a Column or None) over those rows."""
    k = len(columns)
    cols = (_vp * max(k, 1))(*[c.handle.value for c in columns])
    pr = (scan_pred * max(k, 1))(*[scan_pred(lo, hi) for lo, hi in preds])
    out = scan_result()
    _check(load().scan_conj(cols, pr, k, agg.handle if agg is not None else None, SCAN_BRANCHFREE,
                            _stream(stream), ctypes.byref(out)))
    return out


class Conj:
    """A prepared conjunctive query (argument arrays marshalled once) for
    repeated asynchronous runs with the result in device memory."""

    def __init__(self, columns, preds, agg=None):
        self.k = len(columns)
        self._cols = (_vp * max(self.k, 1))(*[c.handle.value for c in columns])
        self._preds = (scan_pred * max(self.k, 1))(*[scan_pred(lo, hi) for lo, hi in preds])
        self._agg = agg.handle if agg is not None else None
        self._keep = (list(columns), agg)

    def run_async(self, dev_out, stream=None):
        _check(load().scan_conj_async(self._cols, self._preds, self.k, self._agg, SCAN_BRANCHFREE, _stream(stream),
                                      _ptr(dev_out)))


def scan_batch_run(columns, preds, strategies=None, stream=None):
    """One-shot batch with host results."""
    n = len(columns)
    cols = (_vp * max(n, 1))(*[c.handle.value for c in columns])
    pr = (scan_pred * max(n, 1))(*[scan_pred(int(lo), int(hi)) for lo, hi in preds])
    out = (scan_result * max(n, 1))()
    _check(load().scan_batch_run(cols, pr, n, _strategy_array(strategies, n), _stream(stream), out))
    return [out[i] for i in range(n)]


STRATEGY_ORDER = ["branchfree", "branchy", "zone_bf", "zone_br"]   # planner output index -> strategy


class Planner:
    """The planner network on the GPU (scan_planner_*): 4 -> 64 -> 64 -> S."""

    def __init__(self, n_strategies: int = 4, seed: int = 1):
        h = _vp()
        _check(load().scan_planner_create(n_strategies, seed, ctypes.byref(h)))
        self._h = h
        self.S = n_strategies
        self.nparams = int(load().scan_planner_param_count(self._h))

    def get_params(self):
        import numpy as np

        out = np.zeros(self.nparams, dtype=np.float32)
        _check(load().scan_planner_get_params(self._h, _ptr(out)))
        return out

    def set_params(self, params):
        import numpy as np

        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == self.nparams
        _check(load().scan_planner_set_params(self._h, _ptr(p)))

    def forward(self, dev_x, rows, dev_y, stream=None):
        _check(load().scan_planner_forward(self._h, _ptr(dev_x), rows, _ptr(dev_y), _stream(stream)))

    def gradients(self, dev_x, dev_t, rows, dev_grads, stream=None):
        loss = ctypes.c_float()
        _check(load().scan_planner_gradients(self._h, _ptr(dev_x), _ptr(dev_t), rows, _ptr(dev_grads),
                                             _stream(stream), ctypes.byref(loss)))
        return float(loss.value)

    def train_step(self, dev_x, dev_t, rows, lr, stream=None, want_loss=False):
        loss = ctypes.c_float()
        _check(load().scan_planner_train_step(self._h, _ptr(dev_x), _ptr(dev_t), rows, float(lr),
                                              _stream(stream), ctypes.byref(loss) if want_loss else None))
        return float(loss.value) if want_loss else None

    def choose(self, dev_x, rows, dev_choice, stream=None, margin=0.0, dev_prior=None):
        if dev_prior is not None:
            _check(load().scan_planner_choose_prior(self._h, _ptr(dev_x), rows, float(margin), _ptr(dev_prior),
                                                    _ptr(dev_choice), _stream(stream)))
        elif margin:
            _check(load().scan_planner_choose_margin(self._h, _ptr(dev_x), rows, float(margin), _ptr(dev_choice),
                                                     _stream(stream)))
        else:
            _check(load().scan_planner_choose(self._h, _ptr(dev_x), rows, _ptr(dev_choice), _stream(stream)))

    def choose_guarded(self, dev_x, rows, margin, dev_fallback, dev_fallback_log_ms, dev_choice, stream=None,
                       feature_box=None):
        """The fallback's choice unless the row lies inside feature_box (lo[4] + hi[4],
        or None) and the network predicts another available strategy faster by more
        than `margin` (scan_planner_choose_guarded)."""
        box = None if feature_box is None else (ctypes.c_float * 8)(*[float(v) for v in feature_box])
        _check(load().scan_planner_choose_guarded(self._h, _ptr(dev_x), rows, float(margin), _ptr(dev_fallback),
                                                  _ptr(dev_fallback_log_ms), box, _ptr(dev_choice),
                                                  _stream(stream)))

    def save(self, path):
        _check(load().scan_planner_save(self._h, path.encode()))

    def load_file(self, path):
        _check(load().scan_planner_load(self._h, path.encode()))

    def close(self):
        if self._h is not None and self._h.value:
            _check(load().scan_planner_destroy(self._h))
            self._h = _vp(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching scan server over a device-resident table (scan_server_*)."""

    def __init__(self, columns, slots=3, device_bytes_per_slot=1 << 20, max_queue=4096):
        self.columns = list(columns)
        n = len(self.columns)
        self._cols = (_vp * n)(*[c.handle.value for c in self.columns])
        h = _vp()
        _check(load().scan_server_create(self._cols, n, slots, device_bytes_per_slot, max_queue,
                                         ctypes.byref(h)))
        self._h = h

    def submit(self, col_ids, preds):
        n = len(col_ids)
        ids = (ctypes.c_uint32 * n)(*col_ids)
        pr = (scan_pred * n)(*[scan_pred(int(lo), int(hi)) for lo, hi in preds])
        q = _u64()
        _check(load().scan_server_submit(self._h, ids, pr, n, ctypes.byref(q)))
        return int(q.value)

    def submit_many(self, queries):
        """Submit a burst of (col_ids, preds) queries atomically; returns their ids."""
        offs = [0]
        ids, prs = [], []
        for c, p in queries:
            ids += list(c)
            prs += list(p)
            offs.append(len(ids))
        n = len(queries)
        o = (ctypes.c_uint32 * (n + 1))(*offs)
        ci = (ctypes.c_uint32 * max(len(ids), 1))(*ids)
        pr = (scan_pred * max(len(prs), 1))(*[scan_pred(int(lo), int(hi)) for lo, hi in prs])
        out = (ctypes.c_uint64 * max(n, 1))()
        _check(load().scan_server_submit_many(self._h, n, o, ci, pr, out))
        return [int(out[i]) for i in range(n)]

    def poll(self, query_id, n, wait=False):
        """(done, results, latency_us); results is a list of scan_result when done."""
        out = (scan_result * max(n, 1))()
        lat = ctypes.c_double()
        done = ctypes.c_int()
        _check(load().scan_server_poll(self._h, query_id, 1 if wait else 0, out, n, ctypes.byref(lat),
                                       ctypes.byref(done)))
        if not done.value:
            return False, None, None
        return True, [out[i] for i in range(n)], float(lat.value)

    def stats(self):
        b, e, r = _u64(), _u64(), _u64()
        q = _u32()
        _check(load().scan_server_stats(self._h, ctypes.byref(b), ctypes.byref(e), ctypes.byref(r),
                                        ctypes.byref(q)))
        return {"batches": int(b.value), "column_scans": int(e.value), "rejected": int(r.value),
                "queued": int(q.value)}

    def close(self):
        if self._h is not None and self._h.value:
            _check(load().scan_server_destroy(self._h))
            self._h = _vp(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
