"""Raw device-to-host copies for tests (the CUDA runtime torch already loaded)."""
import ctypes
import ctypes.util

import numpy as np

_rt = None


def _lib():
    global _rt
    if _rt is None:
        import torch  # noqa: F401  (makes sure the runtime is loaded first)

        for name in ("libcudart.so.13", "libcudart.so"):
            try:
                _rt = ctypes.CDLL(name)
                break
            except OSError:
                continue
        if _rt is None:
            _rt = ctypes.CDLL("/usr/local/cuda/lib64/libcudart.so")
        _rt.cudaMemcpy.restype = ctypes.c_int
        _rt.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    return _rt


def d2h_u32(dev_ptr: int, count: int) -> np.ndarray:
    host = np.empty(count, dtype=np.uint32)
    if count:
        rc = _lib().cudaMemcpy(host.ctypes.data, dev_ptr, host.nbytes, 2)  # cudaMemcpyDeviceToHost
        assert rc == 0, f"cudaMemcpy failed with {rc}"
    return host
