"""gbscan: the fused columnar scan (decode -> range filter -> exact COUNT/SUM)
of "When Is a Columnar Scan Bandwidth-Bound?" as hand-written sm_103a CUDA
behind a C ABI (include/gbscan.h).  Python here is a thin ctypes binding."""
from . import gbscan  # noqa: F401

__all__ = ["gbscan"]
