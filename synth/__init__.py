"""Seeded synthetic inputs for the columnar-scan workloads.

This module is shared by the oracle side and the CUDA side and therefore holds
none of the scan's arithmetic: it only draws values and predicate bounds.
Packing, decoding, filtering and aggregation live in the oracle and in the
library, separately.

Recipes (the paper's own workloads are synthetic, §4):
  * uniform column: N i.i.d. values uniform in [base, base + 2^b);
  * clustered column: the uniform multiset sorted ascending, then a fraction
    p of positions displaced: every position is chosen independently with
    probability p and the chosen positions are randomly permuted among
    themselves (p = 1 is a full uniform shuffle, p = 0 stays sorted).  The
    multiset never changes, so COUNT and SUM are identical for every p;
  * predicate at target selectivity sigma: width w = max(1, round(sigma*2^b)),
    lo drawn uniformly from [0, 2^b - w], hi = lo + w (then shifted by base).
    The realised selectivity COUNT/N is always reported beside sigma.
Host-side draws use numpy's PCG64; device-side draws use torch's CUDA
generator, for sizes where host generation would dominate the run.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 0x5CA1AB1E


def seed_for(config_id: int, column_id: int = 0, salt: int = 0) -> int:
    """Deterministic 63-bit seed per (workload, column, purpose)."""
    return (SEED_BASE ^ (config_id << 40) ^ (column_id << 8) ^ salt) & ((1 << 63) - 1)


def _with_base(u: np.ndarray, base: int) -> np.ndarray:
    if not base:
        return u
    return (u.astype(np.uint64) + np.uint64(base)).astype(np.uint32)


def uniform_values(seed: int, n: int, b: int, base: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    u = rng.integers(0, 1 << b, size=n, dtype=np.uint32)   # 32-bit draws: 10x faster than 64-bit
    return _with_base(u, base)


def clustered_values(seed: int, n: int, b: int, p: float, base: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    u = np.sort(rng.integers(0, 1 << b, size=n, dtype=np.uint32))
    if p >= 1.0:
        u = u[rng.permutation(n)]
    elif p > 0.0:
        idx = np.flatnonzero(rng.random(n) < p)
        u[idx] = u[idx[rng.permutation(idx.size)]]
    return _with_base(u, base)


def pick_range(seed: int, b: int, sigma: float, base: int = 0) -> tuple[int, int]:
    """Half-open [lo, hi) on decoded values with target selectivity sigma."""
    d = 1 << b
    w = max(1, min(d, int(round(sigma * d))))
    rng = np.random.default_rng(seed)
    lo = int(rng.integers(0, d - w + 1))
    return base + lo, base + lo + w


def log_uniform(rng: np.random.Generator, lo: float, hi: float, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))


# ---------------------------------------------------------------- device-side
def _torch():
    import torch  # noqa: PLC0415 - optional, only for device generation

    return torch


def _to_u32_bits(t):
    """int64 tensor of values in [0, 2^32) -> int32 tensor with the same low 32 bits."""
    torch = _torch()
    return torch.where(t >= (1 << 31), t - (1 << 32), t).to(torch.int32)


def uniform_values_device(seed: int, n: int, b: int, base: int = 0, device="cuda"):
    """Like uniform_values, drawn on the GPU; returns an int32 tensor of uint32 bits."""
    torch = _torch()
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    u = torch.randint(0, 1 << b, (n,), generator=g, device=device, dtype=torch.int64)
    if base:
        u += base
    return _to_u32_bits(u)


def clustered_values_device(seed: int, n: int, b: int, p: float, base: int = 0, device="cuda"):
    torch = _torch()
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    u = torch.randint(0, 1 << b, (n,), generator=g, device=device, dtype=torch.int64)
    u, _ = torch.sort(u)
    if p >= 1.0:
        u = u[torch.randperm(n, generator=g, device=device)]
    elif p > 0.0:
        idx = torch.nonzero(torch.rand(n, generator=g, device=device) < p).squeeze(1)
        perm = torch.randperm(idx.numel(), generator=g, device=device)
        u[idx] = u[idx[perm]]
    if base:
        u += base
    return _to_u32_bits(u)


# ------------------------------------------------------------ many columns
def batch_spec(seed: int, ncols: int = 4096, total: int = 1 << 31, len_lo: int = 1 << 10,
               len_hi: int = 1 << 26):
    """Per-column (n, b, p, sigma) for the batched workload.

    Lengths are log-uniform in [len_lo, len_hi], then every length is scaled
    by total / sum (floor, at least 1) so the batch holds about `total`
    values while keeping the log-uniform shape; b is uniform in 1..32; half
    the columns are uniform (p = None), half sorted with a displaced fraction
    p drawn from {0, 0.01, 0.1}; sigma is log-uniform in [1e-4, 1].
    """
    rng = np.random.default_rng(seed)
    lens = log_uniform(rng, len_lo, len_hi, size=ncols)
    lens = np.maximum(1, np.floor(lens * (total / lens.sum()))).astype(np.int64)
    bs = rng.integers(1, 33, size=ncols)
    sorted_mask = rng.random(ncols) < 0.5
    ps = rng.choice([0.0, 0.01, 0.1], size=ncols)
    sig = log_uniform(rng, 1e-4, 1.0, size=ncols)
    out = []
    for i in range(ncols):
        out.append((int(lens[i]), int(bs[i]), float(ps[i]) if sorted_mask[i] else None, float(sig[i])))
    return out
