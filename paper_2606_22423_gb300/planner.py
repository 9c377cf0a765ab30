"""Planner pipeline around the C ABI: features -> labels -> training -> plans.

Labels come from the harness itself: every strategy is timed on training
columns as a one-entry batch (the execution path plans are made for; CUDA
events, median of several runs), and the label is log(milliseconds).  Features are computed on the GPU by
scan_batch_features; training runs on the GPU through scan_planner_train_step.
Planning a batch = features -> network -> argmin (scan_planner_choose), or
the law fallback (scan_batch_law_choose) when no trained network is given.
Whatever the plan, results are the same: only the speed changes.
"""
from __future__ import annotations

import math
import statistics

import numpy as np

from . import gbscan

STRATEGIES = gbscan.STRATEGY_ORDER


def _torch():
    import torch  # noqa: PLC0415

    return torch


def time_strategy(col, lo, hi, strategy, stream, reps=3):
    """Median CUDA-event time (ms) of the column scanned as a one-entry batch.

    The planner chooses strategies for batched execution, so its labels are
    measured on that path (same kernel, fused zone tests, one graph launch),
    not on single-column launches whose fixed per-launch costs differ by
    strategy."""
    torch = _torch()
    out = torch.zeros((1, 4), dtype=torch.int64, device="cuda")
    bt = gbscan.Batch([col], [strategy])
    bt.run([(lo, hi)], stream=stream, dev_out=out, host=False)  # records the graph
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bt.run([(lo, hi)], stream=stream, dev_out=out, host=False)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    bt.close()
    return statistics.median(ts)


def features(columns, preds, stream=None):
    """(ncols, 4) float32 features on the GPU, via a throwaway batch plan."""
    torch = _torch()
    bt = gbscan.Batch(columns)
    f = torch.zeros((len(columns), 4), dtype=torch.float32, device="cuda")
    bt.features(preds, f, stream)
    torch.cuda.synchronize()
    bt.close()
    return f


def collect(columns, preds, stream, reps=3):
    """Features (GPU tensor) and log-time labels (GPU tensor, ncols x 4).

    A label is the marginal device time of the strategy on the column: the
    one-entry batch's time minus the same batch with an empty predicate
    (which launches the same kernels and graph but reads no data), plus 1 us,
    in log milliseconds.  Without the subtraction the fixed per-graph cost
    hides the differences between strategies on all but the largest columns."""
    torch = _torch()
    X = features(columns, preds, stream)
    T = np.zeros((len(columns), len(STRATEGIES)), dtype=np.float32)
    for i, (c, (lo, hi)) in enumerate(zip(columns, preds)):
        base = time_strategy(c, 0, 0, "branchfree", stream, reps)
        for s, name in enumerate(STRATEGIES):
            t = time_strategy(c, lo, hi, name, stream, reps)
            T[i, s] = math.log(max(t - base, 0.0) + 1e-3)
    return X, torch.from_numpy(T).cuda()


def train(planner, X, T, steps=1500, lr=3e-3, stream=None):
    """Full-batch Adam on the GPU; returns the loss history (every 100 steps)."""
    hist = []
    rows = X.shape[0]
    for t in range(steps):
        want = (t % 100 == 0) or t == steps - 1
        loss = planner.train_step(X, T, rows, lr, stream, want_loss=want)
        if want:
            hist.append(loss)
    return hist


def choose(planner, X, stream=None, margin=0.0):
    """Strategy names per row of X from the network (argmin of predicted log time).
    With margin > 0: the first strategy, in STRATEGIES order, whose predicted log
    time is within `margin` of the row's minimum."""
    torch = _torch()
    out = torch.zeros(X.shape[0], dtype=torch.int32, device="cuda")
    planner.choose(X, X.shape[0], out, stream, margin=margin)
    torch.cuda.synchronize()
    return [STRATEGIES[i] for i in out.cpu().tolist()]


def choose_law(batch, X, beta_gbs, t_dec_gvals, stream=None):
    """Strategy names per column from the bandwidth law (fallback plan)."""
    torch = _torch()
    out = torch.zeros(X.shape[0], dtype=torch.int32, device="cuda")
    batch.law_choose(X, beta_gbs * 1e9, [t * 1e9 for t in t_dec_gvals], out, stream)
    torch.cuda.synchronize()
    return [STRATEGIES[i] for i in out.cpu().tolist()]


def training_columns(seed, count=160, n_lo=1 << 22, n_hi=1 << 27, stream=None):
    """Varied training columns: b, N, order and sigma spread over the planner's domain."""
    import synth

    torch = _torch()
    rng = np.random.default_rng(seed)
    cols, preds = [], []
    with torch.cuda.stream(stream) if stream is not None else _null():
        for i in range(count):
            b = int(rng.integers(1, 33))
            n = int(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))))
            p = [None, 0.0, 0.01, 0.1, 1.0][i % 5]
            s = synth.seed_for(5, i, seed)
            v = (synth.uniform_values_device(s, n, b) if p is None
                 else synth.clustered_values_device(s, n, b, p))
            c = gbscan.Column.from_device(v, n, b, stream=stream)
            c.zonemap_build(stream)
            cols.append(c)
            sigma = float(synth.log_uniform(rng, 1e-4, 1.0))
            preds.append(synth.pick_range(int(rng.integers(1 << 30)), b, sigma))
    torch.cuda.synchronize()
    return cols, preds


class _null:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False
