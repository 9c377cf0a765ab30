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


def choose(planner, X, stream=None, margin=0.0, prior=None):
    """Strategy names per row of X from the network (argmin of predicted log time).
    With margin > 0: the first strategy, in STRATEGIES order, whose predicted log
    time is within `margin` of the row's minimum.  With a prior (rows x 4 log
    times on the GPU, e.g. law_log_times): the prediction is network + prior."""
    torch = _torch()
    out = torch.zeros(X.shape[0], dtype=torch.int32, device="cuda")
    planner.choose(X, X.shape[0], out, stream, margin=margin, dev_prior=prior)
    torch.cuda.synchronize()
    return [STRATEGIES[i] for i in out.cpu().tolist()]


def feature_box(X_train):
    """Per-feature bounds (lo[4] + hi[4]) of the training features."""
    lo = X_train.min(dim=0).values.cpu().tolist()
    hi = X_train.max(dim=0).values.cpu().tolist()
    return lo + hi


def choose_guarded(planner, X, law_plan, law_log_ms, margin, stream=None, box=None):
    """The law's plan, except for columns inside the training features' box
    where the network predicts another available strategy faster by more than
    `margin` (its own RMS error): the law is the fallback and the judge, the
    network refines it where it is sure and on familiar ground."""
    torch = _torch()
    rows = X.shape[0]
    fb = torch.tensor([STRATEGIES.index(s) for s in law_plan], dtype=torch.int32, device="cuda")
    out = torch.zeros(rows, dtype=torch.int32, device="cuda")
    # only the law's (branch-free) flavour is open to the network: in a batch a
    # column moved to the branchy flavour adds a width-group kernel to the
    # replay, a fixed cost the one-entry-batch labels never see (and branchy
    # never beats branch-free for counts on this GPU)
    avail = law_log_ms.clone()
    avail[:, [STRATEGIES.index("branchy"), STRATEGIES.index("zone_br")]] = 30.0
    planner.choose_guarded(X, rows, margin, fb, avail, out, stream, feature_box=box)
    torch.cuda.synchronize()
    return [STRATEGIES[i] for i in out.cpu().tolist()]


def law_log_times(columns, X, beta_gbs, t_dec_gvals, stream=None):
    """The bandwidth law's predicted log milliseconds per (column, strategy), on the GPU."""
    torch = _torch()
    bt = gbscan.Batch(columns)
    out = torch.zeros((len(columns), len(STRATEGIES)), dtype=torch.float32, device="cuda")
    bt.law_times(X, beta_gbs * 1e9, [t * 1e9 for t in t_dec_gvals], out, stream)
    torch.cuda.synchronize()
    bt.close()
    return out


def choose_law(batch, X, beta_gbs, t_dec_gvals, stream=None):
    """Strategy names per column from the bandwidth law (fallback plan)."""
    torch = _torch()
    out = torch.zeros(X.shape[0], dtype=torch.int32, device="cuda")
    batch.law_choose(X, beta_gbs * 1e9, [t * 1e9 for t in t_dec_gvals], out, stream)
    torch.cuda.synchronize()
    return [STRATEGIES[i] for i in out.cpu().tolist()]


def calibrate_law(L, T):
    """Per strategy, the least-squares affine map a_s + b_s * L_s from the law's log
    times L to the measured log-time labels T (both rows x S, on the GPU): the law's
    shape with its scale and fixed costs fitted to this machine.  Returns (a, b)."""
    torch = _torch()
    a = torch.zeros(L.shape[1], dtype=torch.float32, device=L.device)
    b = torch.ones(L.shape[1], dtype=torch.float32, device=L.device)
    for s in range(L.shape[1]):
        x, y = L[:, s].double(), T[:, s].double()
        keep = x < 29.0                      # strategies the law marks unavailable stay out
        if int(keep.sum()) < 2:
            continue
        x, y = x[keep], y[keep]
        vx = float(((x - x.mean()) ** 2).sum())
        bs = float(((x - x.mean()) * (y - y.mean())).sum()) / vx if vx > 0 else 0.0
        b[s] = bs
        a[s] = float(y.mean() - bs * x.mean())
    return a, b


def law_prior(L, calib):
    """Calibrated law log times a_s + b_s * L_s (rows x S): the prior the network corrects."""
    a, b = calib
    return (a[None, :] + b[None, :] * L).contiguous()


def choose_prior_only(prior, stream=None):
    """The plan of the prior alone (argmin per row, first on ties): the choice of a
    correction network that predicts no correction, run through the same kernel."""
    torch = _torch()
    rows = prior.shape[0]
    pl = gbscan.Planner(prior.shape[1], seed=1)
    pl.set_params(np.zeros(pl.nparams, dtype=np.float32))
    X = torch.zeros((rows, 4), dtype=torch.float32, device=prior.device)
    plan = choose(pl, X, stream, margin=0.0, prior=prior)
    pl.close()
    return plan


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
