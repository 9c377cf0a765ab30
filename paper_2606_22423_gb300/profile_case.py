"""Run one scan configuration a few times (for ncu captures and quick timing).

  python -m paper_2606_22423_gb300.profile_case --b 8 --n 268435456 \
      --sigma 0.1 --strategy branchfree --reps 3

Builds one device-resident column of n uniform values at width b (device-side
generation and encoding), then launches the scan `reps` times and prints the
CUDA-event time of the last launch.  Under ncu use -k regex:k_scan_full and
-s/-c to pick launches.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import torch

    import synth
    from paper_2606_22423_gb300 import gbscan

    ap = argparse.ArgumentParser()
    ap.add_argument("--b", type=int, default=16)
    ap.add_argument("--n", type=int, default=1 << 27)
    ap.add_argument("--sigma", type=float, default=0.1)
    ap.add_argument("--strategy", default="branchfree")
    ap.add_argument("--order", default="uniform", choices=["uniform", "sorted", "swapped"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--select", action="store_true",
                    help="run the materializing select (positions) instead of the counting scan")
    ap.add_argument("--batch", type=int, default=0,
                    help="scan a batch of this many mixed columns (batched workload recipe, scaled)")
    a = ap.parse_args()
    gbscan.load()
    if a.batch:
        return batch_case(a)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        seed = synth.seed_for(7, a.b)
        if a.order == "uniform":
            v = synth.uniform_values_device(seed, a.n, a.b)
        else:
            v = synth.clustered_values_device(seed, a.n, a.b, 0.0 if a.order == "sorted" else 0.01)
        col = gbscan.Column.from_device(v, a.n, a.b, stream=s)
        del v
    if a.strategy.startswith("zone"):
        col.zonemap_build(s)
    lo, hi = synth.pick_range(synth.seed_for(7, a.b, 1), a.b, a.sigma)
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    pos = torch.empty(a.n if a.select else 1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    ms = 0.0
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        if a.select:
            col.select_async(lo, hi, pos, out, a.strategy, stream=s)
        else:
            col.run_async(lo, hi, out, a.strategy, s)
        e1.record(s)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
    col.status(s)
    r = out.cpu().tolist()
    nbytes = gbscan.scan_packed_words(a.n, a.b) * 4 + (4 * r[0] if a.select else 0)
    print(json.dumps({"b": a.b, "n": a.n, "strategy": a.strategy, "order": a.order,
                      "op": "select" if a.select else "count", "ms": ms,
                      "gbs": nbytes / (ms * 1e-3) / 1e9, "count": r[0], "sum": r[1], "blocks": r[2]}))
    col.close()


def batch_case(a):
    """The batched workload recipe scaled to a.batch columns and a.n values in total."""
    import torch

    import synth
    from paper_2606_22423_gb300 import gbscan

    s = torch.cuda.Stream()
    spec = synth.batch_spec(synth.seed_for(4), ncols=a.batch, total=a.n)
    cols, preds = [], []
    with torch.cuda.stream(s):
        for i, (n, b, p, sigma) in enumerate(spec):
            v = (synth.uniform_values_device(synth.seed_for(4, i), n, b) if p is None
                 else synth.clustered_values_device(synth.seed_for(4, i), n, b, p))
            c = gbscan.Column.from_device(v, n, b, stream=s)
            c.zonemap_build(s)
            cols.append(c)
            preds.append(synth.pick_range(synth.seed_for(4, i, 1), b, sigma))
    torch.cuda.synchronize()
    bt = gbscan.Batch(cols, [a.strategy] * len(cols))
    parr = gbscan.Batch.pred_array(preds)
    out = torch.zeros((len(cols), 4), dtype=torch.int64, device="cuda")
    ms = 0.0
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        bt.run(parr, stream=s, dev_out=out, host=False)
        e1.record(s)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
    nbytes = sum(gbscan.scan_packed_words(x[0], x[1]) * 4 for x in spec)
    print(json.dumps({"batch": len(cols), "values": sum(x[0] for x in spec), "strategy": a.strategy, "ms": ms,
                      "gbs": nbytes / (ms * 1e-3) / 1e9}))
    bt.close()
    for c in cols:
        c.close()


if __name__ == "__main__":
    main()
