"""Host-side helpers of the planner and the bench, on CPU: the per-strategy
calibration of the law's log times, the calibrated prior, and the oracle
timing loop that the bench's CPU baseline reports."""
import os
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_calibrate_law_recovers_an_affine_map_per_strategy():
    from paper_2606_22423_gb300 import planner as plmod

    rng = np.random.default_rng(5)
    L = torch.from_numpy(rng.uniform(-6.0, 2.0, size=(200, 4)).astype(np.float32))
    a_true = np.array([0.5, 1.0, -0.3, 0.2], dtype=np.float64)
    b_true = np.array([0.8, 1.1, 0.4, 0.6], dtype=np.float64)
    T = torch.from_numpy((a_true + b_true * L.double().numpy()
                          + rng.normal(0, 1e-3, size=(200, 4))).astype(np.float32))
    L[:50, 2:] = 30.0             # no zone map: the law marks the zone strategies unavailable
    a, b = plmod.calibrate_law(L, T)
    np.testing.assert_allclose(a.numpy(), a_true, atol=5e-3)
    np.testing.assert_allclose(b.numpy(), b_true, atol=2e-3)
    P = plmod.law_prior(L, (a, b))
    np.testing.assert_allclose(P.numpy(), a.numpy() + b.numpy() * L.numpy(), rtol=1e-6, atol=1e-6)
    # a strategy with fewer than two usable rows keeps the identity map
    L2 = L.clone()
    L2[:, 3] = 30.0
    a2, b2 = plmod.calibrate_law(L2, T)
    assert float(a2[3]) == 0.0 and float(b2[3]) == 1.0


def test_cpu_sample_covers_the_sweep_order_and_reports_per_width_rates():
    import bench
    import oracle
    import synth

    oracle.build()
    cols = []
    for b in (1, 9, 32):
        v = synth.uniform_values(synth.seed_for(2, b), 1 << 14, b)
        cols.append((b, oracle.pack(v, b)))
    gbs, vps, scans, used, per_b = bench.cpu_sample(cols, 1, budget_s=0.0, passes_max=1)
    assert scans == len(bench.SIGMAS) * len(cols)          # one pass: every sigma, every column
    assert gbs > 0 and vps > 0 and used > 0
    assert sorted(per_b) == [1, 9, 32] and all(r > 0 for r in per_b.values())
    _, _, scans2, _, _ = bench.cpu_sample(cols, 2, budget_s=1e9, passes_max=2)
    assert scans2 == 2 * scans                              # the pass cap bounds the sample
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()


def test_headline_line_stays_small_with_every_section_present():
    """The printed bench line must stay a few KB (a consumer that keeps only the
    tail of stdout must still see one whole line); the sections go to a file."""
    import argparse
    import json

    import bench

    W, S = bench.WIDTHS, bench.SIGMAS
    per_b = {str(b): {st: {"f": 0.91234, "gbs": 6000.1} for st in bench.STRATS} for b in W}
    law = {st: {"t_dec_gvals": 4.0, "b_star": 14.2, "median_abs_err": 0.05, "rms_err": 0.1} for st in bench.STRATS}
    roof = {"kernel": "k", "bound": "hbm", "achieved": 6300.0, "peak": 6702.8, "unit": "GB/s", "frac": 0.94,
            "peak_source": "measured", "frac_of_beta_read": 0.9, "achieved_branchfree": 6500.0,
            "achieved_branchy": 6100.0, "time_share_of_step": {"branchfree": 0.45}, "traffic": 808977152,
            "traffic_ratio": 1.0046, "traffic_source": "x" * 150}
    e2e = {"value": 2100.0, "unit": "GB/s", "h2d_bytes_per_step": 17716740096, "d2h_bytes_per_step": 12288,
           "h2d_gbs_raw": 211.0, "path": "y" * 250, "per_scan_roundtrip_gbs": 190.0,
           "per_scan_roundtrip_path": "z" * 120}
    cpu = {"value": 12.4, "unit": "GB/s", "cores": 16, "kind": "oracle", "sample": "s" * 180,
           "cpu_model": "Arm Neoverse V2", "values_per_s": 6.0e9, "single_thread": {"gbs": 0.84}}
    sections = {
        "plain": {"ms_l2_flushed": 0.0105, "gbs_l2_flushed": 1600.0, "ms_l2_warm": 0.0082},
        "probes": {"triad": {"gbs": 6700.0}, "decode_resident": {
            "t_dec_median_below_ridge_gvals": 5.0,
            "l2_control": {"case": "c" * 100, "l2_gbs": 9500.0, "l2_gbs_median_b20_32": 8100.0,
                           "beta_read_gbs": 7100.0, "above_beta_read": True}}},
        "zone": {"rows": [{"p": p, "sigma": s, "speedup": 12.5, "speedup_zone_agg": 13.1, "speedup_auto": 12.4, "exact": True}
                          for p in (0.0, 0.01, 0.1, 1.0) for s in (1e-4, 1e-3, 1e-2, 0.1, 0.5)]},
        "select": {"by_b": {"32": {"best_frac_branchfree": 0.95}, "16": {"best_frac_branchfree": 0.79}},
                   "exact": True},
        "layouts": {"per_layout": {k: {"t_dec_gvals": 3.5} for k in ("lanes", "rowmajor", "bytes")}},
        "conj": {"rows": [{"frac_conj": 0.77} for _ in range(4)]},
        "tune": {"sweep_gain": 1.097},
        "batched": {"ms_per_column_graph": 23.7, "plans": {
            k: {"ms": 0.97, "speedup_vs_per_column_graph": 24.4, "exact": True, "frac_of_law": 0.712}
            for k in ("branchfree", "law", "planned_mlp", "law_calibrated", "planned_mlp_law_prior")},
            "planner_vs_law": {"min": 0.99, "median": 1.01, "max": 1.03}},
        "serving": {"serial": {"qps": 3200.0}, "loads": [
            {"load": f, "achieved_qps": 800.0, "p50_us": 220.0, "p99_us": 600.0, "exact_vs_alone": True}
            for f in (0.25, 0.5, 0.9, 1.5)]},
    }
    args = argparse.Namespace(steps=20, warmup=5, detail=os.path.join(bench.ROOT, "bench_detail.json"))
    clocks = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 100}
    line = bench.headline(args, 1, 5080.0, 838.0, 384, per_b, roof, law, e2e, cpu, sections, 7100.0, clocks)
    text = json.dumps(line)
    assert len(text) <= bench.HEADLINE_MAX, len(text)
    assert "summary" in line                            # it fits with every section present
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "cpu_baseline",
                "gpu_launches", "clocks"):
        assert key in line
    assert line["roofline"]["frac"] == 0.94 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["summary"]["neg_ctrl_iii"] is True and line["summary"]["tune_gain"] > 1
    assert line["gpu_launches"] == 384 * 20


def test_batch_law_bounds_on_a_hand_computed_plan():
    """The batch plan's two law bounds from the blocks each column read, against values worked
    out by hand (beta 2 GB/s; T_dec 2 G values/s branch-free, 1 G branchy)."""
    import bench

    spec = [(4096, 4, None, 0.1), (2048, 4, None, 0.1), (3000, 32, None, 0.1), (1024, 8, None, 0.1)]
    strategies = ["branchfree", "zone_bf", "branchfree", "branchy"]
    blocks = [4, 1, 3, 1]                  # the zone skip read 1 of its 2 blocks
    summed, mixed = bench.batch_law_bounds(spec, strategies, blocks, 2.0, [2.0, 1.0])
    # (bf, 4): 2560 B, 5120 values -> max(1.28, 2.56) us; (bf, 32): 12288 B, 3000 values (the
    # tail block holds 952) -> max(6.144, 1.5) us; (branchy, 8): 1024 B, 1024 values -> 1.024 us
    assert summed == pytest.approx((2.56 + 6.144 + 1.024) * 1e-3, rel=1e-12)
    # all bytes 15872 / 2e9 = 7.936 us against decode 8120 / 2e9 + 1024 / 1e9 = 5.084 us
    assert mixed == pytest.approx(7.936e-3, rel=1e-12)
    assert mixed <= summed
