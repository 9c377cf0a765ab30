"""Host-side helpers of the planner and the bench, on CPU: the per-strategy
calibration of the law's log times, the calibrated prior, and the oracle
timing loop that the bench's CPU baseline reports."""
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
