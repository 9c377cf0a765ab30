"""Pins of the fp64 planner-network reference (oracle/mlp_ref.py)."""
import numpy as np
import pytest

from oracle import mlp_ref


def test_forward_on_a_hand_worked_network():
    # 2 -> 2 -> 2 -> 1 with hand-chosen weights; values worked out by hand:
    # x = (1, -2): z1 = (1*1 + -2*0, 1*-1 + -2*1) + (0.5, 0) = (1.5, -3) -> a1 = (1.5, 0)
    # z2 = (1.5*2 + 0*1, 1.5*-1 + 0*3) + (0, 1) = (3, -0.5) -> a2 = (3, 0)
    # y = 3*0.5 + 0*7 - 1 = 0.5
    params = [
        (np.array([[1.0, -1.0], [0.0, 1.0]]), np.array([0.5, 0.0])),
        (np.array([[2.0, -1.0], [1.0, 3.0]]), np.array([0.0, 1.0])),
        (np.array([[0.5], [7.0]]), np.array([-1.0])),
    ]
    y, _ = mlp_ref.forward(params, np.array([[1.0, -2.0]]))
    assert y.shape == (1, 1) and y[0, 0] == pytest.approx(0.5)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    params = mlp_ref.init(3)
    X = rng.normal(size=(16, 4))
    T = rng.normal(size=(16, 4))
    Y, cache = mlp_ref.forward(params, X)
    grads = mlp_ref.backward(params, cache, Y, T)
    flat = mlp_ref.flatten(params)
    gflat = mlp_ref.flatten(grads)
    h = 1e-6
    idx = rng.choice(flat.size, size=300, replace=False)
    for i in idx:
        up, dn = flat.copy(), flat.copy()
        up[i] += h
        dn[i] -= h
        lu = mlp_ref.loss(mlp_ref.forward(mlp_ref.unflatten(up), X)[0], T)
        ld = mlp_ref.loss(mlp_ref.forward(mlp_ref.unflatten(dn), X)[0], T)
        assert gflat[i] == pytest.approx((lu - ld) / (2 * h), rel=1e-4, abs=1e-8)


def test_adam_first_step_moves_each_parameter_by_lr_against_its_gradient():
    # with zero moments and bias correction, step 1 is -lr * g / (|g| + eps)
    params = [(np.array([[1.0, 2.0]]), np.array([0.0, -3.0]))]
    grads = [(np.array([[0.5, -4.0]]), np.array([1e-3, -2.0]))]
    m, v = mlp_ref.adam_state(params)
    newp, _, _ = mlp_ref.adam_step(params, grads, m, v, t=1, lr=0.01, eps=1e-8)
    for (W, b), (W0, b0), (gW, gb) in zip(newp, params, grads):
        np.testing.assert_allclose(W - W0, -0.01 * np.sign(gW), rtol=1e-4)
        np.testing.assert_allclose(b - b0, -0.01 * np.sign(gb), rtol=1e-4)


def test_adam_training_fits_a_noise_free_target():
    rng = np.random.default_rng(1)
    teacher = mlp_ref.init(11)
    X = rng.uniform(-1, 1, size=(256, 4))
    T, _ = mlp_ref.forward(teacher, X)
    params = mlp_ref.init(12)
    m, v = mlp_ref.adam_state(params)
    first = mlp_ref.loss(mlp_ref.forward(params, X)[0], T)
    for t in range(1, 401):
        Y, cache = mlp_ref.forward(params, X)
        params, m, v = mlp_ref.adam_step(params, mlp_ref.backward(params, cache, Y, T), m, v, t, lr=3e-3)
    last = mlp_ref.loss(mlp_ref.forward(params, X)[0], T)
    assert last < 0.05 * first


def test_flatten_layout_and_parameter_count():
    params = mlp_ref.init(0)
    flat = mlp_ref.flatten(params)
    assert flat.size == 4 * 64 + 64 + 64 * 64 + 64 + 64 * 4 + 4 == 4740
    back = mlp_ref.unflatten(flat)
    for (W, b), (W2, b2) in zip(params, back):
        np.testing.assert_array_equal(W, W2)
        np.testing.assert_array_equal(b, b2)
