"""Pins of the predictor oracle (oracle/mlp_oracle.py): rounding, loss, gradients, Adam."""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def test_bf16_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, 1.0 + 2.0 ** -7 + 2.0 ** -8, -2.5, 0.0],
                 dtype=np.float32)
    # 1 + 2^-8 is half-way between 1 and 1 + 2^-7: ties go to the even neighbour (1)
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -7, 1.0 + 2.0 ** -6, -2.5, 0.0], dtype=np.float32)
    np.testing.assert_array_equal(M.bf16(x), want)
    y = np.random.default_rng(0).normal(size=1000).astype(np.float32)
    r = M.bf16(y)
    assert np.all(np.abs(r - y) <= np.abs(y) * 2.0 ** -8)      # at most half an ulp of an 8-bit mantissa
    assert np.all((r.view(np.uint32) & 0xFFFF) == 0)


def test_loss_closed_form_with_constant_output():
    p = M.init_params(1).astype(np.float64)
    W1, b1, W2, b2, W3, b3 = M.unflatten(p)
    W3[:] = 0.0
    b3[:] = [0.3, -0.7]
    X = np.random.default_rng(2).normal(size=(5, M.F_IN))
    T = np.array([[0.1, 1.0], [0.5, 0.0], [0.2, 1.0], [0.9, 0.0], [0.0, 1.0]])
    o, _ = M.forward(p, X, rounding=False)
    np.testing.assert_allclose(o, np.tile([0.3, -0.7], (5, 1)), atol=1e-12)
    want = np.mean((0.3 - T[:, 0]) ** 2 + np.log1p(np.exp(-0.7)) + 0.7 * T[:, 1])
    assert abs(M.loss(o, T) - want) < 1e-12


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    p = M.init_params(4).astype(np.float64)
    X = rng.normal(size=(7, M.F_IN))
    T = np.column_stack([rng.uniform(size=7), (rng.uniform(size=7) > 0.5).astype(float)])
    L, g = M.backward(p, X, T, rounding=False)
    idx = rng.choice(p.size, size=60, replace=False)
    for i in idx:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (M.loss(M.forward(pp, X, rounding=False)[0], T) - M.loss(M.forward(pm, X, rounding=False)[0], T)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_gradient_of_each_layer_is_nonzero_and_shaped():
    rng = np.random.default_rng(5)
    p = M.init_params(6)
    X = rng.normal(size=(16, M.F_IN)).astype(np.float32)
    T = np.column_stack([rng.uniform(size=16), (rng.uniform(size=16) > 0.5).astype(float)])
    _, g = M.backward(p, X, T)
    assert g.shape == (M.n_params(),)
    for part in M.unflatten(g):
        assert np.any(part != 0.0)


def test_adam_first_step_moves_every_weight_by_lr():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    p1, m, v = M.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # bias-corrected first step: m_hat = g, v_hat = g^2, so the step is lr * sign(g) (up to eps)
    np.testing.assert_allclose(p - p1, 0.01 * np.sign(g), rtol=1e-4)


@pytest.mark.parametrize("steps", [300])
def test_training_fits_a_separable_toy_problem(steps):
    rng = np.random.default_rng(7)
    X = rng.normal(size=(256, M.F_IN))
    T = np.column_stack([0.5 + 0.1 * np.tanh(X[:, 0]), (X[:, 1] > 0).astype(float)])
    p = M.init_params(8).astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    L0, _ = M.backward(p, X, T, rounding=False)
    for t in range(1, steps + 1):
        L, g = M.backward(p, X, T, rounding=False)
        p, m, v = M.adam_step(p, g, m, v, t, lr=3e-3)
    assert L < 0.25 * L0
