"""Pins of the FP64 surrogate-network reference (oracle/mlp.py)."""
import numpy as np
import pytest

from oracle import mlp


def test_bf16_round_matches_library_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=1000) * 10.0 ** rng.integers(-6, 6, 1000),
                        [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 65504.0, 1e-40]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(x), ref)
    # ties round to even: 1 + 2^-8 sits halfway between 1 and 1 + 2^-7
    assert mlp.bf16_round(1.0 + 2 ** -8) == 1.0
    assert mlp.bf16_round(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6


def test_loss_closed_forms():
    out = np.array([[0.5, 0.0], [0.25, 0.0]])
    # BCE at a zero logit is log 2 for either label; MSE of (0.5 - 0.1, 0.25 - 0.25)
    val = mlp.loss(out, np.array([0.1, 0.25]), np.array([1.0, 0.0]))
    assert abs(val - (0.4 ** 2 / 2 + np.log(2.0))) < 1e-15
    big = np.array([[0.0, 40.0]])
    assert mlp.loss(big, np.zeros(1), np.ones(1)) < 1e-16


def test_silu_derivative():
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.silu_grad(z), fd, rtol=0, atol=1e-9)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    widths = (5, 16, 16, 16, 16, 2)
    params = mlp.init_params(seed=1, widths=widths)
    for W, b in params:
        b += rng.normal(scale=0.1, size=b.shape)
    X = rng.normal(size=(7, 5))
    yD = rng.uniform(0, 0.3, 7)
    yB = (rng.uniform(size=7) < 0.5).astype(float)

    def L(ps):
        out, _ = mlp.forward(ps, X, round_weights=False)
        return mlp.loss(out, yD, yB)

    out, cache = mlp.forward(params, X, round_weights=False)
    grads = mlp.backward(params, cache, out, yD, yB, round_weights=False)
    h = 1e-6
    for k, (W, b) in enumerate(params):
        for P, G in ((W, grads[k][0]), (b, grads[k][1])):
            for _ in range(6):
                idx = tuple(rng.integers(s) for s in P.shape)
                old = P[idx]
                P[idx] = old + h
                lp = L(params)
                P[idx] = old - h
                lm = L(params)
                P[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(G[idx] - fd) <= 1e-6 * max(1.0, abs(fd)), (k, idx, G[idx], fd)


def test_adam_first_step_moves_by_lr():
    """With bias correction the first Adam step is lr * g / (|g| + eps)."""
    params = [[np.array([[1.0, -2.0]]), np.array([0.5])]]
    grads = [[np.array([[0.3, -0.02]]), np.array([1e-3])]]
    before = [p.copy() for p in params[0]]
    mlp.adam_step(params, grads, [], lr=0.01, t=1)
    for P, P0, G in zip(params[0], before, grads[0]):
        np.testing.assert_allclose(P0 - P, 0.01 * G / (np.abs(G) + 1e-8), rtol=1e-12)


def test_training_reduces_loss_on_a_smooth_target():
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, size=(256, 5))
    yD = 0.1 * (X[:, 0] + 1) * (1 + 0.5 * X[:, 1])
    yB = (X[:, 0] + 0.3 * X[:, 2] > 0.4).astype(float)
    params = mlp.init_params(seed=2, widths=(5, 32, 32, 32, 32, 2))
    state = []
    out, _ = mlp.forward(params, X)
    l0 = mlp.loss(out, yD, yB)
    for t in range(1, 301):
        out, cache = mlp.forward(params, X)
        grads = mlp.backward(params, cache, out, yD, yB)
        mlp.adam_step(params, grads, state, lr=3e-3, t=t)
    out, _ = mlp.forward(params, X)
    assert mlp.loss(out, yD, yB) < 0.25 * l0
