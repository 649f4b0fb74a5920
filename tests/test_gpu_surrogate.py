"""The surrogate network's CUDA kernels against the FP64 reference
(oracle/mlp.py) on identical BF16-rounded weights."""
import numpy as np
import pytest

from oracle import mlp
from paper_2504_09024_gb300 import lbm

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def sample(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1.0, 1.0, size=(n, 5))
    yD = rng.uniform(0.0, 0.4, n)
    yB = (rng.uniform(size=n) < 0.4).astype(float)
    return X, yD, yB


@pytest.fixture(scope="module")
def net():
    s = lbm.Surrogate(seed=1)
    yield s
    s.close()


def with_biases(seed):
    params = mlp.init_params(seed=seed)
    rng = np.random.default_rng(seed + 100)
    for W, b in params:
        b += rng.normal(scale=0.1, size=b.shape).astype(np.float32).astype(np.float64)
    return params


def test_parameter_layout(net):
    assert net.count == 50562
    params = with_biases(3)
    net.set_params(params)
    back = net.get_params()
    for (W, b), (W2, b2) in zip(params, back):
        np.testing.assert_array_equal(W.astype(np.float32), W2)
        np.testing.assert_array_equal(b.astype(np.float32), b2)


@pytest.mark.parametrize("n", [1, 37, 1000])
def test_forward_matches_reference(net, n):
    params = with_biases(4)
    net.set_params(params)
    X, _, _ = sample(n, 5)
    D, z = net.predict(X)
    ref, _ = mlp.forward(params, X.astype(np.float32).astype(np.float64))
    assert rel(D, ref[:, 0]) <= 1e-5
    assert rel(z, ref[:, 1]) <= 1e-5


@pytest.mark.parametrize("n", [7, 300, 2000])
def test_gradients_match_reference(net, n):
    """Bound: relative L2 error <= 1e-2 per tensor (the reference is pinned
    to central finite differences at 1e-6 in the CPU tests)."""
    params = with_biases(6)
    net.set_params(params)
    X, yD, yB = sample(n, 7)
    X = X.astype(np.float32).astype(np.float64)
    yD = yD.astype(np.float32).astype(np.float64)
    out, cache = mlp.forward(params, X)
    ref = mlp.backward(params, cache, out, yD, yB)
    got, loss = net.grad(X, yD, yB)
    assert abs(loss - mlp.loss(out, yD, yB)) <= 1e-5 * abs(mlp.loss(out, yD, yB))
    worst = 0.0
    for (gW, gb), (rW, rb) in zip(got, ref):
        worst = max(worst, rel(gW, rW), rel(gb, rb))
    assert worst <= 1e-2, worst
    assert worst <= 1e-4, worst   # what FP32 accumulation actually reaches


def test_adam_steps_match_reference(net):
    params = with_biases(8)
    net.set_params(params)
    X, yD, yB = sample(256, 9)
    X = X.astype(np.float32).astype(np.float64)
    yD = yD.astype(np.float32).astype(np.float64)
    state = []
    ref = [[W.copy(), b.copy()] for W, b in params]
    for t in range(1, 4):
        out, cache = mlp.forward(ref, X)
        grads = mlp.backward(ref, cache, out, yD, yB)
        mlp.adam_step(ref, grads, state, lr=1e-3, t=t)
    net.train(X, yD, yB, epochs=3, lr=1e-3)
    got = net.get_params()
    for (W, b), (W0, b0), (rW, rb) in zip(got, params, ref):
        # Adam moves every weight by up to lr per step: compare the updates
        assert rel(W - W0, rW - W0) <= 1e-3
        assert np.abs(b - rb).max() <= 1e-6


def test_training_fits_a_smooth_target(net):
    rng = np.random.default_rng(11)
    X = rng.uniform(-1, 1, size=(1024, 5))
    yD = 0.1 * (X[:, 0] + 1) * (1 + 0.5 * X[:, 1])
    yB = (X[:, 0] + 0.3 * X[:, 2] > 0.4).astype(float)
    net.set_params(mlp.init_params(seed=12))
    _, l0 = net.grad(X, yD, yB)
    l1 = net.train(X, yD, yB, epochs=400, lr=2e-3)
    assert l1 < 0.2 * l0, (l0, l1)
