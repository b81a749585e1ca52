"""Pins for the numpy fp64 reference of the predictor MLP (no GPU): analytic
backpropagation against central finite differences, closed forms of special
networks, and the first Adam step."""
import numpy as np

from oracle import mlp


def _data(seed, B=17):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.3, mlp.NPARAMS)
    X = rng.normal(0, 1, (B, 8))
    T = rng.normal(0, 1, (B, 2))
    return theta, X, T


def test_parameter_count_and_layout():
    assert mlp.NPARAMS == 4866
    theta = np.arange(mlp.NPARAMS, dtype=float)
    p = mlp.unpack(theta)
    assert p["W1"].shape == (64, 8) and p["W1"][0, 1] == 1
    assert p["b3"].tolist() == [4864, 4865]


def test_gradient_matches_finite_differences():
    theta, X, T = _data(1)
    g = mlp.grad(theta, X, T)
    rng = np.random.default_rng(2)
    idx = sorted(set(rng.integers(0, mlp.NPARAMS, 60).tolist()) | {0, 511, 512, 4865, 4800})
    num = mlp.numgrad(theta, X, T, idx)
    assert np.allclose(g[idx], num, rtol=1e-5, atol=1e-8)


def test_closed_forms():
    # all weights zero: y = b3 for every sample, dL/db3 = mean(y - t)
    theta = np.zeros(mlp.NPARAMS)
    theta[-2:] = [0.5, -1.0]
    X = np.random.default_rng(3).normal(size=(5, 8))
    T = np.zeros((5, 2))
    y, _ = mlp.forward(theta, X)
    assert np.allclose(y, [[0.5, -1.0]] * 5)
    g = mlp.grad(theta, X, T)
    assert np.allclose(g[-2:], [0.5, -1.0])
    assert np.allclose(g[:-2], 0.0)  # ReLU of zero pre-activations passes nothing back
    assert np.isclose(mlp.loss(theta, X, T), (0.25 + 1.0) * 5 / 10)


def test_first_adam_step_is_a_signed_step():
    theta = np.ones(10)
    g = np.array([1.0, -2.0, 0.5, 0, 3, -1, 1, 1, 1, 1])
    with np.errstate(invalid="ignore"):  # the zero gradient's 0/0 is excluded below
        th, m, v = mlp.adam_step(theta, g, np.zeros(10), np.zeros(10), 1, lr=0.01, eps=0.0)
    want = 1.0 - 0.01 * np.sign(g)
    want[3] = 1.0  # 0/0 would be nan with eps=0: check the others
    mask = g != 0
    assert np.allclose(th[mask], want[mask])
