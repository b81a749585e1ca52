"""The predictor's CUDA kernels (forward, backward, Adam) against the numpy
fp64 reference, and what the trained network gains over the analytic bound
on the method's own measured timings."""
import numpy as np
import pytest

from helpers import ensure_lib
from oracle import mlp
from paper_2010_12117_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _case(seed, B):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.25, mlp.NPARAMS).astype(np.float32)
    X = rng.normal(0, 1, (B, 8)).astype(np.float32)
    T = rng.normal(0, 1, (B, 2)).astype(np.float32)
    return theta, X, T


@pytest.mark.parametrize("B", [1, 7, 128, 1000])
def test_forward_matches_reference(B):
    from paper_2010_12117_gb300 import binding
    theta, X, T = _case(B, B)
    y = torch.empty(B, 2, device="cuda")
    binding.mlp_forward(_dev(theta), _dev(X), y)
    want, _ = mlp.forward(theta.astype(np.float64), X.astype(np.float64))
    assert np.allclose(y.cpu().numpy(), want, rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("B", [1, 33, 512])
def test_backward_matches_reference_gradients(B):
    from paper_2010_12117_gb300 import binding
    theta, X, T = _case(100 + B, B)
    p, x, t = _dev(theta), _dev(X), _dev(T)
    y = torch.empty(B, 2, device="cuda")
    act = torch.empty(B, 128, device="cuda")
    delta = torch.empty(B, 130, device="cuda")
    g = torch.empty(binding.MLP_PARAMS, device="cuda")
    loss = torch.empty(1, device="cuda")
    binding.mlp_forward(p, x, y, act)
    binding.mlp_backward(p, x, t, y, act, delta, g, loss)
    th64, X64, T64 = theta.astype(np.float64), X.astype(np.float64), T.astype(np.float64)
    want = mlp.grad(th64, X64, T64)
    got = g.cpu().numpy().astype(np.float64)
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-3 * scale
    # relative error per parameter where the gradient is not tiny
    big = np.abs(want) > 1e-3 * scale
    assert np.all(np.abs(got[big] - want[big]) <= 1e-3 * np.abs(want[big]) + 1e-6 * scale)
    assert np.isclose(loss.item(), mlp.loss(th64, X64, T64), rtol=1e-5)
    # finite differences on a sample of parameters
    idx = np.random.default_rng(B).integers(0, mlp.NPARAMS, 24)
    num = mlp.numgrad(th64, X64, T64, idx, h=1e-5)
    assert np.allclose(got[idx], num, rtol=1e-3, atol=1e-4 * scale)
    # deterministic: a second backward gives identical bits
    g2 = torch.empty_like(g)
    binding.mlp_backward(p, x, t, y, act, delta, g2, None)
    assert torch.equal(g, g2)


def test_adam_matches_reference():
    from paper_2010_12117_gb300 import binding
    rng = np.random.default_rng(5)
    theta = rng.normal(0, 1, mlp.NPARAMS).astype(np.float32)
    p = _dev(theta)
    m = torch.zeros(mlp.NPARAMS, device="cuda")
    v = torch.zeros(mlp.NPARAMS, device="cuda")
    th, m64, v64 = theta.astype(np.float64), np.zeros(mlp.NPARAMS), np.zeros(mlp.NPARAMS)
    for step in range(1, 4):
        g = rng.normal(0, 1, mlp.NPARAMS).astype(np.float32)
        binding.mlp_adam(p, _dev(g), m, v, step, 1e-2, weight_decay=1e-3)
        th, m64, v64 = mlp.adam_step(th, g.astype(np.float64), m64, v64, step, 1e-2, wd=1e-3)
    assert np.allclose(p.cpu().numpy(), th, rtol=1e-5, atol=1e-6)


def test_training_fits_a_smooth_function():
    from paper_2010_12117_gb300.predictor import Predictor
    rng = np.random.default_rng(8)
    X = rng.uniform(0, 1, (256, 8)).astype(np.float32)
    secs = np.exp(2 * X[:, 0] + X[:, 1] ** 2 - 3)
    mem = np.exp(5 + 3 * X[:, 2] * X[:, 3])
    Y = np.stack([secs, mem], 1)
    bounds = np.ones_like(Y)  # the network learns log(Y / bound) = log Y here
    pr = Predictor(seed=1)
    hist = pr.fit(X, Y, bounds, steps=1500, lr=3e-3, weight_decay=0.0)
    assert hist[-1] < 0.05 * hist[0]
    err = np.abs(np.log(pr.raw(X, bounds) / Y))
    assert np.median(err) < 0.1


def test_trained_network_beats_the_analytic_bound_on_measured_jobs():
    """Timings and footprints the method generates (each time the mean of 5
    runs): train on 64 jobs of the batched distribution, judge on 32 others."""
    from paper_2010_12117_gb300.predictor import Predictor, shape_of
    from paper_2010_12117_gb300.serve import calibrate
    mats = synth.batched(11, 96)
    X, Y, Bd = calibrate(mats, reps=5)
    pr = Predictor(seed=0)
    pr.fit(X[:64], Y[:64], Bd[:64], steps=2000)
    test = slice(64, 96)
    pred = pr.predict([shape_of(m) for m in mats[64:]])
    calibrated = Bd[test] * pr.ratio
    e_mlp = np.median(np.abs(np.log(pred / Y[test])), axis=0)
    e_ana = np.median(np.abs(np.log(calibrated / Y[test])), axis=0)
    e_raw = np.median(np.abs(np.log(Bd[test] / Y[test])), axis=0)
    print("median |log error| time/mem: mlp", e_mlp, "calibrated bound", e_ana, "bound", e_raw)
    assert np.all(e_mlp < e_ana)
    assert np.all(e_mlp < e_raw)
    # the analytic bound judges the network: no prediction falls below it
    assert np.all(pred >= Bd[test] * (1 - 1e-9))


@pytest.mark.parametrize("mode", [0, 1])
def test_analytic_memory_is_the_layout_of_the_library(mode):
    """The analytic bytes of a mode equal the words the library lays out for
    a one-job batch in that mode (coefficients, partial, determinant values,
    residues, limbs, workspace)."""
    from paper_2010_12117_gb300.binding import Batch
    from paper_2010_12117_gb300.predictor import analytic, analytic_mode, shape_of
    from paper_2010_12117_gb300.runner import variable_order
    rng = np.random.default_rng(5)
    for n, degs in [(6, (2, 1, 2)), (14, (2, 2)), (20, (1, 3, 1)), (16, (4,))]:
        pm = synth.random_matrix(rng, n, degs, 0.5, -99, 99)
        s = shape_of(pm)
        b = Batch([(n, tuple(degs[v] for v in variable_order(n, degs)), s.P)])  # as the runner plans it
        b.set_mode(n, mode)
        words = sum(b.words.values())
        b.close()
        assert analytic_mode(s, mode)[1] == 4.0 * words, (n, degs)
        assert analytic(s)[1] <= 4.0 * words
