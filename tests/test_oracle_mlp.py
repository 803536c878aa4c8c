"""Pins of the FP64 MLP reference: the analytic gradient against central
finite differences, and the forward pass against an explicit per-sample loop."""
import numpy as np

from oracle import mlp_ref as M


def test_parameter_count():
    assert M.NPARAM == 64 * 10 + 64 + 64 * 64 + 64 + 4 * 64 + 4 == 5124


def test_forward_matches_per_sample_loop():
    rng = np.random.default_rng(2)
    p = M.init_params(3) + 0.01 * rng.normal(size=M.NPARAM)
    X = rng.normal(size=(7, M.NIN))
    y, _ = M.forward(p, X)
    d = M.unpack(p)
    silu = lambda z: z / (1.0 + np.exp(-z))
    for s in range(7):
        h1 = [silu(sum(d["W1"][i, k] * X[s, k] for k in range(10)) + d["b1"][i]) for i in range(64)]
        h2 = [silu(sum(d["W2"][i, k] * h1[k] for k in range(64)) + d["b2"][i]) for i in range(64)]
        out = [sum(d["W3"][o, k] * h2[k] for k in range(64)) + d["b3"][o] for o in range(4)]
        np.testing.assert_allclose(y[s], out, rtol=1e-12, atol=1e-14)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    p = M.init_params(1) + 0.05 * rng.normal(size=M.NPARAM)
    X = rng.normal(size=(64, M.NIN))
    Y = rng.normal(size=(64, M.NOUT))
    loss, g = M.loss_and_grad(p, X, Y)
    idx = rng.choice(M.NPARAM, 120, replace=False)
    idx = np.union1d(idx, [0, 639, 640, 703, 704, 4799, 4800, 4863, 4864, 5119, 5120, 5123])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (M.loss_and_grad(pp, X, Y)[0] - M.loss_and_grad(pm, X, Y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-8 + 1e-6 * abs(g[i]), (i, fd, g[i])
