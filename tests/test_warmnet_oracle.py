"""Pins of the FP64 warm-start network oracle: its hand-derived gradients
against central finite differences of its own forward definition, and the
layer count / parameter count of the stated architecture."""
import numpy as np

from oracle import warmnet as WN


import pytest


def test_parameter_count_is_about_one_million():
    _, P = WN.layout(64)
    assert 1.0e6 <= P <= 1.1e6
    _, P4 = WN.layout(64, 4)  # with a dual block per neighbour direction
    assert P4 - P == 64 * 64 * 4 * 9 + 64 * 4


@pytest.mark.parametrize("n_dual", [0, 2])
def test_gradients_match_finite_differences(n_dual):
    rng = np.random.default_rng(0)
    Q, N, H, W = 3, 2, 8, 8
    lay, P = WN.layout(Q, n_dual)
    params = np.zeros(P)
    for w0, b0, ci, co in lay:
        params[w0:w0 + ci * co * 9] = rng.standard_normal(ci * co * 9) * np.sqrt(2.0 / (ci * 9))
        params[b0:b0 + co] = 0.05 * rng.standard_normal(co)
    # round weights to BF16 up front so finite differences see a smooth function of the biases
    for w0, b0, ci, co in lay:
        params[w0:w0 + ci * co * 9] = WN.bf16(params[w0:w0 + ci * co * 9])
    x = rng.random((N, Q + 1, H, W))
    t = rng.random((N, Q * (1 + n_dual), H, W))
    t[:, Q:] = rng.standard_normal((N, Q * n_dual, H, W))  # dual targets take either sign
    loss, g = WN.loss_grad(params, x, t, Q, n_dual=n_dual)
    out = WN.forward(params, x, Q, n_dual=n_dual)
    assert out.shape == t.shape and np.all(out[:, :Q] > 0) and (n_dual == 0 or np.any(out[:, Q:] < 0))
    assert np.isfinite(loss) and loss > 0
    # biases: exact FP64 perturbations (weights are BF16-rounded inside forward)
    for w0, b0, ci, co in lay:
        for k in rng.choice(co, size=min(3, co), replace=False):
            eps = 1e-6
            p1, p2 = params.copy(), params.copy()
            p1[b0 + k] += eps
            p2[b0 + k] -= eps
            fd = (WN.loss_grad(p1, x, t, Q, n_dual=n_dual)[0] - WN.loss_grad(p2, x, t, Q, n_dual=n_dual)[0]) / (2 * eps)
            assert abs(fd - g[b0 + k]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-10, (b0, k, fd, g[b0 + k])
    # weights: the gradient is with respect to the rounded weights the forward
    # pass uses; with rounding switched off (the weights already hold BF16
    # values) the loss is smooth in them and central differences apply
    g0 = WN.loss_grad(params, x, t, Q, round_weights=False, n_dual=n_dual)[1]
    assert np.array_equal(g0, g)
    for w0, b0, ci, co in lay:
        for k in rng.choice(ci * co * 9, size=3, replace=False):
            eps = 1e-6
            p1, p2 = params.copy(), params.copy()
            p1[w0 + k] += eps
            p2[w0 + k] -= eps
            fd = (WN.loss_grad(p1, x, t, Q, False, n_dual)[0] - WN.loss_grad(p2, x, t, Q, False, n_dual)[0]) / (2 * eps)
            assert abs(fd - g[w0 + k]) <= 1e-5 * max(abs(fd), 1e-3) + 1e-10, (w0, k, fd, g[w0 + k])
