"""The warm-start network's CUDA kernels against the FP64 NumPy oracle:
forward output, loss and every parameter's gradient, and one Adam step."""
import numpy as np
import pytest

from oracle import warmnet as WN
from paper_1601_08201_gb300 import wsnet

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def setup(Q=3, N=2, H=8, W=12, seed=0, n_dual=0):
    rng = np.random.default_rng(seed)
    net = wsnet.WarmNet(H, W, Q, max_batch=N, seed=1, n_dual=n_dual)
    lay, P = WN.layout(Q, n_dual)
    assert net.num_params == P
    params = net.get_params().astype(np.float64)
    for w0, b0, ci, co in lay:
        params[b0:b0 + co] = 0.05 * rng.standard_normal(co)
    params = params.astype(np.float32)
    net.set_params(params)
    x = rng.random((N, Q + 1, H, W)).astype(np.float32)
    t = rng.random((N, Q * (1 + n_dual), H, W)).astype(np.float32)
    t[:, Q:] -= 0.5  # dual targets take either sign
    return net, params, x, t, Q, N, lay


@pytest.mark.parametrize("n_dual", [0, 2])
def test_forward_loss_and_gradients_match_oracle(n_dual):
    net, params, x, t, Q, N, lay = setup(n_dual=n_dual)
    assert net.num_outputs == Q * (1 + n_dual)
    xd = torch.from_numpy(x).cuda()
    td = torch.from_numpy(t).cuda()
    out = torch.empty_like(td)
    net.forward(xd.data_ptr(), N, out.data_ptr())
    torch.cuda.synchronize()
    ref = WN.forward(params.astype(np.float64), x.astype(np.float64), Q, n_dual=n_dual)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-5, atol=1e-6)
    loss = net.loss_grad(xd.data_ptr(), td.data_ptr(), N)
    g = net.get_grads().astype(np.float64)
    oloss, og = WN.loss_grad(params.astype(np.float64), x.astype(np.float64), t.astype(np.float64), Q,
                             n_dual=n_dual)
    assert loss == pytest.approx(oloss, rel=1e-5)
    for l, (w0, b0, ci, co) in enumerate(lay):
        for a, b in ((g[w0:b0], og[w0:b0]), (g[b0:b0 + co], og[b0:b0 + co])):
            err = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)
            assert err <= 1e-4, (l, err)


def test_adam_step_matches_formula():
    net, params, x, t, Q, N, lay = setup(seed=3)
    xd = torch.from_numpy(x).cuda()
    td = torch.from_numpy(t).cuda()
    net.loss_grad(xd.data_ptr(), td.data_ptr(), N)
    g = net.get_grads().astype(np.float64)
    net.adam_step(1e-3, 0.9, 0.999, 1e-8)
    new = net.get_params().astype(np.float64)
    m = 0.1 * g
    v = 0.001 * g * g
    expect = params.astype(np.float64) - 1e-3 * (m / 0.1) / (np.sqrt(v / 0.001) + 1e-8)
    np.testing.assert_allclose(new, expect, rtol=1e-5, atol=1e-7)


def test_unpack_dual_layout():
    # c [p][j], j = (x * Nz + z) * Nq + q, from the output's channels Nq + p * Nq + q
    Nx, Nz, Nq, nd = 4, 6, 3, 2
    rng = np.random.default_rng(4)
    out = rng.standard_normal((Nq * (1 + nd), Nx, Nz)).astype(np.float32)
    od = torch.from_numpy(out).cuda()
    c = torch.empty(nd * Nx * Nz * Nq, device="cuda")
    wsnet.unpack_dual(od.data_ptr(), Nx, Nz, Nq, nd, 0.5, c.data_ptr())
    torch.cuda.synchronize()
    expect = 0.5 * out[Nq:].reshape(nd, Nq, Nx, Nz).transpose(0, 2, 3, 1).reshape(-1)
    assert np.array_equal(c.cpu().numpy(), expect)
