"""The learned warm start end to end at a small size: targets from the plain
method, training with the project's kernels, then held-out scans solved by
plain ADMM from the network's start and from the flat start. The network
only sets the starting point; the method, and the optimum it reaches, are the
same from either start.

What is asserted: training fits, the network's image starts closer to the
optimum than the flat start, the solve from it reaches the same optimum, and
a start that carries the dual of the group shrink (sgtv_warm_start with
dual_scale = 1) from a converged image stays near the optimum where the flat
start is still far from it. An image alone saves no iterations: the scaled
dual restarts from zero and sets the pace of convergence. The network with
dual channels (sgtv_warm_start_dual) is the one that gains: on held-out scans
its dual is closer to the converged dual than zero is, and after a fixed
number of iterations the solve from its start sits closer to the optimum
than the solve from the flat start. At the configured 64 x 64 x 64 shape,
with targets and solves at a large penalty (the same minimum, reached in a
few thousand iterations), the image-only start already gains: it reaches a
relative gap of 1e-3 in fewer iterations than the flat start."""
import numpy as np
import pytest

from paper_1601_08201_gb300 import sgtv, synth
from paper_1601_08201_gb300 import warmstart as WS
from paper_1601_08201_gb300 import wsnet

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def solver():
    P = WS.instrument(32, 32, 16, nnz_col=64, seed=777)
    return WS.Solver(P, torch)


def test_trained_network_start_is_closer_and_reaches_the_same_optimum(solver):
    X, T, _ = WS.build_dataset(solver, range(100, 164), 3000, torch)
    net = wsnet.WarmNet(32, 32, 16, 8, seed=0)
    losses = WS.train(net, X, T, epochs=30, batch=8, lr=2e-3)
    assert losses[-1] < 0.2 * losses[0]
    rows = WS.evaluate(solver, net, range(900, 904), 6000, 10, torch, star_iters=20000,
                       starts=(("warm", 0.0),), tols=(1e-3,))
    s = WS.summarize(rows, ("warm",), (1e-3,))
    print(s)
    assert s["warm_start_gap_median"] < s["cold_start_gap_median"]
    for r in rows:
        assert r["warm_iters@0.001"] is not None  # same optimum, to 1e-3, from the network's start


def test_shrink_consistent_dual_keeps_a_converged_start_converged(solver):
    h = solver.h
    for seed in (900, 901):
        M = synth.measure(solver.P, seed)
        solver.load(M)
        h.iterate(30000)
        phi_star = h.objective()[0]
        f_star = h.get_image()
        solver.load(M)
        h.iterate(1000)
        cold = (h.objective()[0] - phi_star) / phi_star
        solver.load(M)
        h.warm_start(f_star, dual_scale=1.0)
        h.iterate(1000)
        warm = (h.objective()[0] - phi_star) / phi_star
        print(seed, cold, warm)
        assert warm < 0.2 * cold


def test_dual_head_start_is_closer_after_fixed_iterations(solver):
    P = solver.P
    X, T, _ = WS.build_dataset(solver, range(3000, 4024), 5000, torch, n_dual=4)
    net = wsnet.WarmNet(32, 32, 16, 8, seed=0, n_dual=4)
    losses = WS.train(net, X, T, epochs=40, batch=8, lr=2e-3)
    assert losses[-1] < 0.2 * losses[0]
    h = solver.h
    dual_err, ratios = [], []
    for seed in range(5000, 5012):
        M = synth.measure(P, seed)
        solver.load(M)
        h.iterate(20000)
        phi_star = h.objective()[0]
        c_star = h.get_state_f64()[2]
        gaps = {}
        for name in ("cold", "warm"):
            solver.load(M)
            if name == "warm":
                f0, c0 = WS.warm_image(solver, net, M, torch, with_dual=True)
                h.warm_start_dual(f0.data_ptr(), c0.data_ptr())
                dual_err.append(float(np.linalg.norm(c0.cpu().numpy() - c_star) / np.linalg.norm(c_star)))
            h.iterate(300)
            g300 = (h.objective()[0] - phi_star) / phi_star
            h.iterate(700)
            gaps[name] = (g300, (h.objective()[0] - phi_star) / phi_star)
        ratios += [max(w, 1e-12) / c for w, c in zip(gaps["warm"], gaps["cold"])]
    print("dual rel. error", np.round(dual_err, 3), "gap ratios after 300 / 1000 iterations", np.round(ratios, 3))
    assert np.median(dual_err) < 1.0  # the predicted dual beats the method's zero start
    # geometric mean over 12 held-out scans and both budgets: the start that
    # carries the network's dual is closer to the optimum than the flat start
    assert np.exp(np.mean(np.log(ratios))) < 1.0


def test_gain_at_64_cubed_with_fast_penalty():
    # The configured shape (64 x 64 spatial x 64 q-bins, 128 nonzeros per
    # column). Targets and phi* come from solves at rho = 4096 (the minimum
    # does not depend on rho; a large penalty converges in a few thousand
    # iterations), and cold and warm solves run at that penalty too. The
    # network's image starts far closer to the optimum, and the solve from it
    # reaches a relative gap of 1e-3 in fewer iterations than the flat start.
    P = WS.instrument(64, 64, 64, 128)
    flags = sgtv.FLAG_GRAPH | sgtv.FLAG_SINGLE_PASS
    solver = WS.Solver(P, torch, flags=flags, rho=4096.0)
    X, T, _ = WS.build_dataset(solver, range(10000, 10128), 3000, torch)
    net = wsnet.WarmNet(64, 64, 64, 8, seed=0)
    losses = WS.train(net, X, T, epochs=20, batch=8, lr=1e-3)
    assert losses[-1] < 0.5 * losses[0]
    rows = WS.evaluate(solver, net, range(20000, 20008), 4000, 100, torch, star_iters=8000,
                       starts=(("warm", 0.0),), tols=(1e-3,))
    s = WS.summarize(rows, ("warm",), (1e-3,))
    print(s)
    assert s["warm_start_gap_median"] < 0.5 * s["cold_start_gap_median"]
    assert s["warm_over_cold_gap@300_median"] < 0.5 and s["warm_over_cold_gap@1000_median"] < 0.5
    r = s["warm@0.001"]
    assert r["reached"] >= 6 and r["warm_fewer_frac"] >= 0.75 and r["iters_ratio"] < 0.9
