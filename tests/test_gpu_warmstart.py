"""The learned warm start end to end at a small size: targets from the plain
method, training with the project's kernels, then held-out scans solved by
plain ADMM from the network's start and from the flat start. The network
only sets the starting point; the method, and the optimum it reaches, are the
same from either start.

What is asserted: training fits, the network's image starts closer to the
optimum than the flat start, the solve from it reaches the same optimum, and
a start that carries the dual of the group shrink (sgtv_warm_start with
dual_scale = 1) from a converged image stays near the optimum where the flat
start is still far from it. Whether the network's start saves iterations is
measured (printed), not asserted: with the scaled dual starting at zero the
dual variable, not the image, sets the pace of convergence."""
import numpy as np
import pytest

from paper_1601_08201_gb300 import synth
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
