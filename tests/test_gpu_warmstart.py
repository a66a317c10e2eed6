"""The learned warm start end to end at a small size: targets from the plain
method, training with the project's kernels, then held-out scans solved by
plain ADMM from the network's start and from the flat start. The network
only sets the starting point; the comparison is iterations and wall time to a
1e-4 relative objective gap of the same method."""
import numpy as np
import pytest

from paper_1601_08201_gb300 import warmstart as WS
from paper_1601_08201_gb300 import wsnet

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def test_trained_warm_start_reaches_tolerance_sooner():
    P = WS.instrument(32, 32, 16, nnz_col=64, seed=777)
    solver = WS.Solver(P, torch)
    X, T, _ = WS.build_dataset(solver, range(100, 228), 1500, torch)
    net = wsnet.WarmNet(32, 32, 16, 8, seed=0)
    losses = WS.train(net, X, T, epochs=40, batch=8, lr=2e-3)
    assert losses[-1] < 0.5 * losses[0]
    rows = WS.evaluate(solver, net, range(900, 912), 3000, 10, torch)
    s = WS.summarize(rows)
    print(s)
    assert s["reached"] == len(rows)
    # the network's start is closer to the solution and the solve reaches the
    # tolerance in fewer iterations on average
    assert s["start_gap_warm_median"] < s["start_gap_cold_median"]
    assert s["warm_iters_mean"] < s["cold_iters_mean"]
