"""Failure detection without a GPU fault: a bounded device-side wait that runs
out is reported, the error is sticky, and the GPU context stays usable.

The persistent launch (one cooperative kernel per iteration) separates its
phases by grid-wide barriers whose waits are bounded. sgtv_set_wait_limit(0)
makes every block that is not the last to arrive give up at its first look,
so the launch returns early and the next synchronising call reports
SGTV_ERR_TIMEOUT. No wait in the kernel is unbounded and no bulk copy is in
flight at a barrier, so the blocks that give up exit cleanly."""
import numpy as np
import pytest

import oracle as O
from paper_1601_08201_gb300 import sgtv, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def test_grid_barrier_wait_runs_out_and_is_reported():
    P = synth.preset("wide_64x16x32")  # 512 row tiles: a grid of many blocks
    with sgtv.Handle(P, precision="fp32", flags=sgtv.FLAG_PERSISTENT) as h:
        h.iterate(2)
        h.sync()  # healthy with the default bound
        with pytest.raises(sgtv.SgtvError) as bad:
            h.set_wait_limit(-1)
        assert bad.value.code == -1
        h.sync()  # a rejected argument is not sticky
        h.set_wait_limit(0)
        h.iterate(1)
        with pytest.raises(sgtv.SgtvError) as err:
            h.sync()
        assert err.value.code == -6  # SGTV_ERR_TIMEOUT
        assert "wait" in sgtv.last_error(h.h)
        # sticky: every later call on the handle is refused
        with pytest.raises(sgtv.SgtvError) as again:
            h.iterate(1)
        assert again.value.code == -5  # SGTV_ERR_STATE
    # the context is intact: a new handle iterates and matches the oracle
    op = O.from_problem(P)
    ref = O.iterate(op, O.init_state(op), 3)
    with sgtv.Handle(P, precision="fp32", flags=sgtv.FLAG_PERSISTENT) as h:
        h.iterate(3)
        f = h.get_state_f64()[0]
    assert rel(f, ref[0]) <= 1e-5
