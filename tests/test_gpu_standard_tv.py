"""The standard isotropic TV (SGTV_FLAG_STANDARD_TV): one group per (site,
q-bin), the regulariser the paper compares its group TV against. CUDA path
against the FP64 oracle run with per_bin = True, in every launch form."""
import numpy as np
import pytest

import oracle as O
from paper_1601_08201_gb300 import sgtv, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

STD = sgtv.FLAG_STANDARD_TV


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("name", ["tiny_16x16x32", "ragged_13x7x37", "paper_41x9x54"])
@pytest.mark.parametrize("flags", [0, sgtv.FLAG_GRAPH, sgtv.FLAG_SINGLE_PASS])
def test_standard_tv_matches_oracle(name, flags):
    P = synth.preset(name)
    op = O.from_problem(P, per_bin=True)
    st = O.init_state(op)
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-5)):
        st = O.init_state(op)
        with sgtv.Handle(P, precision=prec, flags=STD | flags) as h:
            done = 0
            for k in (1, 10, 100):
                h.iterate(k - done)
                st = O.iterate(op, st, k - done)
                done = k
                f, d, c = h.get_state_f64()
                assert rel(f, st[0]) <= tol, (prec, k, rel(f, st[0]))
                if prec == "fp64":
                    assert rel(d, st[1]) <= tol and rel(c, st[2]) <= tol, (k, rel(d, st[1]), rel(c, st[2]))
            phi, dev, tv = h.objective()
            ophi, odev, otv = O.objective(op, f)
            assert tv == pytest.approx(otv, rel=1e-11) and phi == pytest.approx(ophi, rel=1e-11)


def test_standard_tv_differs_from_group_tv():
    P = synth.preset("tiny_16x16x32")
    with sgtv.Handle(P, precision="fp64") as hg, sgtv.Handle(P, precision="fp64", flags=STD) as hs:
        hg.iterate(100)
        hs.iterate(100)
        fg, fs = hg.get_image(), hs.get_image()
        assert hs.objective()[2] != pytest.approx(hg.objective()[2], rel=1e-6)
    assert rel(fs, fg) > 1e-4


def test_standard_tv_persistent_batch():
    shapes = [(5, 4, 7, 90, 12, 20.0), (8, 3, 16, 300, 20, 60.0), (6, 7, 5, 160, 16, 35.0)]
    scans = [synth.make_problem(Nx, Nz, Nq, I, nc, n_regions=2, mean_counts=m, seed=70 + k, rho=0.5 + 0.5 * k)
             for k, (Nx, Nz, Nq, I, nc, m) in enumerate(shapes)]
    ops = [O.from_problem(P, per_bin=True) for P in scans]
    sts = [O.iterate(op, O.init_state(op), 20) for op in ops]
    with sgtv.Handle(scans, precision="fp64", flags=STD | sgtv.FLAG_PERSISTENT | sgtv.FLAG_GRAPH) as h:
        h.iterate(20)
        f = h.get_state_f64()[0]
        off = h.batch_info()["vox_off"]
        for k, op in enumerate(ops):
            fk = f[off[k]:off[k + 1]]
            assert rel(fk, sts[k][0]) <= 1e-12, k
            assert h.objective_scan(k)[2] == pytest.approx(O.objective(op, fk)[2], rel=1e-11)


def test_standard_tv_warm_start_dual_rule():
    P = synth.preset("ragged_13x7x37")
    op = O.from_problem(P, per_bin=True)
    f0 = np.random.default_rng(8).uniform(0.1, 2.0, P.J).astype(np.float32)
    d = O.wgrad(op, f0.astype(np.float64))
    with sgtv.Handle(P, precision="fp64", flags=STD) as h:
        h.warm_start(f0, dual_scale=0.7)
        g = h.get_state_f64()
    assert rel(g[2], O.dual_rule(op, d, 0.7)) <= 1e-12
