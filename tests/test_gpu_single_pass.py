"""The single-pass form (SGTV_FLAG_SINGLE_PASS): A streamed once per
surrogate step by rows, each row's a_ij * ratio_i scattered into e, then an
elementwise f-update. Same iteration as the two-pass form; the sums of e are
formed in an order set by atomic adds, so the comparisons are within the
floating-point tolerances (FP64 1e-12, FP32 1e-5), never bitwise."""
import numpy as np
import pytest

import oracle as O
from paper_1601_08201_gb300 import sgtv, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

SP = sgtv.FLAG_SINGLE_PASS


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def maxrel(a, b, floor=1e-2):
    """max_j |a_j - b_j| / max(|b_j|, floor * max|b|): the worst single element."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.maximum(np.abs(b), floor * max(np.abs(b).max(), 1e-300))
    return float((np.abs(a - b) / den).max())


_cache = {}


def problem(name):
    if name not in _cache:
        _cache[name] = synth.preset(name)
    return _cache[name]


def run_both(P, ks, precision, flags=SP, n_dirs=4, w=None, n_inner=1, csr_val=None, csc_val=None, rho=None):
    op = O.from_problem(P, n_dirs=n_dirs, w=w, csr_val=csr_val, csc_val=csc_val, rho=rho)
    st = O.init_state(op)
    out = []
    kw = {} if rho is None else {"rho": rho}
    with sgtv.Handle(P, n_dirs=n_dirs, w=w, n_inner=n_inner, precision=precision, flags=flags, **kw) as h:
        done = 0
        for k in ks:
            h.iterate(k - done)
            st = O.iterate(op, st, k - done, n_inner)
            done = k
            out.append((k, h.get_state_f64(), st))
    return out


@pytest.mark.parametrize("name", ["tiny_16x16x32", "ragged_13x7x37", "paper_41x9x54", "wide_64x16x32"])
def test_single_pass_fp64_matches_oracle(name):
    for k, g, o in run_both(problem(name), [1, 10, 200], "fp64"):
        for a, b, what in zip(g, o, "fdc"):
            assert rel(a, b) <= 1e-12, (name, k, what, rel(a, b))


@pytest.mark.parametrize("name", ["tiny_16x16x32", "ragged_13x7x37", "paper_41x9x54", "wide_64x16x32"])
def test_single_pass_fp32_matches_oracle(name):
    for k, g, o in run_both(problem(name), [1, 10, 200], "fp32", flags=SP | sgtv.FLAG_GRAPH):
        assert rel(g[0], o[0]) <= 1e-5, (name, k, rel(g[0], o[0]))


@pytest.mark.parametrize("n_dirs,w,n_inner", [(2, [0.7, 1.4], 1), (4, [0.5, 1.3, 2.0, 0.7], 2)])
def test_single_pass_options(n_dirs, w, n_inner):
    P = problem("ragged_13x7x37")
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-5)):
        for k, g, o in run_both(P, [1, 20], prec, n_dirs=n_dirs, w=w, n_inner=n_inner):
            assert rel(g[0], o[0]) <= tol, (prec, k, rel(g[0], o[0]))


def test_single_pass_bf16_values():
    P = problem("tiny_16x16x32")
    out = run_both(P, [1, 10, 200], "bf16", csr_val=synth.round_to_bf16(P.csr_val),
                   csc_val=synth.round_to_bf16(P.csc_val))
    for k, g, o in out:
        assert rel(g[0], o[0]) <= 1e-5, (k, rel(g[0], o[0]))


def test_single_pass_rho_zero_is_mlem():
    P = problem("ragged_13x7x37")
    out = run_both(P, [3], "fp64", flags=SP | sgtv.FLAG_ALLOW_RHO0, rho=0.0)
    assert rel(out[0][1][0], out[0][2][0]) <= 1e-12


def test_single_pass_batch_per_scan():
    shapes = [(5, 4, 7, 90, 12, 20.0), (8, 3, 16, 300, 20, 60.0), (4, 4, 32, 500, 24, 8.0)]
    scans = [synth.make_problem(Nx, Nz, Nq, I, nc, n_regions=2, mean_counts=m, seed=60 + k, rho=0.5 + 0.5 * k)
             for k, (Nx, Nz, Nq, I, nc, m) in enumerate(shapes)]
    ops = [O.from_problem(P) for P in scans]
    sts = [O.iterate(op, O.init_state(op), 30) for op in ops]
    with sgtv.Handle(scans, precision="fp64", flags=SP) as h:
        h.iterate(30)
        f = h.get_state_f64()[0]
        off = h.batch_info()["vox_off"]
    for k in range(len(scans)):
        assert rel(f[off[k]:off[k + 1]], sts[k][0]) <= 1e-12, k


def test_single_pass_agrees_with_two_pass_and_profiles():
    P = problem("wide_64x16x32")
    with sgtv.Handle(P, precision="fp32") as h2:
        h2.iterate(50)
        f2 = h2.get_image()
    with sgtv.Handle(P, precision="fp32", flags=SP) as h1:
        h1.profile(True)
        h1.iterate(50)
        prof = h1.profile_read()
        f1 = h1.get_image()
        # the KKT measure and objective reuse the handle's scratch; the next
        # iterations still start from a cleared accumulator
        h1.residuals()
        h1.objective()
        h1.iterate(5)
        f1b = h1.get_image()
    assert rel(f1, f2) <= 1e-5
    assert prof["k_scatter"][1] == 50 and prof["k_fupdate"][1] == 50 and prof["k_shrink"][1] == 50
    assert prof["k_forward"][1] == 0 and prof["k_back_update"][1] == 0
    with sgtv.Handle(P, precision="fp32") as h2:
        h2.iterate(55)
        assert rel(f1b, h2.get_image()) <= 1e-5


def test_single_pass_rejects_persistent():
    P = problem("tiny_16x16x32")
    with pytest.raises(sgtv.SgtvError):
        sgtv.Handle(P, flags=SP | sgtv.FLAG_PERSISTENT)


@pytest.mark.parametrize("name", ["tiny_16x16x32", "ragged_13x7x37", "paper_41x9x54", "wide_64x16x32"])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5), ("bf16", 1e-5)])
def test_every_scatter_form_matches_oracle(name, prec, tol):
    # every scatter form, the bank-dealt row-stream ("sp_") forms included:
    # window and list tiles, ragged rows, rows longer than the kept chunks
    P = problem(name)
    if prec == "bf16":
        op = O.from_problem(P, csr_val=synth.round_to_bf16(P.csr_val), csc_val=synth.round_to_bf16(P.csc_val))
    else:
        op = O.from_problem(P)
    st = O.iterate(op, O.init_state(op), 10)
    with sgtv.Handle(P, precision=prec, flags=SP | sgtv.FLAG_NO_AUTOTUNE) as h:
        names = h.variant_names()["k_scatter"]
        assert len(names) >= 2 and any(nm.startswith("sp_") for nm in names)
        s0 = h.get_state_f64()
        ran = []
        for v in range(len(names)):
            h.set_state_f64(*s0)
            try:
                h.set_variant(sgtv.K_SCATTER, v)
            except sgtv.SgtvError as err:
                # forms with one accumulator per warp need 9 staging-sized
                # buffers in shared memory: refused (SGTV_ERR_ARG, not
                # sticky) where a tile's staging buffer is too wide for that
                assert err.code == -1, (names[v], err)
                h.sync()
                continue
            ran.append(names[v])
            assert h.get_variant(sgtv.K_SCATTER) == v
            h.iterate(10)
            f = h.get_state_f64()[0]
            assert rel(f, st[0]) <= tol, (names[v], rel(f, st[0]))
            assert maxrel(f, st[0]) <= 100 * tol, (names[v], maxrel(f, st[0]))
        assert len(ran) >= 2 and any(nm.startswith("sp_") for nm in ran), ran
        with pytest.raises(sgtv.SgtvError):
            h.set_variant(sgtv.K_SCATTER, len(names))
