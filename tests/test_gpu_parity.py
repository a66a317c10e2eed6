"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances, relative L2 over the whole array (rel) and the worst single
element, |g_j - o_j| / max(|o_j|, 1e-2 max|o|) (maxrel), after k iterations:
  FP64 mode : rel 1e-12 and maxrel 1e-10 on f, d, c (only summation order differs)
  FP32 mode : rel 1e-5 on f and c (the FP32 bound), 1e-4 on d (a difference
              field: the image's relative error grows by ||f|| / ||w.G f||),
              maxrel 1e-3 on each (about 100x the L2 error, far below the
              O(1) error of a wrong voxel or tile); objective 1e-7 relative
  objective reductions at the GPU's own iterate: 1e-11 (FP64 sums either side)
"""
import numpy as np
import pytest

import oracle as O
from paper_1601_08201_gb300 import sgtv, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def maxrel(a, b, floor=1e-2):
    """Worst element: max_j |a_j - b_j| / max(|b_j|, floor * max|b|) (0 if b = 0 and a = b)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    m = np.abs(b).max() if b.size else 0.0
    if m == 0.0:
        return float(np.abs(a).max()) if a.size else 0.0
    return float((np.abs(a - b) / np.maximum(np.abs(b), floor * m)).max())


_cache = {}


def problem(name, **kw):
    key = (name, tuple(sorted(kw.items())))
    if key not in _cache:
        _cache[key] = synth.preset(name, **kw)
    return _cache[key]


def run_both(P, ks, precision, n_dirs=4, w=None, n_inner=1, csr_val=None, csc_val=None):
    """GPU and oracle states after each k in ks (cumulative)."""
    op = O.from_problem(P, n_dirs=n_dirs, w=w, csr_val=csr_val, csc_val=csc_val)
    st = O.init_state(op)
    out = []
    with sgtv.Handle(P, n_dirs=n_dirs, w=w, n_inner=n_inner, precision=precision) as h:
        g0 = h.get_state_f64()
        out.append((0, g0, st))
        done = 0
        for k in ks:
            h.iterate(k - done)
            st = O.iterate(op, st, k - done, n_inner)
            done = k
            out.append((k, h.get_state_f64(), st))
    return op, out


@pytest.mark.parametrize("name", ["tiny_16x16x32", "ragged_13x7x37", "paper_41x9x54", "wide_64x16x32"])
def test_fp64_matches_oracle(name):
    P = problem(name)
    _, out = run_both(P, [1, 10, 200], "fp64")
    for k, g, o in out:
        for a, b, what in zip(g, o, "fdc"):
            assert rel(a, b) <= 1e-12, (name, k, what, rel(a, b))
            assert maxrel(a, b) <= 1e-10, (name, k, what, maxrel(a, b))


@pytest.mark.parametrize("name", ["tiny_16x16x32", "ragged_13x7x37", "paper_41x9x54", "wide_64x16x32"])
def test_fp32_matches_oracle(name):
    P = problem(name)
    op, out = run_both(P, [1, 10, 200], "fp32")
    for k, g, o in out:
        for a, b, what, tol in zip(g, o, "fdc", (1e-5, 1e-4, 1e-5)):
            assert rel(a, b) <= tol, (name, k, what, rel(a, b))
            assert maxrel(a, b) <= 1e-3, (name, k, what, maxrel(a, b))
        phi, ophi = O.objective(op, g[0])[0], O.objective(op, o[0])[0]
        assert abs(phi - ophi) <= 1e-7 * ophi, (name, k, abs(phi - ophi) / ophi)


@pytest.mark.parametrize("n_dirs,w,n_inner", [(2, [0.7, 1.4], 1), (4, [0.5, 1.3, 2.0, 0.7], 2)])
def test_options_match_oracle(n_dirs, w, n_inner):
    P = problem("ragged_13x7x37")
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-5)):
        _, out = run_both(P, [1, 20], prec, n_dirs=n_dirs, w=w, n_inner=n_inner)
        for k, g, o in out:
            assert rel(g[0], o[0]) <= tol, (prec, k, rel(g[0], o[0]))
            assert maxrel(g[0], o[0]) <= (1e-10 if prec == "fp64" else 1e-3), (prec, k, maxrel(g[0], o[0]))


def test_bf16_values_match_oracle_on_rounded_matrix():
    P = problem("tiny_16x16x32")
    rv = synth.round_to_bf16(P.csr_val)
    cv = synth.round_to_bf16(P.csc_val)
    _, out = run_both(P, [1, 10, 200], "bf16", csr_val=rv, csc_val=cv)
    for k, g, o in out:
        for a, b, what, tol in zip(g, o, "fdc", (1e-5, 1e-4, 1e-5)):
            assert rel(a, b) <= tol, (k, what, rel(a, b))
            assert maxrel(a, b) <= 1e-3, (k, what, maxrel(a, b))


@pytest.mark.parametrize("flags", [0, sgtv.FLAG_GRAPH, sgtv.FLAG_SINGLE_PASS])
def test_objective_and_residuals_at_gpu_iterate(flags):
    # the reductions at the GPU's own iterate, against the oracle's formulas
    # at the same state (d_prev = the GPU's d one iteration earlier)
    # beta at 0.3 of the preset's: at the preset's own beta every group is
    # still shrunk to zero after 30 iterations (d = 0 does not move, so the
    # dual residual is exactly 0 there); here d is active and changing
    P = problem("tiny_16x16x32")
    beta = 0.3 * P.beta
    op = O.from_problem(P, beta=beta)
    for prec in ("fp64", "fp32"):
        with sgtv.Handle(P, lam=beta, precision=prec, flags=flags) as h:
            assert h.residuals()[1] == 0.0  # no iteration yet: d_prev = d
            h.iterate(29)
            d_prev = h.get_state_f64()[1]
            h.iterate(1)
            phi, dev, tv = h.objective()
            f, d, c = h.get_state_f64()
            ophi, odev, otv = O.objective(op, f)
            assert dev == pytest.approx(odev, rel=1e-11)
            assert tv == pytest.approx(otv, rel=1e-11)
            assert phi == pytest.approx(ophi, rel=1e-11)
            primal, dual, kkt = h.residuals()
            oprimal, odual, okkt = O.residuals(op, f, d, c, d_prev)
            assert primal == pytest.approx(oprimal, rel=1e-9)
            assert dual > 0.0
            assert dual == pytest.approx(odual, rel=1e-9)
            tol = 1e-10 if prec == "fp64" else 1e-5
            assert abs(kkt - okkt) <= tol * max(1.0, abs(okkt)) + tol
            # a state set from outside has no previous d
            h.set_state_f64(f, d, c)
            assert h.residuals()[1] == 0.0


def test_objective_trajectory_fp32_against_oracle():
    P = problem("tiny_16x16x32")
    op = O.from_problem(P)
    st = O.init_state(op)
    with sgtv.Handle(P, precision="fp32") as h:
        done = 0
        for k in (1, 10, 200):
            h.iterate(k - done)
            st = O.iterate(op, st, k - done)
            done = k
            phi = h.objective()[0]
            ophi = O.objective(op, st[0])[0]
            assert abs(phi - ophi) <= 1e-7 * abs(ophi), (k, phi, ophi)


def test_rho_zero_is_mlem():
    P = problem("ragged_13x7x37")
    op = O.from_problem(P, rho=0.0)
    with sgtv.Handle(P, rho=0.0, precision="fp64", flags=sgtv.FLAG_ALLOW_RHO0) as h:
        f0 = h.get_state_f64()[0]
        h.iterate(3)
        f3 = h.get_state_f64()[0]
    st = O.iterate(op, (f0, np.zeros(4 * P.J), np.zeros(4 * P.J)), 3)
    assert rel(f3, st[0]) <= 1e-12


def test_state_roundtrip_and_warm_start():
    P = problem("ragged_13x7x37")
    op = O.from_problem(P)
    rng = np.random.default_rng(3)
    f = rng.uniform(0.1, 2.0, P.J)
    with sgtv.Handle(P, precision="fp64") as h:
        h.set_state_f64(f)
        g = h.get_state_f64()
        assert np.array_equal(g[0], f)
        np.testing.assert_allclose(g[1], O.wgrad(op, f), rtol=1e-14, atol=1e-15)
        assert not g[2].any()
        h.iterate(5)
        o = O.iterate(op, (f, O.wgrad(op, f), np.zeros(4 * P.J)), 5)
        assert rel(h.get_state_f64()[0], o[0]) <= 1e-12
        # checkpoint, continue, restore, continue again: identical
        ck = h.get_state_f64()
        h.iterate(7)
        a = h.get_state_f64()
        h.set_state_f64(*ck)
        h.iterate(7)
        b = h.get_state_f64()
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_warm_start_dual_rule(precision, tol):
    P = problem("ragged_13x7x37")
    op = O.from_problem(P)
    rng = np.random.default_rng(5)
    f0 = rng.uniform(-0.2, 2.0, P.J).astype(np.float32)
    f = np.maximum(f0.astype(np.float64), 0.0)
    d = O.wgrad(op, f)
    with sgtv.Handle(P, precision=precision) as h:
        for theta in (1.0, 0.6, 0.0):
            h.warm_start(f0, dual_scale=theta)
            g = h.get_state_f64()
            assert np.array_equal(g[0], f)
            assert rel(g[1], d) <= tol
            assert rel(g[2], O.dual_rule(op, d, theta)) <= tol if theta else not g[2].any()
        h.warm_start(f0, dual_scale=1.0)
        h.iterate(4)
        o = O.iterate(op, (f, d, O.dual_rule(op, d, 1.0)), 4)
        assert rel(h.get_state_f64()[0], o[0]) <= (1e-12 if precision == "fp64" else 1e-4)
        with pytest.raises(sgtv.SgtvError):
            h.warm_start(f0, dual_scale=1.5)


def test_warm_start_with_given_dual():
    P = problem("ragged_13x7x37")
    op = O.from_problem(P)
    rng = np.random.default_rng(6)
    f0 = rng.uniform(-0.2, 2.0, P.J).astype(np.float32)
    c0 = rng.standard_normal(4 * P.J).astype(np.float32)
    f = np.maximum(f0.astype(np.float64), 0.0)
    d = O.wgrad(op, f)
    with sgtv.Handle(P, precision="fp64") as h:
        h.warm_start_dual(f0, c0)
        g = h.get_state_f64()
        assert np.array_equal(g[0], f) and np.array_equal(g[2], c0.astype(np.float64))
        assert rel(g[1], d) <= 1e-12
        h.iterate(4)
        o = O.iterate(op, (f, d, c0.astype(np.float64)), 4)
        assert rel(h.get_state_f64()[0], o[0]) <= 1e-12
        bad = c0.copy()
        bad[7] = np.nan
        with pytest.raises(sgtv.SgtvError):
            h.warm_start_dual(f0, bad)


def test_edge_cases_empty_rows_columns_vector_background():
    # Empty rows and columns, zero counts, per-measurement background, Nq = 1.
    rng = np.random.default_rng(17)
    Nx, Nz, Nq, I = 5, 3, 1, 40
    J = Nx * Nz * Nq
    A = (rng.random((I, J)) < 0.2) * rng.uniform(0.1, 1.0, (I, J))
    A[7, :] = 0.0       # empty row
    A[:, 4] = 0.0       # empty column
    A = A.astype(np.float32)
    import scipy.sparse as sp
    csr = sp.csr_matrix(A)
    csc = sp.csc_matrix(A)
    csr.sort_indices()
    csc.sort_indices()
    b = rng.uniform(0.5, 1.5, I).astype(np.float32)
    y = rng.poisson(A @ np.full(J, 3.0) + b).astype(np.float32)
    y[:3] = 0
    P = synth.Problem(Nx=Nx, Nz=Nz, Nq=Nq, I=I, J=J, nnz=csr.nnz,
                      csc_colptr=csc.indptr.astype(np.int64), csc_row=csc.indices.astype(np.int32),
                      csc_val=csc.data.astype(np.float32), csr_rowptr=csr.indptr.astype(np.int64),
                      csr_col=csr.indices.astype(np.int32), csr_val=csr.data.astype(np.float32),
                      y=y, b=b, beta=2.0, rho=1.0, f_true=np.zeros(J, np.float32))
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-5)):
        _, out = run_both(P, [1, 50], prec)
        for k, g, o in out:
            for a, bb, what in zip(g, o, "fdc"):
                assert rel(a, bb) <= tol, (prec, k, what, rel(a, bb))


def test_single_voxel():
    I, J = 6, 1
    P = synth.Problem(Nx=1, Nz=1, Nq=1, I=I, J=J, nnz=I,
                      csc_colptr=np.array([0, I], np.int64), csc_row=np.arange(I, dtype=np.int32),
                      csc_val=np.linspace(0.2, 1.0, I).astype(np.float32),
                      csr_rowptr=np.arange(I + 1, dtype=np.int64), csr_col=np.zeros(I, np.int32),
                      csr_val=np.linspace(0.2, 1.0, I).astype(np.float32),
                      y=np.array([1, 0, 3, 2, 5, 4], np.float32), b=np.array([0.3], np.float32),
                      beta=0.4, rho=1.0, f_true=np.zeros(1, np.float32))
    _, out = run_both(P, [1, 30], "fp64")
    for k, g, o in out:
        for a, bb in zip(g, o):
            assert rel(a, bb) <= 1e-12


def test_device_validation_rejects_mismatched_copies():
    P = problem("ragged_13x7x37")
    bad = P.csc_val.copy()
    bad[100] += 0.25
    with pytest.raises(sgtv.SgtvError, match="differ"):
        sgtv.setup(P.I, P.J, P.nnz, P.csr_rowptr, P.csr_col, P.csr_val, P.csc_colptr, P.csc_row, bad,
                   P.Nx, P.Nz, P.Nq, P.y, P.b, P.beta, P.rho)
    badi = P.csr_col.copy()
    badi[10] = P.J + 3
    with pytest.raises(sgtv.SgtvError, match="out of range"):
        sgtv.setup(P.I, P.J, P.nnz, P.csr_rowptr, badi, P.csr_val, P.csc_colptr, P.csc_row, P.csc_val,
                   P.Nx, P.Nz, P.Nq, P.y, P.b, P.beta, P.rho)
    unsorted = P.csc_row.copy()
    unsorted[0], unsorted[1] = unsorted[1], unsorted[0]
    with pytest.raises(sgtv.SgtvError, match="ascending"):
        sgtv.setup(P.I, P.J, P.nnz, P.csr_rowptr, P.csr_col, P.csr_val, P.csc_colptr, unsorted,
                   P.csc_val, P.Nx, P.Nz, P.Nq, P.y, P.b, P.beta, P.rho)
    negv = P.csr_val.copy()
    negv[4] = -0.1
    with pytest.raises(sgtv.SgtvError, match="negative"):
        sgtv.setup(P.I, P.J, P.nnz, P.csr_rowptr, P.csr_col, negv, P.csc_colptr, P.csc_row, P.csc_val,
                   P.Nx, P.Nz, P.Nq, P.y, P.b, P.beta, P.rho)


def test_nonfinite_iterate_is_reported():
    # An FP32 image near the float maximum overflows ybar and the gradients: the
    # shrink kernel flags the non-finite group norm and sync reports it.
    P = problem("ragged_13x7x37")
    h = sgtv.Handle(P, precision="fp32")
    h.set_state_f64(np.full(P.J, 3.0e38))
    h.iterate(2)
    with pytest.raises(sgtv.SgtvError) as ei:
        h.sync()
    assert ei.value.code == -7
    with pytest.raises(sgtv.SgtvError) as ei:
        h.iterate(1)
    assert ei.value.code == -5  # sticky
    h.close()


def test_profile_counts_launches():
    P = problem("tiny_16x16x32")
    with sgtv.Handle(P) as h:
        h.profile(True)
        h.iterate(5)
        prof = h.profile_read()
        assert prof["k_forward"][1] == 5 and prof["k_back_update"][1] == 5 and prof["k_shrink"][1] == 5
        assert prof["k_iteration"][1] == 0
        assert all(ms > 0 for ms, n in prof.values() if n)


@pytest.mark.parametrize("flags", [0, sgtv.FLAG_GRAPH])
def test_serial_and_overlapped_shrink_give_the_same_iterate(flags):
    # the shrink on a second stream (default), on the handle's stream
    # (SGTV_FLAG_SERIAL at set-up), and toggled between the two with
    # sgtv_set_serial mid-solve: the same kernels in the same order of
    # dependence, so the same bits (two-pass form, no atomics)
    P = problem("wide_64x16x32")
    states = []
    for mode in ("overlap", "serial", "toggle"):
        fl = flags | (sgtv.FLAG_SERIAL if mode == "serial" else 0)
        with sgtv.Handle(P, flags=fl | sgtv.FLAG_NO_AUTOTUNE) as h:
            if mode == "toggle":
                h.iterate(7)
                h.set_serial(True)
                h.profile(True)
                h.iterate(9)
                prof = h.profile_read()
                h.profile(False)
                h.set_serial(False)
                h.iterate(4)
                if not flags:
                    assert prof["k_shrink"][1] == 9
            else:
                h.iterate(20)
            states.append(h.get_state_f64())
    for a, b in zip(states[0], states[1]):
        assert np.array_equal(a, b)
    for a, b in zip(states[0], states[2]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("name", ["ragged_13x7x37", "wide_64x16x32"])
def test_all_spmv_variants_bit_identical(name):
    P = problem(name)
    with sgtv.Handle(P, precision="fp32", flags=sgtv.FLAG_NO_AUTOTUNE) as h:
        names = h.variant_names()
        assert h.get_variants() == (0, 0)
        h.iterate(5)
        ref = h.get_state_f64()
    nf, nb = len(names["k_forward"]), len(names["k_back_update"])
    assert nf >= 2 and nb >= 2
    ran = set()
    for vf in range(nf):
        for vb in range(nb):
            with sgtv.Handle(P, precision="fp32", flags=sgtv.FLAG_NO_AUTOTUNE) as h:
                try:
                    h.set_variants(vf, vb)
                except sgtv.SgtvError:
                    continue  # that tiled form does not fit this problem
                h.iterate(5)
                st = h.get_state_f64()
            nf_, nb_ = names["k_forward"][vf], names["k_back_update"][vb]
            ran.add((nf_, nb_))
            if "v4" in nf_ or "v4" in nb_:
                # the 4-wide forms split a segment among lanes differently: same
                # arithmetic, another rounding order
                for a, b in zip(st, ref):
                    assert rel(a, b) <= 1e-6, (nf_, nb_, rel(a, b))
            else:
                for a, b in zip(st, ref):
                    assert np.array_equal(a, b), (nf_, nb_)
    # every form was exercised on these small problems
    assert ("tma_ns3_w16", "tma_ns3_w16") in ran and ("tli_u8", "tli_u8") in ran
    with sgtv.Handle(P) as h:
        vf, vb = h.autotune(2)
        assert 0 <= vf < nf and 0 <= vb < nb
        with pytest.raises(sgtv.SgtvError):
            h.set_variants(nf, 0)
        h.iterate(1)  # the rejected index was not sticky


@pytest.mark.parametrize("variants", [("tma_ns3_w16", "tma_ns3_w16"), ("tma_ns3_w8", "tma_ns3_w8"), ("tli_u8", "tli_u8"),
                                      ("tli_v4x2", "tli_v4x3")])
def test_tiled_variants_match_oracle(variants):
    # the tiled kernels against the oracle directly (list, window and mixed tiles)
    P = problem("wide_64x16x32")
    op = O.from_problem(P)
    st = O.iterate(op, O.init_state(op), 30)
    with sgtv.Handle(P, precision="fp32", flags=sgtv.FLAG_NO_AUTOTUNE) as h:
        names = h.variant_names()
        h.set_variants(names["k_forward"].index(variants[0]), names["k_back_update"].index(variants[1]))
        h.iterate(30)
        f = h.get_state_f64()[0]
    assert rel(f, st[0]) <= 1e-5


def test_tiled_forms_built():
    # wide image: row tiles need unique-index lists, column tiles mix windows
    # and lists; ragged: everything fits windows
    with sgtv.Handle(problem("wide_64x16x32")) as h:
        ti = h.tli_info()
        assert ti["csr"]["fmt"] == 1 and ti["csr"]["list_entries"] > 0
        assert ti["csc"]["fmt"] == 3 and ti["csc"]["window_elems"] > 0 and ti["csc"]["list_entries"] > 0
    with sgtv.Handle(problem("ragged_13x7x37")) as h:
        ti = h.tli_info()
        assert ti["csr"]["fmt"] == 2 and ti["csc"]["fmt"] == 2
