"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code: dense NumPy
matrices built from array slicing stand in for A and G, SciPy solvers stand
in for the closed forms, and the optimality certificate at convergence is
written from the problem statement (Sec. II Eqs. 1-2, Sec. III Eq. 4), not
from the iteration. A plausible slip in the oracle (a dropped ghost term, a
wrong neighbour direction, a transposed product, a wrong sign in gamma, the
wrong curvature split) fails at least one of them.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1601_08201_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------------------
# independent dense restatements (array slicing, no oracle code)

def dense_A(P):
    A = np.zeros((P.I, P.J))
    for j in range(P.J):
        lo, hi = P.csc_colptr[j], P.csc_colptr[j + 1]
        A[P.csc_row[lo:hi], j] = P.csc_val[lo:hi]
    return A


def diff_ops(Nx, Nz, Nq, n_dirs):
    """List of functions g_p(f3) -> (G_p f) on (Nx, Nz, Nq) arrays, zero ghosts."""
    def shift(f3, axis, step):
        # value of the neighbour at index + step along axis; 0 outside the domain
        out = np.zeros_like(f3)
        n = f3.shape[axis]
        src = [slice(None)] * 3
        dst = [slice(None)] * 3
        if step > 0:
            src[axis] = slice(step, n)
            dst[axis] = slice(0, n - step)
        else:
            src[axis] = slice(0, n + step)
            dst[axis] = slice(-step, n)
        out[tuple(dst)] = f3[tuple(src)]
        return out

    if n_dirs == 4:
        moves = [(0, +1), (0, -1), (1, +1), (1, -1)]
    else:
        moves = [(0, +1), (1, +1)]
    return [lambda f3, a=a, s=s: f3 - shift(f3, a, s) for a, s in moves]


def dense_WG(Nx, Nz, Nq, n_dirs, w):
    """Dense (n_dirs*J) x J matrix of w.G, direction-major rows."""
    J = Nx * Nz * Nq
    ops = diff_ops(Nx, Nz, Nq, n_dirs)
    M = np.zeros((n_dirs * J, J))
    eye = np.eye(J)
    for j in range(J):
        f3 = eye[j].reshape(Nx, Nz, Nq)
        M[:, j] = np.concatenate([w[p] * ops[p](f3).ravel() for p in range(n_dirs)])
    return M


def group_norms(g, n_dirs, S, Nq):
    J = S * Nq
    g = g.reshape(n_dirs, S, Nq)
    return np.sqrt((g ** 2).sum(axis=(0, 2)))


def tiny_problem(Nx=4, Nz=3, Nq=5, I=48, nnz_col=10, seed=3, **kw):
    return synth.make_problem(Nx, Nz, Nq, I, nnz_col, n_regions=2, mean_counts=30.0,
                              seed=seed, **kw)


# ----------------------------------------------------------------------------------------
# generator sanity (inputs both sides consume)

def test_generator_csr_is_csc_transpose():
    P = synth.preset("ragged_13x7x37")
    A = dense_A(P)
    B = np.zeros_like(A)
    for i in range(P.I):
        lo, hi = P.csr_rowptr[i], P.csr_rowptr[i + 1]
        assert np.all(np.diff(P.csr_col[lo:hi]) > 0)
        B[i, P.csr_col[lo:hi]] = P.csr_val[lo:hi]
    assert np.array_equal(A, B)
    assert np.all(np.diff(P.csc_colptr) == 50)
    assert P.csc_val.min() >= 0.1 and P.csc_val.max() <= 1.0
    assert np.all(P.y == np.round(P.y)) and P.y.min() >= 0


def test_generator_is_seeded():
    a = synth.preset("ragged_13x7x37")
    b = synth.preset("ragged_13x7x37")
    assert np.array_equal(a.csr_val, b.csr_val) and np.array_equal(a.y, b.y)
    c = synth.preset("ragged_13x7x37", seed=6)
    assert not np.array_equal(a.y, c.y)


# ----------------------------------------------------------------------------------------
# O1, O2: sparse products

@pytest.mark.parametrize("name", ["ragged_13x7x37", "tiny_16x16x32"])
def test_products_match_dense_and_adjoint(name):
    P = synth.preset(name)
    op = O.from_problem(P)
    A = dense_A(P)
    rng = np.random.default_rng(11)
    x = rng.random(P.J)
    v = rng.random(P.I)
    ybar, ratio = O.forward(op, x)
    Ax = A @ x
    r = float(P.b[0])
    np.testing.assert_allclose(ybar, Ax + r, rtol=1e-13)
    np.testing.assert_allclose(ratio, P.y / (Ax + r), rtol=1e-13)
    Atv = O.backproject(op, v)
    np.testing.assert_allclose(Atv, A.T @ v, rtol=1e-13)
    # adjoint identity <A x, v> = <x, A^T v>, CSR against CSC
    lhs = np.dot(ybar - r, v)
    rhs = np.dot(x, Atv)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    np.testing.assert_allclose(op.s, A.sum(axis=0), rtol=1e-13)


def test_ratio_zero_counts():
    P = tiny_problem()
    P.y[:5] = 0
    op = O.from_problem(P)
    _, ratio = O.forward(op, np.ones(P.J))
    assert np.all(ratio[:5] == 0)


# ----------------------------------------------------------------------------------------
# O4, O5: the separable surrogate and its minimiser

def test_alpha_closed_forms_golden():
    rows = np.loadtxt(os.path.join(GOLDEN, "alpha_closed_forms.txt"))
    Nx, Nz, Nq = 5, 4, 3
    for n_dirs in (4, 2):
        op = O.OracleProblem(Nx=Nx, Nz=Nz, Nq=Nq, I=1, J=Nx * Nz * Nq, rowptr=None, col=None,
                             rval=None, colptr=None, row=None, cval=None, y=None, r=None,
                             beta=1.0, rho=1.7, w=np.ones(n_dirs), n_dirs=n_dirs)
        rng = np.random.default_rng(1)
        alpha, _ = O.surrogate_coeffs(op, rng.random(op.J), rng.standard_normal(n_dirs * op.J))
        for nd, x, z, a in rows:
            if int(nd) != n_dirs:
                continue
            for q in range(Nq):
                j = (int(x) * Nz + int(z)) * Nq + q
                assert alpha[j] == pytest.approx(1.7 * a, rel=1e-14), (n_dirs, x, z)


@pytest.mark.parametrize("n_dirs,w", [(4, [1.0, 1.0, 1.0, 1.0]), (4, [0.5, 1.3, 2.0, 0.7]),
                                      (2, [1.0, 1.0]), (2, [0.4, 1.9])])
def test_surrogate_majorises_and_is_tangent(n_dirs, w):
    P = tiny_problem()
    w = np.array(w)
    op = O.from_problem(P, n_dirs=n_dirs, w=w, rho=2.5)
    A = dense_A(P)
    WG = dense_WG(P.Nx, P.Nz, P.Nq, n_dirs, w)
    r = float(P.b[0])
    y = P.y.astype(np.float64)
    rng = np.random.default_rng(5)
    f = rng.uniform(0.2, 2.0, P.J)
    u = rng.standard_normal(n_dirs * P.J)

    def psi(t):  # Eq. 5's objective with L the Poisson NLL (Eq. 1), dense
        yb = A @ t + r
        return (yb - y * np.log(yb)).sum() + 0.5 * op.rho * np.sum((u - WG @ t) ** 2)

    def grad_psi(t):
        yb = A @ t + r
        return A.sum(0) - A.T @ (y / yb) - op.rho * WG.T @ (u - WG @ t)

    alpha, gamma = O.surrogate_coeffs(op, f, u)
    e = A.T @ (y / (A @ f + r))
    E = f * e
    s = A.sum(0)

    def q(t):
        return np.sum(s * t - E * np.log(t) + alpha * t * t - gamma * t)

    # tangency: equal gradients at f
    gq = s - E / f + 2 * alpha * f - gamma
    np.testing.assert_allclose(gq, grad_psi(f), rtol=1e-10, atol=1e-10 * np.abs(gq).max())
    # majorisation: q(t) - q(f) >= psi(t) - psi(f) for t > 0
    for scale in (1e-3, 0.1, 0.5, 2.0):
        for _ in range(20):
            t = f * np.exp(scale * rng.standard_normal(P.J))
            lhs = q(t) - q(f)
            rhs = psi(t) - psi(f)
            assert lhs >= rhs - 1e-9 * (abs(lhs) + abs(rhs) + 1.0)


def test_root_minimises_1d_surrogate():
    from scipy.optimize import minimize_scalar

    rng = np.random.default_rng(7)
    cases = []
    for _ in range(300):
        alpha = rng.uniform(0.1, 10)
        s = rng.uniform(0.1, 10)
        E = rng.choice([0.0, rng.uniform(1e-6, 1e-3), rng.uniform(0.1, 100)])
        gamma = rng.uniform(-50, 50)
        cases.append((alpha, s, E, gamma))
    for alpha, s, E, gamma in cases:
        B = s - gamma
        t = O.root(alpha, B, E, s)
        assert t >= 0
        phi = lambda x: s * x - (E * np.log(x) if E > 0 else 0.0) + alpha * x * x - gamma * x
        if E > 0:
            # first-order condition of the 1-D surrogate at the root
            g = s - E / t + 2 * alpha * t - gamma
            assert abs(g) <= 1e-9 * (s + E / t + 2 * alpha * t + abs(gamma))
        else:
            assert t == pytest.approx(max(gamma - s, 0.0) / (2 * alpha), rel=1e-14, abs=1e-300)
        hi = 10 * (t + 1.0)
        res = minimize_scalar(phi, bounds=(1e-300 if E > 0 else 0.0, hi), method="bounded",
                              options={"xatol": 1e-12})
        assert phi(t) <= phi(res.x) + 1e-12 * (1 + abs(phi(t)))
    # rho = 0: the EM (MLEM) step E / s
    assert O.root(0.0, 3.0, 6.0, 3.0) == 2.0


def test_subproblem_decreases_monotonically():
    P = tiny_problem()
    op = O.from_problem(P, rho=1.5)
    A = dense_A(P)
    WG = dense_WG(P.Nx, P.Nz, P.Nq, 4, np.ones(4))
    r = float(P.b[0])
    y = P.y.astype(np.float64)
    rng = np.random.default_rng(2)
    u = rng.standard_normal(4 * P.J)
    f = rng.uniform(0.5, 1.5, P.J)

    def psi(t):
        yb = A @ t + r
        return (yb - y * np.log(yb)).sum() + 0.5 * op.rho * np.sum((u - WG @ t) ** 2)

    prev = psi(f)
    for _ in range(50):
        _, ratio = O.forward(op, f)
        e = O.backproject(op, ratio)
        alpha, gamma = O.surrogate_coeffs(op, f, u)
        f = O.f_update(op, f, e, alpha, gamma)
        cur = psi(f)
        assert cur <= prev + 1e-12 * abs(prev)
        prev = cur


def test_rho_zero_is_one_mlem_step_and_preserves_counts():
    P = tiny_problem()
    P.b[:] = 0.0  # r = 0: MLEM preserves total counts
    op = O.from_problem(P, rho=0.0)
    A = dense_A(P)
    y = P.y.astype(np.float64)
    f0 = np.random.default_rng(4).uniform(0.5, 2.0, P.J)
    f1, d1, c1 = O.iterate(op, (f0, np.zeros(4 * P.J), np.zeros(4 * P.J)), 1)
    mlem = f0 * (A.T @ (y / (A @ f0))) / A.sum(0)
    np.testing.assert_allclose(f1, mlem, rtol=1e-13)
    assert np.dot(A.sum(0), f1) == pytest.approx(y.sum(), rel=1e-12)


# ----------------------------------------------------------------------------------------
# O6, O7: group shrinkage and the dual update

def test_wgrad_and_adjoint_match_dense():
    P = tiny_problem()
    for n_dirs, w in ((4, np.array([0.5, 1.3, 2.0, 0.7])), (2, np.array([0.4, 1.9]))):
        op = O.from_problem(P, n_dirs=n_dirs, w=w)
        WG = dense_WG(P.Nx, P.Nz, P.Nq, n_dirs, w)
        rng = np.random.default_rng(8)
        f = rng.random(P.J)
        z = rng.standard_normal(n_dirs * P.J)
        np.testing.assert_allclose(O.wgrad(op, f), WG @ f, rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(O.wgrad_adjoint(op, z), WG.T @ z, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("n_dirs,w,rho", [(4, [0.5, 1.3, 2.0, 0.7], 1.0), (2, [0.4, 1.9], 2.5)])
def test_residuals_match_dense(n_dirs, w, rho):
    """primal, dual and KKT residuals of an arbitrary state, written with the
    dense A and w.G (Eq. 4's constraint d = w.G f, dual r = rho (w.G)^T
    (d - d_prev), stationarity of Eq. 4 with the dual estimate rho c)."""
    P = tiny_problem()
    w = np.array(w)
    op = O.from_problem(P, n_dirs=n_dirs, w=w, rho=rho)
    A = dense_A(P)
    WG = dense_WG(P.Nx, P.Nz, P.Nq, n_dirs, w)
    rng = np.random.default_rng(31)
    f = rng.random(P.J) * 2.0
    f[rng.random(P.J) < 0.2] = 0.0
    d = rng.standard_normal(n_dirs * P.J)
    d_prev = d + 0.1 * rng.standard_normal(n_dirs * P.J)
    c = rng.standard_normal(n_dirs * P.J)
    primal, dual, kkt = O.residuals(op, f, d, c, d_prev)
    assert primal == pytest.approx(np.linalg.norm(WG @ f - d) / max(1.0, np.linalg.norm(d)), rel=1e-12)
    assert dual == pytest.approx(rho * np.linalg.norm(WG.T @ (d - d_prev))
                                 / max(1.0, rho * np.linalg.norm(WG.T @ c)), rel=1e-12)
    s = A.sum(0)
    g = s - A.T @ (P.y / (A @ f + float(P.b[0]))) + rho * WG.T @ c
    assert kkt == pytest.approx(np.abs(np.minimum(f, g)).max() / max(1.0, s.max()), rel=1e-12)
    assert O.residuals(op, f, d, c)[1] == 0.0
    # one iteration moves d: its dual residual is the change of Eq. 6's output
    f1, d1, c1 = O.iterate(op, (f, d, c), 1)
    assert O.residuals(op, f1, d1, c1, d)[1] == pytest.approx(
        rho * np.linalg.norm(WG.T @ (d1 - d)) / max(1.0, rho * np.linalg.norm(WG.T @ c1)), rel=1e-12)


@pytest.mark.parametrize("n_dirs", [4, 2])
def test_shrink_is_group_prox(n_dirs):
    P = tiny_problem()
    op = O.from_problem(P, n_dirs=n_dirs, beta=3.0, rho=2.0)
    tau = op.beta / op.rho
    WG = dense_WG(P.Nx, P.Nz, P.Nq, n_dirs, np.ones(n_dirs))
    rng = np.random.default_rng(9)
    f = rng.random(P.J)
    site_scale = rng.uniform(0.0, 0.8, P.Nx * P.Nz)
    c = (rng.standard_normal((n_dirs, P.Nx * P.Nz, P.Nq)) * site_scale[None, :, None]).ravel()
    f = 0.2 * f
    d, c_new = O.shrink_dual(op, f, np.zeros_like(c), c)
    v = WG @ f + c
    S = P.Nx * P.Nz
    V = v.reshape(n_dirs, S, P.Nq)
    D = d.reshape(n_dirs, S, P.Nq)
    np.testing.assert_allclose(c_new, v - d, rtol=1e-15, atol=1e-15)
    n_shrunk = 0
    for s_ in range(S):
        vs, ds = V[:, s_, :].ravel(), D[:, s_, :].ravel()
        nd = np.linalg.norm(ds)
        if nd > 0:  # v - d = tau d / ||d||
            np.testing.assert_allclose(vs - ds, tau * ds / nd, rtol=1e-12, atol=1e-14)
        else:
            assert np.linalg.norm(vs) <= tau * (1 + 1e-14)
            n_shrunk += 1
    assert 0 < n_shrunk < S  # both branches exercised
    # rho c^{k+1} lies in beta * subdifferential of ||d_s|| (Eq. 6 optimality)
    C = c_new.reshape(n_dirs, S, P.Nq)
    for s_ in range(S):
        assert np.linalg.norm(op.rho * C[:, s_, :]) <= op.beta * (1 + 1e-12)


@pytest.mark.parametrize("n_dirs", [4, 2])
def test_dual_rule_is_shrink_fixed_point(n_dirs):
    # Eqs. 6-7 at a fixed point: d = w.G f and v = d + c must shrink back to
    # d, which for d_s != 0 means c_s = tau d_s / |d_s| (|c_s| = tau, parallel
    # to d_s); a zero group keeps c_s = 0. Checked against the dense w.G and a
    # hand-written group prox, not the oracle's shrink.
    P = tiny_problem()
    op = O.from_problem(P, n_dirs=n_dirs, beta=3.0, rho=2.0)
    tau = op.beta / op.rho
    S = P.Nx * P.Nz
    WG = dense_WG(P.Nx, P.Nz, P.Nq, n_dirs, np.ones(n_dirs))
    rng = np.random.default_rng(21)
    f = rng.random(P.J)
    d = WG @ f
    D = d.reshape(n_dirs, S, P.Nq).copy()
    D[:, 3, :] = 0.0  # one group with d_s = 0
    d = D.ravel()
    c = O.dual_rule(op, d, 1.0)
    C = c.reshape(n_dirs, S, P.Nq)
    for s_ in range(S):
        ds, cs = D[:, s_, :].ravel(), C[:, s_, :].ravel()
        nd = np.linalg.norm(ds)
        if nd == 0:
            assert not cs.any()
            continue
        assert abs(np.linalg.norm(cs) - tau) <= 1e-13 * tau
        assert abs(cs @ ds - tau * nd) <= 1e-12 * tau * nd
        v = ds + cs
        nv = np.linalg.norm(v)
        prox = max(0.0, 1.0 - tau / nv) * v  # group soft-threshold, written out
        np.testing.assert_allclose(prox, ds, rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(v - prox, cs, rtol=1e-12, atol=1e-14)
    # theta scales linearly; theta = 0 is the flat-start rule c = 0
    np.testing.assert_allclose(O.dual_rule(op, d, 0.25), 0.25 * c, rtol=1e-15, atol=0)
    assert not O.dual_rule(op, d, 0.0).any()
    # hand case: one site, Nq = 1, n_dirs = 2, d = (3, 4) -> c = tau (0.6, 0.8)
    one = O.OracleProblem(Nx=1, Nz=1, Nq=1, I=1, J=1, rowptr=None, col=None, rval=None, colptr=None, row=None,
                          cval=None, y=None, r=None, beta=1.5, rho=0.5, w=np.ones(2), n_dirs=2)
    np.testing.assert_allclose(O.dual_rule(one, np.array([3.0, 4.0])), [1.8, 2.4], rtol=1e-15)


def test_shrink_matches_bruteforce_convex_solve():
    from scipy.optimize import minimize

    rng = np.random.default_rng(10)
    # Nx=Nz=1: one site, Nq bins, the group is the Nq*n_dirs vector v = ghost diffs + c
    for Nq in (1, 2, 3, 4):
        for n_dirs in (2, 4):
            op = O.OracleProblem(Nx=1, Nz=1, Nq=Nq, I=1, J=Nq, rowptr=None, col=None, rval=None,
                                 colptr=None, row=None, cval=None, y=None, r=None, beta=1.3,
                                 rho=1.0, w=np.ones(n_dirs), n_dirs=n_dirs)
            for _ in range(3):
                f = rng.standard_normal(Nq)
                c = rng.standard_normal(n_dirs * Nq)
                d, _ = O.shrink_dual(op, f, np.zeros_like(c), c)
                v = np.tile(f, n_dirs) + c  # every neighbour is a ghost
                tau = op.beta / op.rho
                obj = lambda x: tau * np.sqrt(np.sum(x * x) + 1e-300) + 0.5 * np.sum((x - v) ** 2)
                best = None
                for start in (v, np.zeros_like(v) + 1e-3, rng.standard_normal(v.size)):
                    res = minimize(obj, start, method="Nelder-Mead",
                                   options={"xatol": 1e-10, "fatol": 1e-14, "maxiter": 40000,
                                            "maxfev": 40000})
                    if best is None or res.fun < best.fun:
                        best = res
                assert obj(d) <= best.fun + 1e-9
                np.testing.assert_allclose(d, best.x, atol=1e-4)


def test_shrink_reduces_to_textbook_isotropic_tv():
    # Q = 1 and forward differences (+x, +z): the group of site s is the 2-vector
    # (D_x f, D_z f) + c and Eq. 6 is the isotropic-TV vector shrinkage
    # d = v * max(||v|| - tau, 0) / ||v||.
    Nx, Nz = 6, 5
    op = O.OracleProblem(Nx=Nx, Nz=Nz, Nq=1, I=1, J=Nx * Nz, rowptr=None, col=None, rval=None,
                         colptr=None, row=None, cval=None, y=None, r=None, beta=0.7, rho=1.0,
                         w=np.ones(2), n_dirs=2)
    rng = np.random.default_rng(12)
    f = rng.random(Nx * Nz)
    c = 0.3 * rng.standard_normal(2 * Nx * Nz)
    d, _ = O.shrink_dual(op, f, np.zeros_like(c), c)
    F = f.reshape(Nx, Nz)
    Fx = np.zeros_like(F)
    Fz = np.zeros_like(F)
    Fx[:-1] = F[:-1] - F[1:]
    Fx[-1] = F[-1]
    Fz[:, :-1] = F[:, :-1] - F[:, 1:]
    Fz[:, -1] = F[:, -1]
    vx = Fx.ravel() + c[:Nx * Nz]
    vz = Fz.ravel() + c[Nx * Nz:]
    n = np.hypot(vx, vz)
    k = np.maximum(n - 0.7, 0) / n
    np.testing.assert_allclose(d[:Nx * Nz], vx * k, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(d[Nx * Nz:], vz * k, rtol=1e-13, atol=1e-15)


# ----------------------------------------------------------------------------------------
# O8 objective and the whole iteration

def test_objective_matches_dense():
    P = tiny_problem()
    op = O.from_problem(P, beta=2.0)
    A = dense_A(P)
    WG = dense_WG(P.Nx, P.Nz, P.Nq, 4, np.ones(4))
    f = np.random.default_rng(13).random(P.J)
    yb = A @ f + float(P.b[0])
    y = P.y.astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        dev = np.sum(yb - y + np.where(y > 0, y * np.log(y / yb), 0.0))
    tv = np.sum(group_norms(WG @ f, 4, P.Nx * P.Nz, P.Nq))
    phi, d_, t_ = O.objective(op, f)
    assert d_ == pytest.approx(dev, rel=1e-13) and d_ >= 0
    assert t_ == pytest.approx(tv, rel=1e-13)
    assert phi == pytest.approx(dev + 2.0 * tv, rel=1e-13)
    assert O.nll(op, f) == pytest.approx(np.sum(yb - y * np.log(yb)), rel=1e-13)


def kkt_certificate(P, f, c, beta, rho, n_dirs, w):
    """Optimality of f for min L(f) + beta R(w.G f), f >= 0 (Eq. 4), from the
    dual estimate p = rho c / beta, written with dense matrices:
      ||p_s|| <= 1, p_s = g_s / ||g_s|| where g = w.G f is nonzero,
      grad = grad L(f) + beta (w.G)^T p >= 0 and f * grad = 0."""
    A = dense_A(P)
    WG = dense_WG(P.Nx, P.Nz, P.Nq, n_dirs, w)
    y = P.y.astype(np.float64)
    S = P.Nx * P.Nz
    yb = A @ f + float(P.b[0])
    p = rho * c / beta
    g = WG @ f
    pn = group_norms(p, n_dirs, S, P.Nq)
    gn = group_norms(g, n_dirs, S, P.Nq)
    Pm = p.reshape(n_dirs, S, P.Nq)
    Gm = g.reshape(n_dirs, S, P.Nq)
    align = 0.0
    for s_ in range(S):
        if gn[s_] > 1e-7 * max(1.0, gn.max()):
            align = max(align, np.abs(Pm[:, s_] - Gm[:, s_] / gn[s_]).max())
    grad = A.sum(0) - A.T @ (y / yb) + beta * WG.T @ p
    comp = np.abs(np.minimum(f, grad)).max() / max(1.0, A.sum(0).max())
    return pn.max(), align, comp


@pytest.mark.parametrize("n_dirs,w", [(4, [1.0, 1.0, 1.0, 1.0]), (2, [1.0, 0.6]),
                                      (4, [0.8, 0.8, 1.2, 1.2])])
def test_converged_iterate_is_optimal(n_dirs, w):
    P = tiny_problem()
    w = np.array(w)
    op = O.from_problem(P, n_dirs=n_dirs, w=w)
    f0, d0, c0 = O.solve(op, 19999)
    f, d, c = O.iterate(op, (f0, d0, c0), 1)
    pmax, align, comp = kkt_certificate(P, f, c, op.beta, op.rho, n_dirs, w)
    assert pmax <= 1 + 1e-9
    assert align <= 1e-6
    assert comp <= 1e-8
    primal, dual, kkt = O.residuals(op, f, d, c, d0)
    assert primal < 1e-8 and dual < 1e-8 and kkt < 1e-8
    # no feasible perturbation does better (convex problem: KKT => optimal)
    phi0 = O.objective(op, f)[0]
    rng = np.random.default_rng(14)
    for _ in range(50):
        t = np.maximum(f + 1e-3 * rng.standard_normal(P.J) * (f.mean() + f), 0.0)
        assert O.objective(op, t)[0] >= phi0 - 1e-9 * phi0


def test_beta_zero_reaches_ml_fixed_point():
    P = tiny_problem(Nx=3, Nz=3, Nq=4, I=60, nnz_col=12, seed=21)
    op = O.from_problem(P, beta=0.0)
    f, d, c = O.solve(op, 20000)
    A = dense_A(P)
    y = P.y.astype(np.float64)
    e = A.T @ (y / (A @ f + float(P.b[0])))
    s = A.sum(0)
    # ML KKT: f_j (s_j - e_j) = 0 and s_j - e_j >= 0 where f_j = 0
    assert np.abs(f * (s - e)).max() <= 1e-6 * s.max() * max(1.0, f.max())
    assert (s - e).min() >= -1e-6 * s.max()
    assert np.abs(c).max() == 0.0


def test_relative_gap_is_never_negative():
    P = tiny_problem()
    op = O.from_problem(P)
    f_star, _, _ = O.solve(op, 20000)
    phi_star = O.objective(op, f_star)[0]
    st = O.init_state(op)
    for k in range(200):
        st = O.iterate(op, st, 1)
        assert st[0].min() >= 0
        phi = O.objective(op, st[0])[0]
        assert (phi - phi_star) / phi_star >= -1e-12


def test_init_state():
    P = tiny_problem()
    op = O.from_problem(P)
    f, d, c = O.init_state(op)
    A = dense_A(P)
    kappa = (P.y.astype(np.float64).sum() - P.I * float(P.b[0])) / A.sum()
    np.testing.assert_allclose(f, kappa, rtol=1e-13)
    WG = dense_WG(P.Nx, P.Nz, P.Nq, 4, np.ones(4))
    np.testing.assert_allclose(d, WG @ f, rtol=1e-13, atol=1e-15)
    assert not c.any()


# ----------------------------------------------------------------------------------------
# standard (per-bin) isotropic TV, the paper's comparison regulariser: the sum
# over q sits outside the square root, so every (s, q) is its own group

def bin_norms(g, n_dirs, S, Nq):
    return np.sqrt((g.reshape(n_dirs, S, Nq) ** 2).sum(axis=0))


@pytest.mark.parametrize("n_dirs", [4, 2])
def test_standard_tv_shrink_is_per_bin_prox(n_dirs):
    P = tiny_problem()
    op = O.from_problem(P, n_dirs=n_dirs, beta=3.0, rho=2.0, per_bin=True)
    tau = op.beta / op.rho
    S = P.Nx * P.Nz
    WG = dense_WG(P.Nx, P.Nz, P.Nq, n_dirs, np.ones(n_dirs))
    rng = np.random.default_rng(31)
    f = 0.2 * rng.random(P.J)
    c = rng.standard_normal(n_dirs * P.J) * rng.uniform(0.0, 0.9, P.J)[None, :].repeat(n_dirs, 0).ravel()
    d, c_new = O.shrink_dual(op, f, np.zeros_like(c), c)
    V = (WG @ f + c).reshape(n_dirs, P.J)
    D = d.reshape(n_dirs, P.J)
    n_zero = 0
    for j in range(P.J):
        v = V[:, j]
        nv = np.linalg.norm(v)
        prox = max(0.0, 1.0 - tau / nv) * v if nv > 0 else 0.0 * v  # written out per (s, q)
        np.testing.assert_allclose(D[:, j], prox, rtol=1e-13, atol=1e-15)
        n_zero += not D[:, j].any()
    assert 0 < n_zero < P.J  # both branches
    np.testing.assert_allclose(c_new, (V - D).ravel(), rtol=1e-15, atol=1e-15)
    assert np.all(bin_norms(op.rho * c_new, n_dirs, S, P.Nq) <= op.beta * (1 + 1e-12))


def test_standard_tv_value_and_decomposition_by_bin():
    # R is the dense per-(s, q) formula, and both R and the shrink split into
    # one-bin problems (Nq = 1, where groups per s and per (s, q) coincide)
    P = tiny_problem()
    op = O.from_problem(P, beta=2.0, rho=1.5, per_bin=True)
    S = P.Nx * P.Nz
    WG = dense_WG(P.Nx, P.Nz, P.Nq, 4, np.ones(4))
    rng = np.random.default_rng(32)
    f = rng.random(P.J)
    c = 0.3 * rng.standard_normal(4 * P.J)
    assert O.group_tv(op, WG @ f) == pytest.approx(np.sum(bin_norms(WG @ f, 4, S, P.Nq)), rel=1e-13)
    d, c_new = O.shrink_dual(op, f, np.zeros_like(c), c)
    one = O.OracleProblem(Nx=P.Nx, Nz=P.Nz, Nq=1, I=1, J=S, rowptr=None, col=None, rval=None, colptr=None,
                          row=None, cval=None, y=None, r=None, beta=op.beta, rho=op.rho, w=np.ones(4), n_dirs=4)
    F = f.reshape(S, P.Nq)
    Cq = c.reshape(4, S, P.Nq)
    D = d.reshape(4, S, P.Nq)
    Cn = c_new.reshape(4, S, P.Nq)
    for q in range(P.Nq):
        dq, cq = O.shrink_dual(one, F[:, q], np.zeros(4 * S), Cq[:, :, q].ravel())
        np.testing.assert_allclose(D[:, :, q].ravel(), dq, rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(Cn[:, :, q].ravel(), cq, rtol=1e-14, atol=1e-15)
    # and for one bin the two regularisers are the same iteration
    P1 = tiny_problem(Nq=1, I=30, nnz_col=8, seed=33)
    a = O.solve(O.from_problem(P1), 50)
    b = O.solve(O.from_problem(P1, per_bin=True), 50)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_standard_tv_converged_iterate_is_optimal():
    # KKT of min L(f) + beta sum_{s,q} ||(w.G f)_{s,q,.}|| over f >= 0, written
    # with dense matrices from p = rho c / beta: ||p_{s,q}|| <= 1, p aligned with
    # g = w.G f where g_{s,q} != 0, grad L + beta (w.G)^T p >= 0 complementary to f
    P = tiny_problem()
    op = O.from_problem(P, per_bin=True)
    f, d, c = O.solve(op, 20000)
    A = dense_A(P)
    WG = dense_WG(P.Nx, P.Nz, P.Nq, 4, np.ones(4))
    y = P.y.astype(np.float64)
    yb = A @ f + float(P.b[0])
    p = (op.rho * c / op.beta).reshape(4, P.J)
    g = (WG @ f).reshape(4, P.J)
    assert np.sqrt((p ** 2).sum(0)).max() <= 1 + 1e-9
    gn = np.sqrt((g ** 2).sum(0))
    big = gn > 1e-7 * max(1.0, gn.max())
    assert np.abs(p[:, big] - g[:, big] / gn[big]).max() <= 1e-6
    grad = A.sum(0) - A.T @ (y / yb) + op.beta * WG.T @ p.ravel()
    assert np.abs(np.minimum(f, grad)).max() / max(1.0, A.sum(0).max()) <= 1e-8
    # the two regularisers give different images on a multi-bin problem
    fg = O.solve(O.from_problem(P), 2000)[0]
    assert np.linalg.norm(fg - f) > 1e-3 * np.linalg.norm(f)


def test_dual_rule_standard_tv():
    P = tiny_problem()
    op = O.from_problem(P, beta=3.0, rho=2.0, per_bin=True)
    rng = np.random.default_rng(34)
    d = rng.standard_normal(4 * P.J)
    d.reshape(4, P.J)[:, 5] = 0.0
    c = O.dual_rule(op, d, 1.0).reshape(4, P.J)
    D = d.reshape(4, P.J)
    tau = 1.5
    for j in range(P.J):
        nd = np.linalg.norm(D[:, j])
        if nd == 0:
            assert not c[:, j].any()
        else:
            np.testing.assert_allclose(c[:, j], tau * D[:, j] / nd, rtol=1e-14)
