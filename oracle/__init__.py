"""FP64 CPU oracle for spectrally grouped TV reconstruction with ADMM.

TEST INFRASTRUCTURE ONLY: the tests, the package's smoke check and the
benchmark's CPU-baseline leg are the only callers. The product path never
imports this package. The arithmetic lives in ``sgtv_oracle.c`` (plain C,
FP64, OpenMP over rows/columns/sites only); this module compiles it with gcc
on first use and marshals NumPy arrays to it.

Parity status per function (what pins it, see tests/test_oracle_pins.py):
  forward / backproject / sensitivity : adjoint identity, dense A product
  surrogate_coeffs / f_update         : majorisation + tangency against a
                                        dense restatement of Eq. 5's objective,
                                        1-D minimisation, MLEM special case
  shrink_dual                         : prox optimality, brute-force convex solve,
                                        textbook 2-D shrinkage special case
  iterate                             : beta = 0 ML fixed point, KKT residuals
                                        at convergence on tiny problems
  objective                           : deviance >= 0, dense restatement
  residuals (primal, dual, kkt)       : dense A and w.G restatement; all three
                                        below 1e-8 at a converged iterate
The iterate-by-iterate trajectory itself is fixed only by these invariants
(the paper prints no worked example): parity of the trajectory is unpinned
beyond them.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgtv_oracle.c")
_LIB = os.path.join(_HERE, "libsgtv_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
            lib.oracle_root.restype = dbl
            lib.oracle_root.argtypes = [dbl, dbl, dbl, dbl]
            lib.oracle_deviance.restype = dbl
            lib.oracle_nll.restype = dbl
            lib.oracle_group_tv.restype = dbl
            for name in ["oracle_forward", "oracle_backproject", "oracle_sensitivity",
                         "oracle_surrogate_coeffs", "oracle_f_update", "oracle_wgrad",
                         "oracle_wgrad_adjoint", "oracle_shrink_dual", "oracle_init",
                         "oracle_iterate"]:
                getattr(lib, name).restype = None
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclasses.dataclass
class OracleProblem:
    """FP64 copy of a problem (A values promoted exactly from their stored type)."""
    Nx: int
    Nz: int
    Nq: int
    I: int
    J: int
    rowptr: np.ndarray
    col: np.ndarray
    rval: np.ndarray
    colptr: np.ndarray
    row: np.ndarray
    cval: np.ndarray
    y: np.ndarray
    r: np.ndarray
    beta: float
    rho: float
    w: np.ndarray
    n_dirs: int
    s: np.ndarray = None
    per_bin: bool = False  # standard TV: one group per (s, q) instead of per s

    @property
    def S(self):
        return self.Nx * self.Nz


def from_problem(P, n_dirs: int = 4, w=None, csr_val=None, csc_val=None, beta=None,
                 rho=None, per_bin: bool = False) -> OracleProblem:
    """Build the FP64 oracle view of a synth.Problem. csr_val/csc_val override
    A's values (e.g. bf16-rounded copies); beta/rho override the weights."""
    if w is None:
        w = np.ones(n_dirs)
    op = OracleProblem(
        Nx=P.Nx, Nz=P.Nz, Nq=P.Nq, I=P.I, J=P.J,
        rowptr=np.ascontiguousarray(P.csr_rowptr, dtype=np.int64),
        col=np.ascontiguousarray(P.csr_col, dtype=np.int32),
        rval=_f64(P.csr_val if csr_val is None else csr_val),
        colptr=np.ascontiguousarray(P.csc_colptr, dtype=np.int64),
        row=np.ascontiguousarray(P.csc_row, dtype=np.int32),
        cval=_f64(P.csc_val if csc_val is None else csc_val),
        y=_f64(P.y), r=_f64(np.atleast_1d(P.b)),
        beta=float(P.beta if beta is None else beta),
        rho=float(P.rho if rho is None else rho),
        w=_f64(w), n_dirs=int(n_dirs), per_bin=bool(per_bin))
    op.s = sensitivity(op)
    return op


# ---- O1, O2: the two sparse products -------------------------------------------------

def forward(op: OracleProblem, f):
    """ybar = A f + r and ratio = y / ybar (Eq. 1)."""
    lib = _load()
    f = _f64(f)
    ybar = np.empty(op.I)
    ratio = np.empty(op.I)
    lib.oracle_forward(ctypes.c_int64(op.I), _p(op.rowptr), _p(op.col), _p(op.rval), _p(f),
                       _p(op.r), ctypes.c_int64(op.r.size), _p(op.y), _p(ybar), _p(ratio))
    return ybar, ratio


def backproject(op: OracleProblem, v):
    """A^T v through the CSC copy."""
    lib = _load()
    v = _f64(v)
    out = np.empty(op.J)
    lib.oracle_backproject(ctypes.c_int64(op.J), _p(op.colptr), _p(op.row), _p(op.cval),
                           _p(v), _p(out))
    return out


def sensitivity(op: OracleProblem):
    lib = _load()
    s = np.empty(op.J)
    lib.oracle_sensitivity(ctypes.c_int64(op.J), _p(op.colptr), _p(op.cval), _p(s))
    return s


# ---- O4, O5: the hyper-voxel update -------------------------------------------------

def surrogate_coeffs(op: OracleProblem, f, u):
    """alpha, gamma of De Pierro's separable majoriser of rho/2 ||u - w.G t||^2 at f."""
    lib = _load()
    f = _f64(f)
    u = _f64(u)
    alpha = np.empty(op.J)
    gamma = np.empty(op.J)
    lib.oracle_surrogate_coeffs(ctypes.c_int32(op.Nx), ctypes.c_int32(op.Nz),
                                ctypes.c_int32(op.Nq), ctypes.c_int(op.n_dirs), _p(op.w),
                                ctypes.c_double(op.rho), _p(f), _p(u), _p(alpha), _p(gamma))
    return alpha, gamma


def root(alpha, B, E, s):
    return _load().oracle_root(float(alpha), float(B), float(E), float(s))


def f_update(op: OracleProblem, f, e, alpha, gamma):
    lib = _load()
    f, e, alpha, gamma = _f64(f), _f64(e), _f64(alpha), _f64(gamma)
    out = np.empty(op.J)
    lib.oracle_f_update(ctypes.c_int64(op.J), _p(f), _p(e), _p(op.s), _p(alpha), _p(gamma),
                        _p(out))
    return out


# ---- O6, O7: group shrink and dual update ----------------------------------------------

def wgrad(op: OracleProblem, f):
    lib = _load()
    f = _f64(f)
    out = np.empty(op.n_dirs * op.J)
    lib.oracle_wgrad(ctypes.c_int32(op.Nx), ctypes.c_int32(op.Nz), ctypes.c_int32(op.Nq),
                     ctypes.c_int(op.n_dirs), _p(op.w), _p(f), _p(out))
    return out


def wgrad_adjoint(op: OracleProblem, z):
    lib = _load()
    z = _f64(z)
    out = np.empty(op.J)
    lib.oracle_wgrad_adjoint(ctypes.c_int32(op.Nx), ctypes.c_int32(op.Nz),
                             ctypes.c_int32(op.Nq), ctypes.c_int(op.n_dirs), _p(op.w),
                             _p(z), _p(out))
    return out


def shrink_dual(op: OracleProblem, f, d, c):
    """Returns the new (d, c) after Eqs. 6-7 (inputs are not modified)."""
    lib = _load()
    f = _f64(f)
    d = _f64(d).copy()
    c = _f64(c).copy()
    tau = op.beta / op.rho
    lib.oracle_shrink_dual(ctypes.c_int32(op.Nx), ctypes.c_int32(op.Nz),
                           ctypes.c_int32(op.Nq), ctypes.c_int(op.n_dirs), _p(op.w),
                           ctypes.c_double(tau), ctypes.c_int(int(op.per_bin)), _p(f), _p(d), _p(c))
    return d, c


def dual_rule(op: OracleProblem, d, theta: float = 1.0):
    """Scaled dual that the group shrink (Eq. 6) leaves in place at a fixed
    point of Eqs. 6-7: per group g (a spatial site s, or a pair (s, q) for the
    standard TV), c_g = theta * tau * d_g / |d_g|
    (tau = beta / rho), and c_g = 0 where d_g = 0. d and c are direction-major
    [p][J], j = site * Nq + q. Plain numpy; no blocking or reordering."""
    tau = op.beta / op.rho
    D = _f64(d).reshape(op.n_dirs, op.S, op.Nq)
    if op.per_bin:  # standard TV: groups (s, q)
        n = np.sqrt(np.sum(D * D, axis=0))
        k = np.zeros_like(n)
        nz = n > 0
        k[nz] = theta * tau / n[nz]
        return (D * k[None, :, :]).reshape(-1)
    n = np.sqrt(np.sum(D * D, axis=(0, 2)))
    k = np.zeros(op.S)
    nz = n > 0
    k[nz] = theta * tau / n[nz]
    return (D * k[None, :, None]).reshape(-1)


# ---- O8: objective and optimality measures -----------------------------------------------

def group_tv(op: OracleProblem, g):
    g = _f64(g)
    return _load().oracle_group_tv(ctypes.c_int32(op.Nx), ctypes.c_int32(op.Nz),
                                   ctypes.c_int32(op.Nq), ctypes.c_int(op.n_dirs),
                                   ctypes.c_int(int(op.per_bin)), _p(g))


def objective(op: OracleProblem, f):
    """(phi, deviance, tv): phi = D(f) + beta * R(w.G f)."""
    lib = _load()
    ybar, _ = forward(op, f)
    dev = lib.oracle_deviance(ctypes.c_int64(op.I), _p(ybar), _p(op.y))
    tv = group_tv(op, wgrad(op, f))
    return dev + op.beta * tv, dev, tv


def nll(op: OracleProblem, f):
    lib = _load()
    ybar, _ = forward(op, f)
    return lib.oracle_nll(ctypes.c_int64(op.I), _p(ybar), _p(op.y))


def residuals(op: OracleProblem, f, d, c, d_prev=None):
    """(primal, dual, kkt) of the ADMM state after an iteration (Sec. III,
    Eqs. 5-7, constraint d = w.G f of Eq. 4):
      primal = ||w.G f - d|| / max(1, ||d||)
      dual   = rho ||(w.G)^T (d - d_prev)|| / max(1, ||rho (w.G)^T c||),
               d_prev = the split variable before the iteration's Eq. 6 step
               (the change of d seen through the constraint's adjoint; 0 when
               d_prev is None)
      kkt    = ||min(f, g)||_inf / max(1, ||s||_inf), g = s - e(f) + rho (w.G)^T c."""
    f = _f64(f)
    d = _f64(d)
    c = _f64(c)
    g_f = wgrad(op, f)
    primal = np.linalg.norm(g_f - d) / max(1.0, np.linalg.norm(d))
    adj_c = op.rho * wgrad_adjoint(op, c)
    dual = 0.0
    if d_prev is not None:
        dual = (op.rho * np.linalg.norm(wgrad_adjoint(op, d - _f64(d_prev)))
                / max(1.0, np.linalg.norm(adj_c)))
    _, ratio = forward(op, f)
    e = backproject(op, ratio)
    g = op.s - e + adj_c
    kkt = np.max(np.abs(np.minimum(f, g))) / max(1.0, np.max(op.s))
    return primal, dual, kkt


# ---- O9 and the full iteration -----------------------------------------------------------

def init_state(op: OracleProblem):
    lib = _load()
    f = np.empty(op.J)
    d = np.empty(op.n_dirs * op.J)
    c = np.empty(op.n_dirs * op.J)
    lib.oracle_init(ctypes.c_int32(op.Nx), ctypes.c_int32(op.Nz), ctypes.c_int32(op.Nq),
                    ctypes.c_int(op.n_dirs), _p(op.w), ctypes.c_int64(op.I), _p(op.y),
                    _p(op.r), ctypes.c_int64(op.r.size), _p(op.s), _p(f), _p(d), _p(c))
    return f, d, c


def iterate(op: OracleProblem, state, n_iter: int, n_inner: int = 1):
    """Run n_iter ADMM iterations from state = (f, d, c); returns a new state."""
    lib = _load()
    f, d, c = (_f64(a).copy() for a in state)
    lib.oracle_iterate(ctypes.c_int32(op.Nx), ctypes.c_int32(op.Nz), ctypes.c_int32(op.Nq),
                       ctypes.c_int(op.n_dirs), _p(op.w), ctypes.c_int64(op.I),
                       _p(op.rowptr), _p(op.col), _p(op.rval), _p(op.colptr), _p(op.row),
                       _p(op.cval), _p(op.y), _p(op.r), ctypes.c_int64(op.r.size), _p(op.s),
                       ctypes.c_double(op.beta), ctypes.c_double(op.rho),
                       ctypes.c_int(n_iter), ctypes.c_int(n_inner), ctypes.c_int(int(op.per_bin)),
                       _p(f), _p(d), _p(c))
    return f, d, c


def solve(op: OracleProblem, n_iter: int, n_inner: int = 1):
    return iterate(op, init_state(op), n_iter, n_inner)
