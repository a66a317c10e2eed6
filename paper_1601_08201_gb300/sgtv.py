"""Thin ctypes binding of libsgtv.so (C ABI in include/sgtv.h).

Argument marshalling only: every step of the reconstruction runs in the CUDA
kernels of libsgtv.so. The module refuses to work without the compiled
library (there is no CPU fallback); build it with
``python -m paper_1601_08201_gb300.build`` or ``__graft_entry__.build()``.

Function names follow the C ABI: setup, iterate, sync, objective, residuals,
get_image, get_state_f64, set_state_f64, info, profile, profile_read,
get_stream, destroy, last_error, strerror. ``Handle`` wraps them as methods.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

SGTV_OK = 0
ERR = {-1: "SGTV_ERR_ARG", -2: "SGTV_ERR_DOMAIN", -3: "SGTV_ERR_CUDA", -4: "SGTV_ERR_OOM",
       -5: "SGTV_ERR_STATE", -6: "SGTV_ERR_TIMEOUT", -7: "SGTV_ERR_NONFINITE"}
PRECISION = {"fp32": 0, "bf16": 1, "fp64": 2}
FLAG_ALLOW_RHO0 = 1
FLAG_NO_AUTOTUNE = 2
FLAG_PERSISTENT = 4
FLAG_GRAPH = 8
FLAG_SINGLE_PASS = 16
FLAG_STANDARD_TV = 32
FLAG_SERIAL = 64
K_FORWARD, K_BACK_UPDATE, K_SHRINK, K_ITERATION, K_SCATTER, K_FUPDATE, K_COUNT = 0, 1, 2, 3, 4, 5, 6
KERNEL_NAMES = ("k_forward", "k_back_update", "k_shrink", "k_iteration", "k_scatter", "k_fupdate")


class SgtvError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR.get(code, code)}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("w", ctypes.c_double * 4), ("n_dirs", ctypes.c_int32), ("n_inner", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("alloc", ctypes.c_void_p), ("free_", ctypes.c_void_p), ("alloc_user", ctypes.c_void_p)]


class ScanDesc(ctypes.Structure):
    """sgtv_scan: one scan of a batch (host pointers, copied by the library)."""
    _fields_ = [("I", ctypes.c_int64), ("J", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("csr_rowptr", ctypes.c_void_p), ("csr_col", ctypes.c_void_p), ("csr_val", ctypes.c_void_p),
                ("csc_colptr", ctypes.c_void_p), ("csc_row", ctypes.c_void_p), ("csc_val", ctypes.c_void_p),
                ("Nx", ctypes.c_int32), ("Nz", ctypes.c_int32), ("Nq", ctypes.c_int32),
                ("y", ctypes.c_void_p), ("b", ctypes.c_void_p), ("b_len", ctypes.c_int64),
                ("lam", ctypes.c_double), ("rho", ctypes.c_double)]


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_D = ctypes.c_double


def load():
    """Load libsgtv.so; raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -m paper_1601_08201_gb300.build)")
        lib = ctypes.CDLL(LIB_PATH)
        sig = {
            "sgtv_default_opts": (None, [_P]),
            "sgtv_setup": (ctypes.c_int, [_P, _I64, _I64, _I64, _P, _P, _P, _P, _P, _P, _I32, _I32,
                                          _I32, _P, _P, _I64, _D, _D, _P]),
            "sgtv_setup_batch": (ctypes.c_int, [_P, _I32, _P, _P]),
            "sgtv_batch_info": (ctypes.c_int, [_P, _P, _P, _P, _P]),
            "sgtv_objective_scan": (ctypes.c_int, [_P, _I32, _P, _P, _P]),
            "sgtv_set_data": (ctypes.c_int, [_P, _P, _P, _I64, _D]),
            "sgtv_normalized_backprojection": (ctypes.c_int, [_P, _P, _I32]),
            "sgtv_warm_start": (ctypes.c_int, [_P, _P, _I32, ctypes.c_double]),
            "sgtv_warm_start_dual": (ctypes.c_int, [_P, _P, _P, _I32]),
            "sgtv_iterate": (ctypes.c_int, [_P, _I32]),
            "sgtv_sync": (ctypes.c_int, [_P]),
            "sgtv_objective": (ctypes.c_int, [_P, _P, _P, _P]),
            "sgtv_residuals": (ctypes.c_int, [_P, _P, _P, _P]),
            "sgtv_get_image": (ctypes.c_int, [_P, _P, _I64]),
            "sgtv_get_state_f64": (ctypes.c_int, [_P, _P, _P, _P]),
            "sgtv_set_state_f64": (ctypes.c_int, [_P, _P, _P, _P]),
            "sgtv_info": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
            "sgtv_profile": (ctypes.c_int, [_P, _I32]),
            "sgtv_profile_read": (ctypes.c_int, [_P, _P, _P, _I32]),
            "sgtv_get_stream": (ctypes.c_int, [_P, _P]),
            "sgtv_set_wait_limit": (ctypes.c_int, [_P, _I64]),
            "sgtv_set_serial": (ctypes.c_int, [_P, _I32]),
            "sgtv_destroy": (ctypes.c_int, [_P]),
            "sgtv_autotune": (ctypes.c_int, [_P, _I32]),
            "sgtv_get_variants": (ctypes.c_int, [_P, _P, _P]),
            "sgtv_set_variants": (ctypes.c_int, [_P, _I32, _I32]),
            "sgtv_get_variant": (ctypes.c_int, [_P, _I32, _P]),
            "sgtv_set_variant": (ctypes.c_int, [_P, _I32, _I32]),
            "sgtv_variant_count": (ctypes.c_int, [_P, _I32]),
            "sgtv_variant_name": (ctypes.c_char_p, [_P, _I32, _I32]),
            "sgtv_tli_info": (ctypes.c_int, [_P, _P, _P, _P, _P]),
            "sgtv_kkt_residual_noalloc": (ctypes.c_int, [_I64, _I64, _P, _P, _P, _P, _P, _P, _I32, _I32, _I32,
                                                         _I32, _P, _P, _P, _I64, _P, _P, _P, _D, _P, _P]),
            "sgtv_noalloc_last_error": (ctypes.c_char_p, []),
            "sgtv_last_error": (ctypes.c_char_p, [_P]),
            "sgtv_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def exported_symbols():
    """Names of every entry point the binding expects (all declared in sgtv.h)."""
    return ["sgtv_default_opts", "sgtv_setup", "sgtv_iterate", "sgtv_sync", "sgtv_objective",
            "sgtv_residuals", "sgtv_get_image", "sgtv_get_state_f64", "sgtv_set_state_f64",
            "sgtv_info", "sgtv_profile", "sgtv_profile_read", "sgtv_get_stream", "sgtv_destroy",
            "sgtv_last_error", "sgtv_strerror", "sgtv_autotune", "sgtv_get_variants",
            "sgtv_set_variants", "sgtv_variant_count", "sgtv_variant_name", "sgtv_tli_info",
            "sgtv_kkt_residual_noalloc", "sgtv_noalloc_last_error", "sgtv_setup_batch", "sgtv_batch_info",
            "sgtv_objective_scan", "sgtv_set_data", "sgtv_normalized_backprojection", "sgtv_warm_start",
            "sgtv_get_variant", "sgtv_set_variant", "sgtv_warm_start_dual", "sgtv_set_wait_limit",
            "sgtv_set_serial"]


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _host(a, dtype, n, name):
    a = np.asarray(a)
    if a.dtype != dtype:
        raise TypeError(f"{name} must be {np.dtype(dtype).name}, got {a.dtype}")
    if not a.flags.c_contiguous:
        raise ValueError(f"{name} must be C-contiguous")
    if n is not None and a.size != n:
        raise ValueError(f"{name} must have {n} elements, got {a.size}")
    return a


def last_error(h=None) -> str:
    return load().sgtv_last_error(h).decode()


def strerror(code: int) -> str:
    return load().sgtv_strerror(code).decode()


def _check(rc, h=None):
    if rc != SGTV_OK:
        raise SgtvError(rc, last_error(h))


def make_opts(n_dirs=4, w=None, n_inner=1, precision="fp32", flags=0, stream=None) -> Opts:
    o = Opts()
    load().sgtv_default_opts(ctypes.byref(o))
    o.n_dirs = n_dirs
    w = [1.0] * n_dirs if w is None else list(w)
    for p in range(4):
        o.w[p] = float(w[p]) if p < len(w) else 0.0
    o.n_inner = n_inner
    o.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    o.flags = flags
    o.stream = stream
    return o


def setup(I, J, nnz, csr_rowptr, csr_col, csr_val, csc_colptr, csc_row, csc_val, Nx, Nz, Nq, y, b,
          lam, rho, opts: Opts | None = None):
    """sgtv_setup with host NumPy arrays; returns the raw handle (c_void_p)."""
    lib = load()
    csr_rowptr = _host(csr_rowptr, np.int64, I + 1, "csr_rowptr")
    csr_col = _host(csr_col, np.int32, nnz, "csr_col")
    csr_val = _host(csr_val, np.float32, nnz, "csr_val")
    csc_colptr = _host(csc_colptr, np.int64, J + 1, "csc_colptr")
    csc_row = _host(csc_row, np.int32, nnz, "csc_row")
    csc_val = _host(csc_val, np.float32, nnz, "csc_val")
    y = _host(y, np.float32, I, "y")
    b = _host(np.atleast_1d(b), np.float32, None, "b")
    h = ctypes.c_void_p()
    rc = lib.sgtv_setup(ctypes.byref(h), I, J, nnz, _ptr(csr_rowptr), _ptr(csr_col), _ptr(csr_val),
                        _ptr(csc_colptr), _ptr(csc_row), _ptr(csc_val), Nx, Nz, Nq, _ptr(y), _ptr(b),
                        b.size, float(lam), float(rho), ctypes.byref(opts) if opts is not None else None)
    _check(rc, None)
    return h


def setup_batch(problems, opts: Opts | None = None, lams=None, rhos=None):
    """sgtv_setup_batch over a list of synth.Problem-like objects (host arrays)."""
    lib = load()
    n = len(problems)
    descs = (ScanDesc * n)()
    keep = []
    for k, P in enumerate(problems):
        arrs = dict(csr_rowptr=_host(P.csr_rowptr, np.int64, P.I + 1, "csr_rowptr"),
                    csr_col=_host(P.csr_col, np.int32, P.nnz, "csr_col"),
                    csr_val=_host(P.csr_val, np.float32, P.nnz, "csr_val"),
                    csc_colptr=_host(P.csc_colptr, np.int64, P.J + 1, "csc_colptr"),
                    csc_row=_host(P.csc_row, np.int32, P.nnz, "csc_row"),
                    csc_val=_host(P.csc_val, np.float32, P.nnz, "csc_val"),
                    y=_host(P.y, np.float32, P.I, "y"), b=_host(np.atleast_1d(P.b), np.float32, None, "b"))
        keep.append(arrs)
        dsc = descs[k]
        dsc.I, dsc.J, dsc.nnz = P.I, P.J, P.nnz
        for name, a in arrs.items():
            setattr(dsc, name, a.ctypes.data)
        dsc.Nx, dsc.Nz, dsc.Nq = P.Nx, P.Nz, P.Nq
        dsc.b_len = arrs["b"].size
        dsc.lam = float(P.beta if lams is None else lams[k])
        dsc.rho = float(P.rho if rhos is None else rhos[k])
    h = ctypes.c_void_p()
    rc = lib.sgtv_setup_batch(ctypes.byref(h), n, descs, ctypes.byref(opts) if opts is not None else None)
    _check(rc, None)
    return h


def batch_info(h):
    n = _I32()
    _check(load().sgtv_batch_info(h, ctypes.byref(n), None, None, None), h)
    vo = (ctypes.c_int64 * (n.value + 1))()
    mo = (ctypes.c_int64 * (n.value + 1))()
    so = (ctypes.c_int64 * (n.value + 1))()
    _check(load().sgtv_batch_info(h, None, vo, mo, so), h)
    return dict(nscans=n.value, vox_off=list(vo), meas_off=list(mo), site_off=list(so))


def objective_scan(h, k):
    phi, dev, tv = _D(), _D(), _D()
    _check(load().sgtv_objective_scan(h, int(k), ctypes.byref(phi), ctypes.byref(dev), ctypes.byref(tv)), h)
    return phi.value, dev.value, tv.value


def set_data(h, y, b, lam):
    J_I = info(h)
    y = _host(y, np.float32, J_I["I"], "y")
    b = _host(np.atleast_1d(b), np.float32, None, "b")
    _check(load().sgtv_set_data(h, _ptr(y), _ptr(b), b.size, float(lam)), h)


def normalized_backprojection(h, out=None):
    """A^T y / A^T 1: into a new host array, or into `out` (an int device address)."""
    if isinstance(out, int):
        _check(load().sgtv_normalized_backprojection(h, ctypes.c_void_p(out), 1), h)
        return None
    J = info(h)["J"]
    arr = np.empty(J, np.float32)
    _check(load().sgtv_normalized_backprojection(h, _ptr(arr), 0), h)
    return arr


def warm_start(h, f0, dual_scale: float = 0.0):
    """f0: a host float32 array of J values, or an int device address;
    dual_scale in [0, 1] scales the group-shrink-consistent dual (0: c = 0)."""
    if isinstance(f0, int):
        _check(load().sgtv_warm_start(h, ctypes.c_void_p(f0), 1, float(dual_scale)), h)
    else:
        a = _host(np.ascontiguousarray(f0, np.float32), np.float32, info(h)["J"], "f0")
        _check(load().sgtv_warm_start(h, _ptr(a), 0, float(dual_scale)), h)


def warm_start_dual(h, f0, c0):
    """f0 (J) and c0 (n_dirs * J): host float32 arrays, or int device addresses."""
    if isinstance(f0, int) and isinstance(c0, int):
        _check(load().sgtv_warm_start_dual(h, ctypes.c_void_p(f0), ctypes.c_void_p(c0), 1), h)
    else:
        nf = info(h)
        a = _host(np.ascontiguousarray(f0, np.float32), np.float32, nf["J"], "f0")
        b = _host(np.ascontiguousarray(c0, np.float32), np.float32, nf["J"] * nf["n_dirs"], "c0")
        _check(load().sgtv_warm_start_dual(h, _ptr(a), _ptr(b), 0), h)


def iterate(h, n: int):
    _check(load().sgtv_iterate(h, int(n)), h)


def sync(h):
    _check(load().sgtv_sync(h), h)


def objective(h):
    phi, dev, tv = _D(), _D(), _D()
    _check(load().sgtv_objective(h, ctypes.byref(phi), ctypes.byref(dev), ctypes.byref(tv)), h)
    return phi.value, dev.value, tv.value


def residuals(h):
    """(primal, dual, kkt) of the current state."""
    p, d, k = _D(), _D(), _D()
    _check(load().sgtv_residuals(h, ctypes.byref(p), ctypes.byref(d), ctypes.byref(k)), h)
    return p.value, d.value, k.value


def info(h):
    I, J, nnz, nd, prec, nbytes = _I64(), _I64(), _I64(), _I32(), _I32(), _I64()
    _check(load().sgtv_info(h, ctypes.byref(I), ctypes.byref(J), ctypes.byref(nnz), ctypes.byref(nd),
                            ctypes.byref(prec), ctypes.byref(nbytes)), h)
    return dict(I=I.value, J=J.value, nnz=nnz.value, n_dirs=nd.value, precision=prec.value,
                device_bytes=nbytes.value)


def get_image(h, out=None):
    J = info(h)["J"]
    out = np.empty(J, np.float32) if out is None else _host(out, np.float32, J, "out")
    _check(load().sgtv_get_image(h, _ptr(out), J), h)
    return out


def get_state_f64(h):
    inf = info(h)
    J, nd = inf["J"], inf["n_dirs"]
    f, d, c = np.empty(J), np.empty(nd * J), np.empty(nd * J)
    _check(load().sgtv_get_state_f64(h, _ptr(f), _ptr(d), _ptr(c)), h)
    return f, d, c


def set_state_f64(h, f, d=None, c=None):
    inf = info(h)
    J, nd = inf["J"], inf["n_dirs"]
    f = _host(np.ascontiguousarray(f, np.float64), np.float64, J, "f")
    if d is not None:
        d = _host(np.ascontiguousarray(d, np.float64), np.float64, nd * J, "d")
        c = _host(np.ascontiguousarray(c, np.float64), np.float64, nd * J, "c")
    _check(load().sgtv_set_state_f64(h, _ptr(f), _ptr(d), _ptr(c)), h)


def profile(h, enable: bool):
    _check(load().sgtv_profile(h, 1 if enable else 0), h)


def profile_read(h):
    ms = (ctypes.c_double * K_COUNT)()
    n = (ctypes.c_int64 * K_COUNT)()
    _check(load().sgtv_profile_read(h, ms, n, K_COUNT), h)
    return {KERNEL_NAMES[k]: (ms[k], n[k]) for k in range(K_COUNT)}


def autotune(h, reps: int = 3):
    _check(load().sgtv_autotune(h, int(reps)), h)
    return get_variants(h)


def get_variants(h):
    f, b = _I32(), _I32()
    _check(load().sgtv_get_variants(h, ctypes.byref(f), ctypes.byref(b)), h)
    return f.value, b.value


def set_variants(h, fwd: int, back: int):
    _check(load().sgtv_set_variants(h, int(fwd), int(back)), h)


def get_variant(h, kernel: int) -> int:
    v = _I32()
    _check(load().sgtv_get_variant(h, int(kernel), ctypes.byref(v)), h)
    return v.value


def set_variant(h, kernel: int, v: int):
    _check(load().sgtv_set_variant(h, int(kernel), int(v)), h)


def variant_names(h):
    lib = load()
    out = {}
    for k, name in ((K_FORWARD, "k_forward"), (K_BACK_UPDATE, "k_back_update"), (K_SCATTER, "k_scatter")):
        n = lib.sgtv_variant_count(h, k)
        out[name] = [lib.sgtv_variant_name(h, k, v).decode() for v in range(n)]
    return out


def tli_info(h):
    fmt = (ctypes.c_int32 * 2)()
    nl = (ctypes.c_int64 * 2)()
    nw = (ctypes.c_int64 * 2)()
    mx = (ctypes.c_int64 * 2)()
    _check(load().sgtv_tli_info(h, fmt, nl, nw, mx), h)
    return {name: dict(fmt=fmt[k], list_entries=nl[k], window_elems=nw[k], max_stage=mx[k])
            for k, name in enumerate(("csr", "csc"))}


def kkt_residual_noalloc(I, J, csr_rowptr, csr_col, csr_val, csc_colptr, csc_row, csc_val, Nx, Nz, Nq,
                         n_dirs, w, y, b, s, f, c, rho, out, stream=0):
    """sgtv_kkt_residual_noalloc: array arguments are device addresses (ints,
    e.g. torch_tensor.data_ptr()) except w (a sequence of n_dirs floats);
    out is the device address of 2 doubles. b is (address, length)."""
    wa = (ctypes.c_double * 4)(*([float(v) for v in w] + [0.0] * (4 - len(w))))
    b_ptr, b_len = b
    rc = load().sgtv_kkt_residual_noalloc(
        I, J, csr_rowptr, csr_col, csr_val, csc_colptr, csc_row, csc_val, Nx, Nz, Nq, n_dirs, wa, y, b_ptr,
        b_len, s, f, c, float(rho), out, stream)
    if rc != SGTV_OK:
        raise SgtvError(rc, load().sgtv_noalloc_last_error().decode())


def set_serial(h, on: bool):
    """Every kernel on the handle's stream (on) or the shrink overlapped on a
    second stream (off), for the iterations enqueued after the call."""
    _check(load().sgtv_set_serial(h, int(bool(on))), h)


def set_wait_limit(h, ns: int):
    """Bound (ns) on a block's wait in the persistent launch's grid barriers."""
    _check(load().sgtv_set_wait_limit(h, int(ns)), h)


def get_stream(h) -> int:
    s = ctypes.c_void_p()
    _check(load().sgtv_get_stream(h, ctypes.byref(s)), h)
    return s.value or 0


def destroy(h):
    if h:
        load().sgtv_destroy(h)


class Handle:
    """One reconstruction problem (or, given a list, a batch of independent
    scans) resident on the current CUDA device."""

    def __init__(self, problem, lam=None, rho=None, n_dirs=4, w=None, n_inner=1, precision="fp32",
                 flags=0, stream=None):
        opts = make_opts(n_dirs=n_dirs, w=w, n_inner=n_inner, precision=precision, flags=flags,
                         stream=stream)
        if isinstance(problem, (list, tuple)):
            self.h = setup_batch(problem, opts, lams=lam, rhos=rho)
            return
        P = problem
        self.h = setup(P.I, P.J, P.nnz, P.csr_rowptr, P.csr_col, P.csr_val, P.csc_colptr, P.csc_row,
                       P.csc_val, P.Nx, P.Nz, P.Nq, P.y, P.b, P.beta if lam is None else lam,
                       P.rho if rho is None else rho, opts)

    def batch_info(self):
        return batch_info(self.h)

    def set_data(self, y, b, lam):
        set_data(self.h, y, b, lam)

    def normalized_backprojection(self, out=None):
        return normalized_backprojection(self.h, out)

    def warm_start(self, f0, dual_scale=0.0):
        warm_start(self.h, f0, dual_scale)

    def warm_start_dual(self, f0, c0):
        warm_start_dual(self.h, f0, c0)

    def objective_scan(self, k):
        return objective_scan(self.h, k)

    def iterate(self, n):
        iterate(self.h, n)

    def sync(self):
        sync(self.h)

    def objective(self):
        return objective(self.h)

    def residuals(self):
        return residuals(self.h)

    def get_image(self):
        return get_image(self.h)

    def get_state_f64(self):
        return get_state_f64(self.h)

    def set_state_f64(self, f, d=None, c=None):
        set_state_f64(self.h, f, d, c)

    def info(self):
        return info(self.h)

    def profile(self, enable=True):
        profile(self.h, enable)

    def profile_read(self):
        return profile_read(self.h)

    def autotune(self, reps=3):
        return autotune(self.h, reps)

    def get_variants(self):
        return get_variants(self.h)

    def set_variants(self, fwd, back):
        set_variants(self.h, fwd, back)

    def variant_names(self):
        return variant_names(self.h)

    def get_variant(self, kernel):
        return get_variant(self.h, kernel)

    def set_variant(self, kernel, v):
        set_variant(self.h, kernel, v)

    def tli_info(self):
        return tli_info(self.h)

    def set_wait_limit(self, ns):
        set_wait_limit(self.h, ns)

    def set_serial(self, on):
        set_serial(self.h, on)

    @property
    def stream(self):
        return get_stream(self.h)

    def close(self):
        if self.h:
            destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
