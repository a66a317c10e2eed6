"""The C ABI without a GPU: the library loads, exports every declared entry
point, and rejects bad arguments on the host before touching CUDA."""
import os
import re

import numpy as np
import pytest

from paper_1601_08201_gb300 import build as B
from paper_1601_08201_gb300 import sgtv, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return sgtv.load()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b((?:sgtv|wsnet)_[a-z0-9_]+)\s*\(", text))
    return names


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert {"sgtv_setup", "sgtv_iterate", "sgtv_objective", "sgtv_get_image"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(sgtv.exported_symbols()) <= names
    from paper_1601_08201_gb300 import wsnet
    assert set(wsnet.exported_symbols()) <= names


def test_strerror(lib):
    assert sgtv.strerror(0) == "SGTV_OK"
    assert sgtv.strerror(-2) == "SGTV_ERR_DOMAIN"


@pytest.fixture(scope="module")
def P():
    return synth.preset("ragged_13x7x37")


def call(P, **kw):
    a = dict(I=P.I, J=P.J, nnz=P.nnz, csr_rowptr=P.csr_rowptr, csr_col=P.csr_col, csr_val=P.csr_val,
             csc_colptr=P.csc_colptr, csc_row=P.csc_row, csc_val=P.csc_val, Nx=P.Nx, Nz=P.Nz, Nq=P.Nq,
             y=P.y, b=P.b, lam=P.beta, rho=P.rho, opts=None)
    a.update(kw)
    return sgtv.setup(**a)


def expect(code, P, match, **kw):
    with pytest.raises(sgtv.SgtvError) as ei:
        call(P, **kw)
    assert ei.value.code == code, str(ei.value)
    assert re.search(match, str(ei.value)), str(ei.value)


def test_rejects_bad_arguments_on_host(lib, P):
    ARG, DOM = -1, -2
    expect(ARG, P, "J != Nx", Nx=P.Nx + 1)
    expect(ARG, P, "I and J", I=0, csr_rowptr=np.zeros(1, np.int64), y=np.zeros(0, np.float32))
    expect(ARG, P, "n_dirs", opts=sgtv.make_opts(n_dirs=3))
    expect(ARG, P, "n_inner", opts=sgtv.make_opts(n_inner=0))
    expect(ARG, P, "flag", opts=sgtv.make_opts(flags=128))
    expect(ARG, P, "precision", opts=sgtv.make_opts(precision=7))
    expect(DOM, P, "rho", rho=0.0)
    expect(DOM, P, "rho", rho=float("nan"))
    expect(DOM, P, "lambda", lam=-1.0)
    expect(DOM, P, "weights", opts=sgtv.make_opts(w=[1, -1, 1, 1]))
    rp = P.csr_rowptr.copy()
    rp[5], rp[6] = rp[6], rp[5] - 1
    expect(DOM, P, "nondecreasing", csr_rowptr=rp)
    cp = P.csc_colptr.copy()
    cp[-1] -= 1
    expect(DOM, P, "nnz", csc_colptr=cp)
    y = P.y.copy()
    y[3] = -1
    expect(DOM, P, "y must", y=y)
    y[3] = np.nan
    expect(DOM, P, "y must", y=y)
    expect(DOM, P, "b must", b=np.array([-0.5], np.float32))
    expect(ARG, P, "b_len", b=np.ones(7, np.float32))


def test_empty_row_without_background_is_rejected(lib, P):
    # row 0 emptied in both copies, y_0 > 0 and r = 0: ybar_0 = 0 forever
    keep_r = np.ones(P.nnz, bool)
    keep_r[P.csr_rowptr[0]:P.csr_rowptr[1]] = False
    rp = P.csr_rowptr.copy()
    rp[1:] -= P.csr_rowptr[1] - P.csr_rowptr[0]
    y = P.y.copy()
    y[0] = 3
    cm = P.csc_row != 0
    cp = np.concatenate([[0], np.cumsum([cm[P.csc_colptr[j]:P.csc_colptr[j + 1]].sum()
                                         for j in range(P.J)])]).astype(np.int64)
    expect(-2, P, "empty row", nnz=int(keep_r.sum()), csr_rowptr=rp, csr_col=P.csr_col[keep_r],
           csr_val=P.csr_val[keep_r], csc_colptr=cp, csc_row=P.csc_row[cm], csc_val=P.csc_val[cm],
           y=y, b=np.zeros(1, np.float32))


def test_binding_type_checks(lib, P):
    with pytest.raises(TypeError):
        call(P, csr_val=P.csr_val.astype(np.float64))
    with pytest.raises(ValueError):
        call(P, y=P.y[:-1])
