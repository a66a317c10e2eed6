"""The batched form: several independent scans of uneven shape in one handle
(block-diagonal system), against the FP64 oracle run on each scan alone and
against separate one-scan handles."""
import numpy as np
import pytest

import oracle as O
from paper_1601_08201_gb300 import sgtv, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a, np.float64) - b) / (nb if nb > 0 else 1.0)


SHAPES = [(5, 4, 7, 90, 12, 20.0), (8, 3, 16, 300, 20, 60.0), (4, 4, 32, 500, 24, 8.0), (6, 7, 5, 160, 16, 35.0)]


@pytest.fixture(scope="module")
def scans():
    out = []
    for k, (Nx, Nz, Nq, I, nnz_col, counts) in enumerate(SHAPES):
        out.append(synth.make_problem(Nx, Nz, Nq, I, nnz_col, n_regions=2, mean_counts=counts, seed=40 + k,
                                      beta_frac=0.02 + 0.02 * k, rho=0.5 + 0.5 * k))
    return out


def split(h, arr, key="vox_off", ndirs=None):
    info = h.batch_info()
    off = info[key]
    if ndirs is None:
        return [arr[off[k]:off[k + 1]] for k in range(info["nscans"])]
    J = off[-1]
    return [np.concatenate([arr[p * J + off[k]:p * J + off[k + 1]] for p in range(ndirs)])
            for k in range(info["nscans"])]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_batch_matches_oracle_per_scan(scans, prec, tol):
    ops = [O.from_problem(P) for P in scans]
    sts = [O.init_state(op) for op in ops]
    with sgtv.Handle(scans, precision=prec) as h:
        done = 0
        for k_it in (1, 10, 100):
            h.iterate(k_it - done)
            sts = [O.iterate(op, st, k_it - done) for op, st in zip(ops, sts)]
            done = k_it
            f, d, c = h.get_state_f64()
            for k, (fk, dk, ck) in enumerate(zip(split(h, f), split(h, d, ndirs=4), split(h, c, ndirs=4))):
                assert rel(fk, sts[k][0]) <= tol, (prec, k_it, k, rel(fk, sts[k][0]))
                if prec == "fp64":
                    assert rel(dk, sts[k][1]) <= tol and rel(ck, sts[k][2]) <= tol
        for k, op in enumerate(ops):
            phi, dev, tv = h.objective_scan(k)
            ophi, odev, otv = O.objective(op, split(h, h.get_state_f64()[0])[k])
            assert phi == pytest.approx(ophi, rel=1e-10) and tv == pytest.approx(otv, rel=1e-10)
        phi_all = h.objective()[0]
        assert phi_all == pytest.approx(sum(h.objective_scan(k)[0] for k in range(len(scans))), rel=1e-12)


def test_batch_bit_identical_to_separate_handles(scans):
    flags = sgtv.FLAG_NO_AUTOTUNE
    with sgtv.Handle(scans, flags=flags) as h:
        h.iterate(20)
        fb = split(h, h.get_state_f64()[0])
    for k, P in enumerate(scans):
        with sgtv.Handle(P, flags=flags) as hk:
            hk.iterate(20)
            assert np.array_equal(hk.get_state_f64()[0], fb[k]), k


def test_batch_rejects_bad_scan(scans):
    bad = synth.make_problem(4, 4, 4, 40, 8, seed=9)
    bad.y = bad.y.copy()
    bad.y[0] = -1
    with pytest.raises(sgtv.SgtvError, match="scan 1"):
        sgtv.Handle([scans[0], bad])


def _pinned(h):
    names = h.variant_names()
    h.set_variants(names["k_forward"].index("tli_u8"), names["k_back_update"].index("tli_v4x2"))


@pytest.mark.parametrize("flags", [sgtv.FLAG_PERSISTENT, sgtv.FLAG_PERSISTENT | sgtv.FLAG_GRAPH, sgtv.FLAG_GRAPH])
def test_persistent_and_graph_modes_identical_to_launches(scans, flags):
    # 21 iterations: two 8-iteration graphs plus five direct iterations, then
    # 8 more from the other buffer order (a second graph)
    with sgtv.Handle(scans, flags=sgtv.FLAG_NO_AUTOTUNE) as h:
        _pinned(h)
        h.iterate(21)
        ref = h.get_state_f64()
    with sgtv.Handle(scans, flags=sgtv.FLAG_NO_AUTOTUNE | flags) as h:
        _pinned(h)
        h.profile(True)
        h.iterate(21)
        prof = h.profile_read()
        st = h.get_state_f64()
        h.iterate(8)  # graph of the other buffer order
        h.sync()
    for a, b in zip(st, ref):
        assert np.array_equal(a, b), flags
    if flags & sgtv.FLAG_PERSISTENT or flags & sgtv.FLAG_GRAPH:
        assert prof["k_iteration"][1] == (21 if flags & sgtv.FLAG_PERSISTENT else 16)


def test_persistent_fp64_matches_oracle(scans):
    ops = [O.from_problem(P) for P in scans]
    sts = [O.iterate(op, O.init_state(op), 30) for op in ops]
    with sgtv.Handle(scans, precision="fp64", flags=sgtv.FLAG_PERSISTENT | sgtv.FLAG_GRAPH) as h:
        h.iterate(30)
        f = h.get_state_f64()[0]
        for k in range(len(scans)):
            assert rel(split(h, f)[k], sts[k][0]) <= 1e-12


def test_persistent_autotune_and_single_scan():
    P = synth.preset("tiny_16x16x32")
    op = O.from_problem(P)
    ref = O.iterate(op, O.init_state(op), 40)
    with sgtv.Handle(P, flags=sgtv.FLAG_PERSISTENT | sgtv.FLAG_GRAPH) as h:
        names = h.variant_names()
        vf, vb = h.get_variants()
        assert names["k_forward"][vf] in ("tli_u8", "tli_v4x2")
        assert names["k_back_update"][vb] in ("tli_u8", "tli_v4x2")
        with pytest.raises(sgtv.SgtvError):
            h.set_variants(0, 0)  # a plain form cannot run fused
        h.iterate(40)
        assert rel(h.get_state_f64()[0], ref[0]) <= 1e-5


def test_wide_tile_range_uses_chunked_unique_lists():
    # 2M hyper-voxels, 64 measurements whose columns spread over the whole
    # image: a 64-row tile's index range exceeds one shared-memory bitmap, so
    # its unique-index list is built chunk by chunk.
    import scipy.sparse as sp
    Nx, Nz, Nq, I = 1000, 1000, 2, 64
    J = Nx * Nz * Nq
    rows, cols = [], []
    for i in range(I):
        c = np.unique((i * 31 + np.arange(32, dtype=np.int64) * 65537) % J)
        rows.append(np.full(c.size, i))
        cols.append(c)
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    vals = np.random.default_rng(5).uniform(0.1, 1.0, rows.size).astype(np.float32)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(I, J))
    A.sort_indices()
    C = A.tocsc()
    C.sort_indices()
    y = np.random.default_rng(6).poisson(A @ np.full(J, 0.01) + 1.0).astype(np.float32)
    P = synth.Problem(Nx=Nx, Nz=Nz, Nq=Nq, I=I, J=J, nnz=A.nnz, csc_colptr=C.indptr.astype(np.int64),
                      csc_row=C.indices.astype(np.int32), csc_val=C.data.astype(np.float32),
                      csr_rowptr=A.indptr.astype(np.int64), csr_col=A.indices.astype(np.int32),
                      csr_val=A.data.astype(np.float32), y=y, b=np.array([1.0], np.float32), beta=0.5, rho=1.0,
                      f_true=np.zeros(J, np.float32))
    op = O.from_problem(P)
    ref = O.iterate(op, O.init_state(op), 3)
    with sgtv.Handle(P, precision="fp64", flags=sgtv.FLAG_NO_AUTOTUNE) as h:
        assert h.tli_info()["csr"]["fmt"] == 1
        names = h.variant_names()
        h.set_variants(names["k_forward"].index("tli_u8"), names["k_back_update"].index("tli_u8"))
        h.iterate(3)
        f = h.get_state_f64()[0]
    assert rel(f, ref[0]) <= 1e-12
