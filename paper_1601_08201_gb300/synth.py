"""Seeded synthetic scatter-imaging problems (inputs only).

This module draws the inputs both the CUDA path and the CPU oracle consume:
a sparse nonnegative system matrix A (stored as CSC and CSR), a
piecewise-constant phantom whose momentum-transfer profiles (MTPs) are
Gaussian mixtures in q, Poisson counts y ~ Poisson(A f_true + r) (Sec. II,
Eq. 1) and the regularisation weight. It holds none of the reconstruction
method's arithmetic; the one forward product it needs (A f_true, to draw y)
and the backprojection that sets beta = 0.05 * max(A^T y) are scipy.sparse
library products.

Index conventions (shared by every consumer):
  hyper-voxel j = (x * Nz + z) * Nq + q   (q fastest; Sec. II "lexicographic")
  measurement i in [0, I)

System-matrix recipe (a stand-in for a coded-aperture fan-beam forward model,
whose real matrix the paper does not give):
  * one Bernoulli(0.5) code vector of length I;
  * column j = (x, z, q) starts its window at o = floor((z*Nq + q) * I / (Nz*Nq));
  * walking i = o, o+1, ... (mod I), row i is kept iff
    code[(i + x * floor(I / Nx)) mod I] == 1, until exactly nnz_col rows are kept;
  * rows are stored ascending inside each column, values are U(0.1, 1) drawn
    in CSC storage order; CSR is the stable transpose of CSC.
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = ["Problem", "make_problem", "PRESETS", "preset", "round_to_bf16", "batch_specs", "make_batch",
           "measure"]


@dataclasses.dataclass
class Problem:
    Nx: int
    Nz: int
    Nq: int
    I: int
    J: int
    nnz: int
    csc_colptr: np.ndarray  # int64 [J+1]
    csc_row: np.ndarray     # int32 [nnz]
    csc_val: np.ndarray     # float32 [nnz]
    csr_rowptr: np.ndarray  # int64 [I+1]
    csr_col: np.ndarray     # int32 [nnz]
    csr_val: np.ndarray     # float32 [nnz]
    y: np.ndarray           # float32 [I] (integer counts)
    b: np.ndarray           # float32 [1] (scalar background r)
    beta: float             # regularisation weight (the API's lambda)
    rho: float              # ADMM penalty (the paper's lambda)
    f_true: np.ndarray      # float32 [J] phantom
    seed: int = 0

    @property
    def shape(self):
        return (self.Nx, self.Nz, self.Nq)


# Sizes of the standard workloads.
PRESETS = {
    # 16x16 spatial x 32 q-bins = 8192 hyper-voxels, 4096 measurements.
    "tiny_16x16x32": dict(Nx=16, Nz=16, Nq=32, I=4096, nnz_col=64,
                          n_regions=4, mean_counts=50.0, seed=0),
    # 128x128 spatial x 64 q-bins = 1,048,576 hyper-voxels and measurements,
    # 256 nnz per column (2^28 nnz).
    "scale_128x128x64": dict(Nx=128, Nz=128, Nq=64, I=1 << 20, nnz_col=256,
                             n_regions=6, mean_counts=20.0, seed=1),
    # Same recipe at a quarter of the q-bins (67M nnz, about 1.1 GB on the device):
    # still far larger than L2, small enough for many-pass profiler captures.
    "mid_128x128x16": dict(Nx=128, Nz=128, Nq=16, I=1 << 18, nnz_col=256,
                           n_regions=6, mean_counts=20.0, seed=1),
    # Shape of the paper's Teflon scan (Sec. IV): about 41 x 9 spatial bins,
    # 54 q bins, 128-pixel x 64-channel detector, mean about 26 photons.
    "paper_41x9x54": dict(Nx=41, Nz=9, Nq=54, I=128 * 64, nnz_col=64,
                          n_regions=2, mean_counts=26.0, seed=2),
    # Wide image, few nonzeros: row tiles span more columns than a staging
    # window holds (exercises the unique-list tiles), column tiles mix windows
    # and lists (the windows that wrap around I).
    "wide_64x16x32": dict(Nx=64, Nz=16, Nq=32, I=32768, nnz_col=64,
                          n_regions=4, mean_counts=40.0, seed=7),
    # Ragged sizes: nothing is a multiple of a warp, a tile or a vector width.
    "ragged_13x7x37": dict(Nx=13, Nz=7, Nq=37, I=3001, nnz_col=50,
                           n_regions=3, mean_counts=30.0, seed=5),
    # Large image, few nonzeros per column (67M nnz, about 1.5 GB on the
    # device): the elementwise passes' vectors (about 185 MB) exceed L2, as
    # they do inside a full-size iteration, for profiler captures.
    "elem_256x256x64": dict(Nx=256, Nz=256, Nq=64, I=1 << 20, nnz_col=16,
                            n_regions=6, mean_counts=20.0, seed=11),
}


def preset(name: str, **overrides) -> "Problem":
    kw = dict(PRESETS[name])
    kw.update(overrides)
    return make_problem(**kw)


def _system_matrix_csc(rng, Nx, Nz, Nq, I, nnz_col):
    code = rng.random(I) < 0.5
    ones = np.flatnonzero(code).astype(np.int64)
    n1 = ones.size
    if n1 < nnz_col:
        raise ValueError(f"code has {n1} ones < nnz_col={nnz_col}; raise I")
    ZQ = Nz * Nq
    J = Nx * ZQ
    shift = I // Nx
    o = (np.arange(ZQ, dtype=np.int64) * I) // ZQ
    m = np.arange(nnz_col, dtype=np.int64)
    row = np.empty(J * nnz_col, dtype=np.int32)
    for x in range(Nx):
        p0 = (o + x * shift) % I                  # code position of each window start
        k0 = np.searchsorted(ones, p0)            # first set code bit at or after p0
        pos = ones[(k0[:, None] + m[None, :]) % n1]
        rows = (pos - x * shift) % I
        rows.sort(axis=1)
        row[x * ZQ * nnz_col:(x + 1) * ZQ * nnz_col] = rows.ravel()
    colptr = np.arange(0, J * nnz_col + 1, nnz_col, dtype=np.int64)
    val = rng.uniform(0.1, 1.0, J * nnz_col).astype(np.float32)
    return colptr, row, val


def _transpose(I, J, colptr, row, val):
    """Stable CSC -> CSR transpose (columns ascending inside each row)."""
    import torch  # a library stable sort; used only to build the CSR copy

    counts = np.bincount(row, minlength=I).astype(np.int64)
    rowptr = np.zeros(I + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    _, order = torch.sort(torch.from_numpy(row), stable=True)
    order = order.numpy()
    colidx = np.repeat(np.arange(J, dtype=np.int32), np.diff(colptr))
    return rowptr, colidx[order], val[order]


def _phantom(rng, Nx, Nz, Nq, n_regions):
    f = np.zeros((Nx, Nz, Nq), dtype=np.float64)
    q = np.arange(Nq, dtype=np.float64)
    for _ in range(n_regions):
        wx = int(rng.integers(max(1, Nx // 8), max(1, Nx // 2) + 1))
        wz = int(rng.integers(max(1, Nz // 8), max(1, Nz // 2) + 1))
        x0 = int(rng.integers(0, Nx - wx + 1))
        z0 = int(rng.integers(0, Nz - wz + 1))
        M = int(rng.integers(2, 5))
        mu = rng.uniform(0.0, Nq, M)
        sigma = rng.uniform(1.0, max(1.0, Nq / 8.0), M)
        amp = rng.uniform(0.5, 1.0, M)
        mtp = np.zeros(Nq)
        for a, m_, s_ in zip(amp, mu, sigma):
            mtp += a * np.exp(-((q - m_) ** 2) / (2.0 * s_ * s_))
        f[x0:x0 + wx, z0:z0 + wz, :] = mtp[None, None, :]
    return f.reshape(-1)


def make_problem(Nx, Nz, Nq, I, nnz_col, n_regions=4, mean_counts=50.0, seed=0,
                 beta_frac=0.05, rho=1.0) -> Problem:
    """Draw one problem. Generation order: code, A rows, A values, phantom, y."""
    import scipy.sparse as sp

    rng = np.random.Generator(np.random.PCG64(seed))
    J = Nx * Nz * Nq
    colptr, row, val = _system_matrix_csc(rng, Nx, Nz, Nq, I, nnz_col)
    rowptr, col, cval = _transpose(I, J, colptr, row, val)
    f = _phantom(rng, Nx, Nz, Nq, n_regions)

    A = sp.csc_matrix((val.astype(np.float64), row, colptr), shape=(I, J))
    Af = A @ f
    m = float(Af.mean())
    scale = (mean_counts / 1.1) / m if m > 0 else 1.0
    f *= scale
    Af *= scale
    r = 0.1 * float(Af.mean())
    y = rng.poisson(Af + r).astype(np.float32)
    bp = A.T @ y.astype(np.float64)
    beta = beta_frac * float(bp.max())
    return Problem(Nx=Nx, Nz=Nz, Nq=Nq, I=I, J=J, nnz=int(colptr[-1]),
                   csc_colptr=colptr, csc_row=row, csc_val=val,
                   csr_rowptr=rowptr, csr_col=col, csr_val=cval,
                   y=y, b=np.array([r], dtype=np.float32), beta=beta, rho=float(rho),
                   f_true=f.astype(np.float32), seed=seed)


def round_to_bf16(a: np.ndarray) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def batch_specs(n=64, seed=3000, nx=(32, 96), nq=(32, 64, 128), counts=(5.0, 100.0), nnz_col=128,
                n_regions=4):
    """Shapes of a batch of independent scans: Nx and Nz uniform on the
    integers of nx, Nq from nq, one measurement per hyper-voxel, nnz_col
    nonzeros per column, mean counts uniform on `counts`; scan k is drawn with
    seed + k."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for k in range(n):
        Nx = int(rng.integers(nx[0], nx[1] + 1))
        Nz = int(rng.integers(nx[0], nx[1] + 1))
        Nq = int(rng.choice(np.array(nq)))
        c = float(rng.uniform(counts[0], counts[1]))
        J = Nx * Nz * Nq
        specs.append(dict(Nx=Nx, Nz=Nz, Nq=Nq, I=J, nnz_col=nnz_col, n_regions=n_regions, mean_counts=c,
                          seed=seed + 1 + k))
    return specs


def make_batch(specs, workers=None):
    """Draw every scan of a batch (threads: the heavy NumPy / sort steps release the GIL)."""
    import concurrent.futures as cf
    import os

    workers = workers or min(len(specs), os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(workers) as ex:
        return list(ex.map(lambda kw: make_problem(**kw), specs))


def measure(P: Problem, seed, mean_counts=None, counts=(5.0, 100.0), n_regions=4, beta_frac=0.05) -> Problem:
    """A new seeded phantom and its counts through the system matrix of P (the
    same instrument): phantom as in make_problem, count level mean_counts or
    uniform on `counts`, y ~ Poisson(A f_true + r), beta = beta_frac max(A^T y).
    Shares P's matrix arrays."""
    import scipy.sparse as sp

    rng = np.random.Generator(np.random.PCG64(seed))
    c = float(rng.uniform(*counts)) if mean_counts is None else float(mean_counts)
    f = _phantom(rng, P.Nx, P.Nz, P.Nq, n_regions)
    A = sp.csc_matrix((P.csc_val.astype(np.float64), P.csc_row, P.csc_colptr), shape=(P.I, P.J))
    Af = A @ f
    m = float(Af.mean())
    scale = (c / 1.1) / m if m > 0 else 1.0
    f *= scale
    Af *= scale
    r = 0.1 * float(Af.mean())
    y = rng.poisson(Af + r).astype(np.float32)
    beta = beta_frac * float((A.T @ y.astype(np.float64)).max())
    return dataclasses.replace(P, y=y, b=np.array([r], dtype=np.float32), beta=beta, f_true=f.astype(np.float32),
                               seed=seed)
