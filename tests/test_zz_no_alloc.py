"""The allocation-free KKT residual entry point against the handle-based one.

sgtv_kkt_residual_noalloc serves callers that cannot allocate device memory
(a stream being captured into a CUDA graph, an external memory budget, a
real-time loop): its scratch is a fixed array inside the library. Here it is
called through the C ABI on device copies of a handle's state and must agree
with sgtv_residuals on two calls in a row (the shared scratch keeps the
previous call's contents, which must not leak into the next result).
"""
import numpy as np
import pytest

from paper_1601_08201_gb300 import sgtv, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def test_noalloc_kkt_matches_residuals_twice():
    P = synth.preset("ragged_13x7x37")
    with sgtv.Handle(P, precision="fp32") as h:
        h.iterate(25)
        kkt_ref = h.residuals()[2]
        f, _, c = h.get_state_f64()
    dev = torch.device("cuda", torch.cuda.current_device())

    def on_dev(a, dt):
        return torch.from_numpy(np.ascontiguousarray(a).astype(dt)).to(dev)

    A = {k: on_dev(getattr(P, k), dt) for k, dt in (
        ("csr_rowptr", np.int64), ("csr_col", np.int32), ("csr_val", np.float32),
        ("csc_colptr", np.int64), ("csc_row", np.int32), ("csc_val", np.float32))}
    s_host = np.add.reduceat(P.csc_val.astype(np.float64), P.csc_colptr[:-1]).astype(np.float32)
    y, b, s = on_dev(P.y, np.float32), on_dev(P.b, np.float32), on_dev(s_host, np.float32)
    fd, cd = on_dev(f, np.float32), on_dev(c, np.float32)
    out = torch.full((2,), -1.0, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    results = []
    for _ in range(2):
        out.fill_(-1.0)
        sgtv.kkt_residual_noalloc(P.I, P.J, A["csr_rowptr"].data_ptr(), A["csr_col"].data_ptr(),
                                  A["csr_val"].data_ptr(), A["csc_colptr"].data_ptr(), A["csc_row"].data_ptr(),
                                  A["csc_val"].data_ptr(), P.Nx, P.Nz, P.Nq, 4, [1.0] * 4, y.data_ptr(),
                                  (b.data_ptr(), 1), s.data_ptr(), fd.data_ptr(), cd.data_ptr(), P.rho,
                                  out.data_ptr(), stream)
        torch.cuda.synchronize()
        num, smax = out.cpu().numpy()
        results.append(num / max(1.0, smax))
    for kkt in results:
        assert abs(kkt - kkt_ref) <= 1e-5 * max(1.0, abs(kkt_ref)) + 1e-6, (kkt, kkt_ref)
    assert results[0] == results[1]


def test_noalloc_rejects_sizes_beyond_its_scratch():
    dev = torch.device("cuda", torch.cuda.current_device())
    dummy = torch.zeros(16, dtype=torch.float64, device=dev)
    p = dummy.data_ptr()
    J = 1 << 21  # more hyper-voxels than the fixed scratch holds
    with pytest.raises(sgtv.SgtvError, match="scratch"):
        sgtv.kkt_residual_noalloc(8, J, p, p, p, p, p, p, 1 << 10, 1 << 11, 1, 4, [1.0] * 4, p, (p, 1), p, p, p,
                                  1.0, p, 0)
