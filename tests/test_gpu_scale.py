"""Full-size parity (1M hyper-voxels, 2^28 nonzeros) in the launch configuration
the benchmark times: whole-array comparison against the FP64 oracle after a few
iterations, and the FP64 objective at the GPU's iterate."""
import numpy as np
import pytest

import oracle as O
from paper_1601_08201_gb300 import sgtv, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def big():
    P = synth.preset("scale_128x128x64")
    return P, O.from_problem(P)


def rel(a, b):
    # relative L2 error; absolute when the reference is exactly zero (e.g. d
    # after the first iterations, when every group is shrunk to zero)
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a, np.float64) - b) / (nb if nb > 0 else 1.0)


def test_full_size_fp32_iterations(big):
    P, op = big
    st = O.init_state(op)
    stream = torch.cuda.Stream()
    with sgtv.Handle(P, precision="fp32", stream=stream.cuda_stream) as h:
        g = h.get_state_f64()
        assert rel(g[0], st[0]) <= 1e-6
        done = 0
        for k in (1, 3):
            h.iterate(k - done)
            st = O.iterate(op, st, k - done)
            done = k
            f, d, c = h.get_state_f64()
            assert rel(f, st[0]) <= 1e-5, (k, rel(f, st[0]))
            assert rel(d, st[1]) <= 1e-4, (k, rel(d, st[1]))
        phi, dev, tv = h.objective()
        ophi, odev, otv = O.objective(op, f)
        assert dev == pytest.approx(odev, rel=1e-10)
        assert tv == pytest.approx(otv, rel=1e-10)
        assert abs(phi - O.objective(op, st[0])[0]) <= 1e-6 * abs(phi)


def test_full_size_bf16_values(big):
    P, _ = big
    op = O.from_problem(P, csr_val=synth.round_to_bf16(P.csr_val), csc_val=synth.round_to_bf16(P.csc_val))
    st = O.iterate(op, O.init_state(op), 1)
    with sgtv.Handle(P, precision="bf16") as h:
        h.iterate(1)
        f = h.get_state_f64()[0]
    assert rel(f, st[0]) <= 1e-5


def test_full_size_single_pass(big):
    # one pass over the rows per iteration (the bench's alternative launch form)
    P, op = big
    st = O.iterate(op, O.init_state(op), 2)
    stream = torch.cuda.Stream()
    with sgtv.Handle(P, precision="fp32", stream=stream.cuda_stream,
                     flags=sgtv.FLAG_SINGLE_PASS | sgtv.FLAG_GRAPH) as h:
        h.iterate(2)
        f = h.get_state_f64()[0]
    assert rel(f, st[0]) <= 1e-5


def test_full_size_precision_report(big):
    # BF16 values against the FP64 oracle after 50 and 500 iterations, next to
    # the FP32 run: the arithmetic error (oracle on the BF16-rounded matrix)
    # and the precision effect of rounding A (oracle on the original matrix)
    P, op = big
    opb = O.from_problem(P, csr_val=synth.round_to_bf16(P.csr_val), csc_val=synth.round_to_bf16(P.csc_val))
    st, stb = O.init_state(op), O.init_state(opb)
    stream = torch.cuda.Stream()
    report = {}
    with sgtv.Handle(P, precision="fp32", stream=stream.cuda_stream) as h32, \
            sgtv.Handle(P, precision="bf16", stream=stream.cuda_stream) as h16:
        done = 0
        for k in (50, 500):
            h32.iterate(k - done)
            h16.iterate(k - done)
            st = O.iterate(op, st, k - done)
            if k == 50:
                stb = O.iterate(opb, stb, k)
            done = k
            f32 = h32.get_state_f64()[0]
            f16 = h16.get_state_f64()[0]
            phi = O.objective(op, st[0])[0]
            report[k] = dict(fp32_image=rel(f32, st[0]), bf16_image=rel(f16, st[0]),
                             fp32_phi=abs(h32.objective()[0] - phi) / phi,
                             bf16_phi=abs(O.objective(op, f16)[0] - phi) / phi)
            if k == 50:
                report[k]["bf16_vs_rounded_oracle"] = rel(f16, stb[0])
    print(report)
    assert report[50]["fp32_image"] <= 1e-5 and report[50]["bf16_vs_rounded_oracle"] <= 1e-5
    assert report[500]["fp32_image"] <= 1e-4
    # rounding A to BF16 changes the iterate by about its relative rounding (2^-9)
    assert report[500]["bf16_image"] <= 1e-2
