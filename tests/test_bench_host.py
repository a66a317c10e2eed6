"""Host-side pieces of bench.py that need no GPU: the sliced oracle that
times the CPU baseline does exactly the oracle's iteration, and the
algorithmic byte counts follow their formulas."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle as O  # noqa: E402
from paper_1601_08201_gb300 import synth  # noqa: E402


@pytest.mark.parametrize("F", [1, 2, 8])
def test_sliced_oracle_steps_make_whole_iterations(F):
    P = synth.preset("ragged_13x7x37")
    so = bench.SlicedOracle(P, F)
    for _ in range(2 * F):
        so.step()
    op = O.from_problem(P)
    f, d, c = O.iterate(op, O.init_state(op), 2)
    np.testing.assert_allclose(so.f, f, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(so.d, d, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(so.c, c, rtol=1e-12, atol=1e-13)


def test_algorithmic_bytes_formulas():
    P = synth.preset("tiny_16x16x32")
    ab = bench.algorithmic_bytes(P, "fp32")
    nnz, I, J = P.nnz, P.I, P.J
    # forward: A by rows and row pointers, f gathered once, y and r read, ratio written
    assert ab["k_forward"] == nnz * 8 + (I + 1) * 8 + 4 * (J + 2 * I) + 4 * P.b.size
    assert ab["k_back_update"] == nnz * 8 + (J + 1) * 8 + 4 * I + 12 * J + 32 * J
    assert ab["k_shrink"] == 4 * J * 13
    assert ab["k_iteration"] == ab["k_forward"] + ab["k_back_update"] + ab["k_shrink"]
    tli = {"csr": {"list_entries": 1000}, "csc": {"list_entries": 0}}
    t = bench.algorithmic_bytes(P, "bf16", {"k_forward": "tli_u8", "k_scatter": "tli_u8_private_keep"}, tli)
    ntiles = (I + 63) // 64
    assert t["k_forward"] == nnz * 4 + 16 * ntiles + 8 + 4000 + (I + 1) * 8 + 4 * (J + 2 * I) + 4 * P.b.size
    assert t["k_scatter"] == nnz * 4 + 16 * ntiles + 8 + 4000 + (I + 1) * 8 + 4 * (J + I + J) + 4 * P.b.size
    # single-pass form: the f-update reads e, s, f and u = d - c and writes
    # f_new and the cleared e; the shrink also writes u
    assert t["k_fupdate"] == 4 * J * 9
    assert t["k_shrink"] == 4 * J * 17
    # the row stream: every row padded to a multiple of 4 elements, its own row pointers
    rl = np.diff(P.csr_rowptr)
    nsp = int(((rl + 3) // 4 * 4).sum())
    sp = bench.algorithmic_bytes(P, "fp32", {"k_scatter": "sp_v4x3_nopf_min4_l2pf"}, tli)
    assert sp["k_scatter"] == (nsp * 6 + 16 * ntiles + 8 + 4000 + (I + 1) * 8 + (I + 1) * 8
                               + 4 * (J + I + J) + 4 * P.b.size)
    # the planning survey's basis: a plain 4-byte index and value per nonzero
    sb = bench.algorithmic_bytes(P, "fp32", {"k_scatter": "sp_v4x3_nopf_min4_l2pf"}, tli, survey_basis=True)
    assert sb["k_scatter"] == nnz * 8 + (I + 1) * 8 + 4 * (J + I + J) + 4 * P.b.size


def test_recorded_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    # roofline.traffic comes from a committed ncu record only while the kernel
    # sources it was taken on are unchanged (comments and white space aside)
    # and only for the variant it was taken on
    import json
    import shutil
    rec = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    mid = rec["k_scatter|mid_128x128x16|fp32"]
    full = rec["k_scatter|scale_128x128x64|fp32"]
    assert full["dram_bytes_per_launch"] == 4 * mid["dram_bytes_per_launch"]  # the stated scaling
    v = full["variant"]
    got = bench.recorded_traffic("k_scatter", "scale_128x128x64", "fp32", v)
    assert got == (full["dram_bytes_per_launch"] if full["source_sha"] == bench.kernel_source_hash() else None)
    assert bench.recorded_traffic("k_scatter", "scale_128x128x64", "fp32", v + "_other") is None
    assert bench.recorded_traffic("k_scatter", "no_such_workload", "fp32", v) is None

    # a copy of the sources: a comment or blank line leaves the hash, code changes it
    real = bench.kernel_source_hash()
    csrc = os.path.join(ROOT, "paper_1601_08201_gb300", "csrc")
    copy = tmp_path / "paper_1601_08201_gb300" / "csrc"
    shutil.copytree(csrc, copy, ignore=shutil.ignore_patterns("*.o", "*.so"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    assert h0 == real
    k = copy / "sgtv_kernels.cuh"
    text = k.read_text()
    k.write_text("// a comment\n\n" + text.replace("{", "{ /* block */", 1) + "\n   \n")
    assert bench.kernel_source_hash() == h0
    k.write_text(text.replace("T(0)", "T(0.0)", 1))
    assert bench.kernel_source_hash() != h0
