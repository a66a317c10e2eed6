#!/usr/bin/env python3
"""Benchmark: ADMM iterations per second of spectrally grouped TV reconstruction
on the 1M-hyper-voxel workload (128 x 128 spatial x 64 q-bins, 1,048,576
measurements, 256 nonzeros per column = 2^28 nonzeros, FP32).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One step = one ADMM iteration (forward projection + ratio, backprojection
fused with the hyper-voxel update, group shrink + dual update) over the whole
problem, inputs resident in HBM. The matrix (4.3 GB as CSR + CSC) is far
larger than L2, so no flush is needed between iterations. With N > 1 (launched
by torchrun) every rank solves its own independent scan: replicas, weak
scaling. Rank 0 prints one JSON line.

--impl reference times the FP64 CPU oracle on the host cores on the same
workload; each step is 1/F of one oracle iteration (row and column blocks),
F chosen so the run stays within a few minutes.
"""
from __future__ import annotations

import argparse
import ctypes
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ADMM iter/s at 1M hyper-voxels"
WORKLOAD = "scale_128x128x64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ttt", action="store_true", help="skip the time-to-tolerance measurement")
    ap.add_argument("--form", default="single_pass", choices=["single_pass", "two_pass"],
                    help="iteration form of the headline: A streamed once per surrogate step (CSR forward + "
                         "scatter, then an elementwise f-update) or twice (CSR forward, CSC backprojection "
                         "fused with the f-update)")
    ap.add_argument("--single-pass", dest="form", action="store_const", const="single_pass")
    ap.add_argument("--two-pass", dest="form", action="store_const", const="two_pass")
    ap.add_argument("--no-other-form", action="store_true", help="skip the timing of the other iteration form")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-scan batched form's timing")
    ap.add_argument("--no-single-pass", dest="no_other_form", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--scatter-variant", default=None,
                    help="pin the single-pass scatter form by name (no autotuning)")
    ap.add_argument("--ttt-iters", type=int, default=8000, help="length of the time-to-tolerance trace")
    ap.add_argument("--ttt-every", type=int, default=10, help="iterations between objective evaluations")
    ap.add_argument("--ttt-rho-tuned", type=float, default=4096.0,
                    help="also trace the time to tolerance at this ADMM penalty (0: skip); the penalty is not "
                         "part of the problem (Eq. 4's minimum does not depend on it)")
    ap.add_argument("--phi-star", default=None,
                    help="JSON record of phi* (default: profiles/phi_star_<workload>.json when present; "
                         "else phi* = the lowest traced value, labelled as such)")
    ap.add_argument("--variants", default=None,
                    help="pin the SpMV variants as 'forward_name,back_name' (no autotuning), e.g. for "
                         "profiler captures, where the profiler's overhead would skew the autotuner")
    return ap.parse_args()


def max_over_ranks(x, ws, device):
    """The largest of every rank's x (the job's time is its slowest rank's)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws, steps, ms):
    """Iterations per second of the whole job: every rank ran `steps`
    iterations of its own scan, and the slowest took `ms` milliseconds."""
    return ws * steps / (ms / 1e3)


def replica_seed(workload, rank):
    """Each rank solves its own scan of the workload's shape: seed offset by rank."""
    from paper_1601_08201_gb300 import synth
    return synth.PRESETS[workload]["seed"] + 1000 * rank


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_config(name, P, ws=1):
    """The workload, identical in both arms (the arithmetic type is the line's dtype)."""
    return {"workload": f"{name}: {P.Nx}x{P.Nz} spatial x {P.Nq} q-bins = {P.J} hyper-voxels, "
                        f"{P.I} measurements, {P.nnz // P.J} nnz/column ({P.nnz} nnz)",
            "Nx": P.Nx, "Nz": P.Nz, "Nq": P.Nq, "I": P.I, "J": P.J, "nnz": P.nnz,
            "n_dirs": 4, "beta": P.beta, "rho": P.rho,
            "l2_flush": "not needed: the matrix streamed every iteration (>= 1.1 GB) is >> 129 MB L2",
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"}


# ------------------------------------------------------------------------------------------
# oracle timing (the CPU baseline; also the whole --impl reference arm)

def oracle_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


class SlicedOracle:
    """Runs the FP64 oracle's own functions over 1/F of one ADMM iteration per
    step, in the iteration's order: with F = 1 one step is a whole iteration;
    with F even, steps 0 .. F/2 - 1 project row blocks (the surrogate
    coefficients at the first) and steps F/2 .. F - 1 backproject column
    blocks with their f-update (the group shrink at the last). F consecutive
    steps compute exactly one oracle iteration."""

    def __init__(self, P, F):
        import oracle as O
        if F != 1 and F % 2:
            raise ValueError("F must be 1 or even")
        self.O = O
        self.lib = O._load()
        self.op = O.from_problem(P)
        self.F = F
        self.f, self.d, self.c = O.init_state(self.op)
        op = self.op
        self.ybar = np.empty(op.I)
        self.ratio = np.zeros(op.I)
        self.e = np.empty(op.J)
        self.alpha = np.empty(op.J)
        self.gamma = np.empty(op.J)
        self.fn = self.f.copy()
        self.u = np.empty_like(self.d)
        self.k = 0

    @staticmethod
    def _at(a, off):
        return ctypes.c_void_p(a.ctypes.data + off * a.itemsize)

    def _coeffs(self):
        op, at = self.op, self._at
        np.subtract(self.d, self.c, out=self.u)
        self.lib.oracle_surrogate_coeffs(ctypes.c_int32(op.Nx), ctypes.c_int32(op.Nz), ctypes.c_int32(op.Nq),
                                         ctypes.c_int(op.n_dirs), at(op.w, 0), ctypes.c_double(op.rho),
                                         at(self.f, 0), at(self.u, 0), at(self.alpha, 0), at(self.gamma, 0))

    def _rows(self, i0, i1):
        op, at = self.op, self._at
        self.lib.oracle_forward(ctypes.c_int64(i1 - i0), at(op.rowptr, i0), at(op.col, 0), at(op.rval, 0),
                                at(self.f, 0), at(op.r, 0), ctypes.c_int64(op.r.size), at(op.y, i0),
                                at(self.ybar, i0), at(self.ratio, i0))

    def _cols(self, j0, j1):
        op, at = self.op, self._at
        self.lib.oracle_backproject(ctypes.c_int64(j1 - j0), at(op.colptr, j0), at(op.row, 0), at(op.cval, 0),
                                    at(self.ratio, 0), at(self.e, j0))
        self.lib.oracle_f_update(ctypes.c_int64(j1 - j0), at(self.f, j0), at(self.e, j0), at(op.s, j0),
                                 at(self.alpha, j0), at(self.gamma, j0), at(self.fn, j0))

    def _shrink(self):
        op, at = self.op, self._at
        self.f, self.fn = self.fn, self.f
        if op.rho > 0.0:
            self.lib.oracle_shrink_dual(ctypes.c_int32(op.Nx), ctypes.c_int32(op.Nz), ctypes.c_int32(op.Nq),
                                        ctypes.c_int(op.n_dirs), at(op.w, 0), ctypes.c_double(op.beta / op.rho),
                                        ctypes.c_int(int(op.per_bin)), at(self.f, 0), at(self.d, 0),
                                        at(self.c, 0))

    def step(self):
        op, F = self.op, self.F
        if F == 1:
            self._coeffs()
            self._rows(0, op.I)
            self._cols(0, op.J)
            self._shrink()
        else:
            H = F // 2
            b = self.k % F
            if b < H:
                if b == 0:
                    self._coeffs()
                self._rows(op.I * b // H, op.I * (b + 1) // H)
            else:
                b -= H
                self._cols(op.J * b // H, op.J * (b + 1) // H)
                if b == H - 1:
                    self._shrink()
        self.k += 1


def time_oracle(P, steps, warmup, budget_s=120.0, F=None):
    """Returns (iter/s, F, seconds timed, steps)."""
    if F is None:
        probe = SlicedOracle(P, 16)
        t0 = time.perf_counter()
        for _ in range(4):
            probe.step()
        t_iter = (time.perf_counter() - t0) / 4 * 16
        del probe
        F = 1
        while steps * t_iter / F > budget_s and F < 4096:
            F *= 2
    so = SlicedOracle(P, F)
    for _ in range(warmup):
        so.step()
    t0 = time.perf_counter()
    for _ in range(steps):
        so.step()
    dt = time.perf_counter() - t0
    return (steps / F) / dt, F, dt, steps


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1601_08201_gb300 import synth
    P = synth.preset(args.workload)
    rate, F, dt, steps = time_oracle(P, args.steps, args.warmup)
    cores = oracle_threads()
    sample = (f"each step = 1/{F} of one FP64 oracle ADMM iteration on the full {args.workload} "
              f"problem (row blocks, then column blocks with their f-update; whole-image passes once "
              f"per {F} steps)")
    line = {"metric": METRIC, "value": rate, "unit": "iter/s", "impl": "reference", "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.workload, P, ws),
            "cpu_baseline": {"value": rate, "unit": "iter/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_uuid=None):
        self.proc = None
        self.path = None
        self.uuid = gpu_uuid

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.out, stderr=subprocess.DEVNULL)
            time.sleep(0.6)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def gpu_uuid(torch):
    try:
        u = str(torch.cuda.get_device_properties(0).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# ------------------------------------------------------------------------------------------
# roofline bookkeeping

def algorithmic_bytes(P, precision, variants=None, tli=None, n_dirs=4, survey_basis=False):
    """Bytes each kernel must move per launch (compulsory traffic, gathers of
    the L2-resident dense vectors counted once).

    Format basis (default): what the kernel's stored form streams. The tiled
    local-index (TLI) variants stream 2-byte indices plus per-tile metadata
    (window base and length, list offsets and unique-index lists); their staged
    window copies are L2 re-reads of f / ratio and are not counted. The
    single-pass row-stream variants ("sp_") stream the same 2-byte indices and
    values with each row padded to a multiple of 4 elements, plus their own
    row pointers. Survey basis (survey_basis=True): every SpMV streams a plain
    int32 index and a value per nonzero (4 + V bytes), the accounting of the
    planning survey's roofline table."""
    T = 8 if precision == "fp64" else 4
    V = {"fp32": 4, "bf16": 2, "fp64": 8}[precision]
    nnz, I, J = P.nnz, P.I, P.J
    variants = variants or {}
    out = {}

    def stream(kernel, side, nseg):
        name = variants.get(kernel, "")
        if survey_basis or not tli:
            return nnz * (4 + V)
        ntiles = (nseg + 63) // 64
        meta = 8 * (ntiles + 1) + 8 * ntiles + 4 * tli[side]["list_entries"]
        if name.startswith("tli"):
            return nnz * (2 + V) + meta
        if name.startswith("sp_"):
            rl = np.diff(P.csr_rowptr)
            nsp = int(((rl + 3) // 4 * 4).sum())
            return nsp * (2 + V) + meta + 8 * (I + 1)
        return nnz * (4 + V)

    # A by rows, row pointers, f gathered once, y, r, ratio written
    out["k_forward"] = stream("k_forward", "csr", I) + (I + 1) * 8 + J * T + I * T + I * T + P.b.size * T
    # A by columns, column pointers, ratio gathered once, f (read), s, f_new (write), d and c
    out["k_back_update"] = (stream("k_back_update", "csc", J) + (J + 1) * 8 + I * T + 3 * J * T
                            + 2 * n_dirs * J * T)
    single = "k_scatter" in variants
    # f_new, c read; d, c written (and, in the single-pass form, u = d - c
    # for the f-update)
    out["k_shrink"] = J * T + (4 if single else 3) * n_dirs * J * T
    # single-pass form: the CSR stream once, f gathered once, y, r, e written
    # once (its atomic adds stay in L2); the f-update reads e, s, f, u and
    # writes f_new and the cleared e
    out["k_scatter"] = stream("k_scatter", "csr", I) + (I + 1) * 8 + J * T + I * T + P.b.size * T + J * T
    out["k_fupdate"] = J * T * (5 + n_dirs)
    # the persistent one-launch iteration moves what the three kernels move
    out["k_iteration"] = out["k_forward"] + out["k_back_update"] + out["k_shrink"]
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the sources that define and launch the iteration's kernels
    (kernel bodies, launchers, shared types, the per-precision instantiations)
    with comments and white space removed: a comment or host-API edit does not
    change the kernels the recorded counters describe."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1601_08201_gb300", "csrc")
    files = ["sgtv_kernels.cuh", "sgtv_kset.cuh", "sgtv_internal.h", "kset_f32.cu", "kset_bf16.cu", "kset_f64.cu"]
    for f in files:
        text = open(os.path.join(csrc, f), encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update(re.sub(r"\s+", "", text).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload, precision, variant=None):
    """dram bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources and the same variant; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    ent = rec.get(f"{kernel}|{workload}|{precision}")
    if not ent or ent.get("source_sha") != kernel_source_hash():
        return None
    if variant is not None and ent.get("variant") not in (None, variant):
        return None
    return ent.get("dram_bytes_per_launch")


# ------------------------------------------------------------------------------------------

def batch_bytes(scans, precision, form, tli):
    """Algorithmic bytes of one iteration over all scans of a batch (format
    basis, as algorithmic_bytes for one problem; the tiled forms' unique lists
    counted from the handle)."""
    T = 8 if precision == "fp64" else 4
    V = {"fp32": 4, "bf16": 2, "fp64": 8}[precision]
    I = sum(P.I for P in scans)
    J = sum(P.J for P in scans)
    nnz = sum(P.nnz for P in scans)
    nt_r, nt_c = (I + 63) // 64, (J + 63) // 64
    meta_r = 16 * nt_r + 8 + 4 * tli["csr"]["list_entries"]
    meta_c = 16 * nt_c + 8 + 4 * tli["csc"]["list_entries"]
    return sum(batch_bytes_by_kernel(scans, precision, form, tli).values())


def batch_bytes_by_kernel(scans, precision, form, tli):
    """batch_bytes split by kernel."""
    T = 8 if precision == "fp64" else 4
    V = {"fp32": 4, "bf16": 2, "fp64": 8}[precision]
    I = sum(P.I for P in scans)
    J = sum(P.J for P in scans)
    nnz = sum(P.nnz for P in scans)
    nt_r, nt_c = (I + 63) // 64, (J + 63) // 64
    meta_r = 16 * nt_r + 8 + 4 * tli["csr"]["list_entries"]
    meta_c = 16 * nt_c + 8 + 4 * tli["csc"]["list_entries"]
    if form == "single_pass":
        nsp = sum(int(((np.diff(P.csr_rowptr) + 3) // 4 * 4).sum()) for P in scans)
        # f-update: e, s, f, u (4 directions), f_new, e cleared; shrink: f, c read, d, c, u written
        return {"k_scatter": nsp * (2 + V) + meta_r + 16 * (I + 1) + T * (J + 2 * I + J),
                "k_fupdate": T * J * 9, "k_shrink": T * J * 17}
    return {"k_forward": nnz * (2 + V) + meta_r + 8 * (I + 1) + T * (J + 3 * I),
            "k_back_update": nnz * (2 + V) + meta_c + 8 * (J + 1) + T * I + 3 * T * J + 8 * T * J,
            "k_shrink": 13 * T * J}


def batched_form(sgtv, synth, args, stream, torch, form, K, W, sample_clocks=False):
    """The 64-scan batched workload (uneven Nx x Nz x Nq, I = J, 128 nnz per
    column) in one handle, against the same scans solved one after another as
    64 one-scan handles, both in the given iteration form with CUDA-graph
    replay (and, for the two-pass form, the persistent one-launch iteration):
    K iterations of every scan after W warm-up ones, CUDA events."""
    t0 = time.perf_counter()
    scans = synth.make_batch(synth.batch_specs())
    t_gen = time.perf_counter() - t0
    base = form_flags(sgtv, form) | sgtv.FLAG_GRAPH

    def run(problem, flags, clocks=False, attribute=False):
        h = sgtv.Handle(problem, precision=args.precision, stream=stream.cuda_stream, flags=flags)
        h.iterate(W)
        h.sync()
        if attribute:  # each kernel alone (no graphs, one stream), CUDA events per launch
            h.profile(True)
            h.iterate(K)
            prof = {k: v for k, v in h.profile_read().items() if v[1] > 0}
            h.profile(False)
            h.sync()
            tli = h.tli_info()
            h.close()
            return {"prof": prof, "tli": tli}
        sampler = ClockSampler(gpu_uuid(torch)) if clocks else None
        if sampler:
            sampler.start()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.iterate(K)
        e1.record(stream)
        torch.cuda.synchronize()
        out = dict(ms=e0.elapsed_time(e1) / K, clocks=sampler.stop() if sampler else None)
        if isinstance(problem, list):
            out.update(f=h.get_state_f64()[0], info=h.batch_info(), tli=h.tli_info())
            names = h.variant_names()
            out["tuning"] = ({"k_scatter": names["k_scatter"][h.get_variant(sgtv.K_SCATTER)]}
                             if form == "single_pass" else
                             {"k_forward": names["k_forward"][h.get_variants()[0]],
                              "k_back_update": names["k_back_update"][h.get_variants()[1]]})
        else:
            out["f"] = h.get_state_f64()[0]
        h.close()
        return out

    b = run(scans, base, sample_clocks)
    pers = run(scans, sgtv.FLAG_PERSISTENT | sgtv.FLAG_GRAPH) if form == "two_pass" else None
    seq_ms, max_rel = 0.0, 0.0
    off = b["info"]["vox_off"]
    for k, P in enumerate(scans):
        o = run(P, base)
        seq_ms += o["ms"]
        ref = b["f"][off[k]:off[k + 1]]
        max_rel = max(max_rel, float(np.linalg.norm(o["f"] - ref) / max(np.linalg.norm(o["f"]), 1e-300)))
    peak, peak_kind = measured_peaks()
    by = batch_bytes(scans, args.precision, form, b["tli"])
    att = run(scans, form_flags(sgtv, form) | sgtv.FLAG_SERIAL, attribute=True)
    kb = batch_bytes_by_kernel(scans, args.precision, form, att["tli"])
    per_kernel = {k: {"avg_us": 1e3 * v[0] / v[1], "launches": v[1], "algorithmic_bytes": kb.get(k),
                      "frac_of_measured_hbm": (kb[k] / (v[0] / v[1] / 1e3) / 1e9 / peak) if k in kb else None}
                  for k, v in att["prof"].items()}
    J = sum(P.J for P in scans)
    nnz = sum(P.nnz for P in scans)
    rec = {"value": 1e3 / b["ms"], "unit": "iter/s (all 64 scans)", "ms_per_step": b["ms"],
           "iteration_form": FORMS[form] + ", CUDA-graph replay", "tuning": b["tuning"],
           "workload": f"batched64: 64 scans, Nx,Nz in [32,96], Nq in {{32,64,128}}, I = J, 128 nnz/col; "
                       f"{J} hyper-voxels, {nnz} nnz in total",
           "sequential_one_scan_handles": {"value": 1e3 / seq_ms, "ms_per_step": seq_ms},
           "speedup_vs_sequential": seq_ms / b["ms"],
           "batched_vs_sequential_max_rel_l2": max_rel,
           "roofline": {"bound": "hbm", "achieved": by / (b["ms"] / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": by / (b["ms"] / 1e3) / 1e9 / peak, "peak_source": peak_kind,
                        "bytes_per_iteration": by},
           "kernels_alone": {"per_kernel": per_kernel,
                             "note": "the batch again without graphs, every kernel on one stream "
                                     "(SGTV_FLAG_SERIAL), K iterations, CUDA events per launch"},
           "generation_s": round(t_gen, 1), "clocks": b["clocks"]}
    if pers is not None:
        rec["persistent_one_launch"] = {"value": 1e3 / pers["ms"], "ms_per_step": pers["ms"]}
    return rec


def run_batched(args):
    """The batched workload alone: one JSON line."""
    import torch
    from paper_1601_08201_gb300 import sgtv, synth

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    rec = batched_form(sgtv, synth, args, stream, torch, args.form, args.steps, args.warmup, sample_clocks=True)
    line = {"metric": "ADMM iter/s, 64-scan batch", "value": rec["value"], "unit": "iter/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16": "bf16-values/f32", "fp64": "f64"}[args.precision],
            "data": "synthetic", "config": {"workload": rec["workload"]}, **{k: v for k, v in rec.items()
                                                                             if k not in ("value", "workload")}}
    print(json.dumps(line), flush=True)
    return 0


FORMS = {
    "single_pass": "single pass: CSR forward + scatter into e (bank-dealt row stream), elementwise f-update, shrink",
    "two_pass": "two passes: CSR forward, CSC backprojection fused with the f-update, shrink",
}


def form_flags(sgtv, form):
    return sgtv.FLAG_SINGLE_PASS if form == "single_pass" else 0


def time_form(sgtv, P, args, form, stream, torch, barrier, ws, sample_clocks=False):
    """One handle in the given iteration form: W warm-up iterations, then
    exactly K timed ones between barriers, CUDA events on the handle's stream
    (per-kernel events from sgtv_profile inside the same region)."""
    flags = form_flags(sgtv, form)
    pin_fwd = args.variants and form == "two_pass"
    pin_sc = args.scatter_variant and form == "single_pass"
    if pin_fwd or pin_sc:
        flags |= sgtv.FLAG_NO_AUTOTUNE
    h = sgtv.Handle(P, precision=args.precision, stream=stream.cuda_stream, flags=flags)
    names = h.variant_names()
    if pin_fwd:
        vf, vb = args.variants.split(",")
        h.set_variants(names["k_forward"].index(vf), names["k_back_update"].index(vb))
    if pin_sc:
        h.set_variant(sgtv.K_SCATTER, names["k_scatter"].index(args.scatter_variant))
    if form == "single_pass":
        tuning = {"k_scatter": names["k_scatter"][h.get_variant(sgtv.K_SCATTER)], "k_fupdate": "per site",
                  "k_shrink": "per site"}
    else:
        vf, vb = h.get_variants()
        tuning = {"k_forward": names["k_forward"][vf], "k_back_update": names["k_back_update"][vb],
                  "k_shrink": "per site"}
    h.iterate(args.warmup)
    h.sync()
    sampler = ClockSampler(gpu_uuid(torch)) if sample_clocks else None
    if sampler:
        sampler.start()
    barrier()
    h.profile(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.iterate(args.steps)
    e1.record(stream)
    barrier()
    clocks = sampler.stop() if sampler else None
    prof = {k: v for k, v in h.profile_read().items() if v[1] > 0}
    h.profile(False)
    h.sync()
    ms = max_over_ranks(e0.elapsed_time(e1), ws, "cuda")
    # attribution pass after the timed region: the same K iterations with every
    # kernel on one stream (the shrink not overlapped), so that each kernel's
    # events time it alone
    h.set_serial(True)
    h.profile(True)
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    h.iterate(args.steps)
    a1.record(stream)
    prof_alone = {k: v for k, v in h.profile_read().items() if v[1] > 0}
    h.profile(False)
    h.sync()
    h.set_serial(False)
    ms_serial = a0.elapsed_time(a1)
    tli = h.tli_info()
    h.close()
    ab = algorithmic_bytes(P, args.precision, tuning, tli)
    peak, peak_kind = measured_peaks()

    def table(pr):
        tot = sum(x[0] for x in pr.values())
        return {k: {"avg_us": 1e3 * v[0] / v[1], "launches": v[1], "share": v[0] / tot,
                    "algorithmic_bytes": ab[k], "achieved_gbs": ab[k] / (v[0] / v[1] / 1e3) / 1e9,
                    "frac_of_measured_hbm": ab[k] / (v[0] / v[1] / 1e3) / 1e9 / peak}
                for k, v in pr.items()}

    alone = {"ms_per_step": ms_serial / args.steps, "per_kernel": table(prof_alone),
             "note": "the same K iterations after the timed region with every kernel on one stream "
                     "(sgtv_set_serial): each kernel timed alone; in the timed region the shrink runs on a "
                     "second stream beside the next forward pass, and its events span that overlap"}
    return {"form": form, "ms": ms, "value": whole_job_rate(ws, args.steps, ms), "prof": prof,
            "per_kernel": table(prof), "alone": alone, "tuning": tuning, "tli": tli, "clocks": clocks, "ab": ab,
            "launches": int(sum(n for _, n in prof.values()))}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched64":
        return run_batched(args)
    import torch
    import torch.distributed as dist
    from paper_1601_08201_gb300 import sgtv, synth

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the CUDA path has no CPU fallback)")
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sgtv.load()

    seed = replica_seed(args.workload, rank)
    P = synth.preset(args.workload, seed=seed)
    # a dedicated torch stream: the handle issues its kernels on it and the
    # timing events are recorded on the same stream
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    form = args.form
    head = time_form(sgtv, P, args, form, stream, torch, barrier, ws, sample_clocks=True)

    # roofline of the dominant kernel
    prof, ab, peak_kind = head["prof"], head["ab"], measured_peaks()[1]
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms = prof[dom][0] / prof[dom][1]
    achieved = ab[dom] / (dom_ms / 1e3) / 1e9
    peak = measured_peaks()[0]
    sb = algorithmic_bytes(P, args.precision, head["tuning"], head["tli"], survey_basis=True)
    it_survey = sum(sb[k] * v[1] for k, v in prof.items()) / args.steps
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "bytes_basis": "the kernel's stored format (16-bit local indices, padded rows)",
                "survey_basis": {"kernel_bytes": sb[dom], "achieved": sb[dom] / (dom_ms / 1e3) / 1e9,
                                 "frac": sb[dom] / (dom_ms / 1e3) / 1e9 / peak,
                                 "iteration_bytes": it_survey,
                                 "iteration_frac": it_survey / (head["ms"] / args.steps / 1e3) / 1e9 / peak,
                                 "note": "4-byte index + value per nonzero per SpMV pass, the planning "
                                         "survey's accounting"},
                "traffic": recorded_traffic(dom, args.workload, args.precision, head["tuning"].get(
                    "k_scatter" if form == "single_pass" else ("k_forward" if dom == "k_forward" else "k_back_update"))),
                "per_kernel": head["per_kernel"], "kernels_alone": head["alone"]}

    # the other iteration form on the same workload
    other = None
    if not args.no_other_form:
        o = time_form(sgtv, P, args, "two_pass" if form == "single_pass" else "single_pass", stream, torch,
                      barrier, ws)
        other = {"value": o["value"], "unit": "iter/s", "ms_per_step": o["ms"] / args.steps,
                 "iteration_form": FORMS[o["form"]], "tuning": o["tuning"], "per_kernel": o["per_kernel"],
                 "kernels_alone": o["alone"]}
        if o["form"] == "single_pass":
            other["note"] = "same iteration; e's sums are formed in an order set by atomic adds"

    # time to relative objective gaps of 1e-2, 1e-3, 1e-4 against a recorded phi*
    ttt = None
    if not args.no_ttt and rank == 0:
        ttt = time_to_tolerance(sgtv, P, args, stream, torch, form_flags(sgtv, form))
        if args.ttt_rho_tuned > 0:
            ttt["tuned_rho"] = time_to_tolerance(sgtv, P, args, stream, torch, form_flags(sgtv, form),
                                                 rho=args.ttt_rho_tuned)
            ttt["tuned_rho"]["note"] = ("the same method and problem with a larger ADMM penalty (the paper's "
                                        "lambda, Eqs. 5-7); the configured rho converges slowly on this problem")

    # end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(sgtv, P, args, stream, torch, barrier, ws, form_flags(sgtv, form))

    # the batched workload (64 uneven scans in one handle) against 64 one-scan handles
    batched = None
    if not args.no_batched and rank == 0:
        batched = batched_form(sgtv, synth, args, stream, torch, form, min(args.steps, 20), 3)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # about 10-30 s of oracle work: probe one iteration, then time n of them
        _, _, t_one, _ = time_oracle(P, steps=16, warmup=0, F=16)
        n_it = max(1, min(200, int(np.ceil(12.0 / max(t_one, 1e-3)))))
        rate, F, dt, steps = time_oracle(P, steps=16 * n_it, warmup=0, F=16)
        cpu = {"value": rate, "unit": "iter/s", "cores": oracle_threads(), "kind": "oracle",
               "sample": f"{n_it} FP64 oracle ADMM iterations ({16 * n_it} steps of 1/16 iteration) "
                         f"on the full {args.workload} problem, {dt:.1f} s"}

    if rank == 0:
        line = {"metric": METRIC, "value": head["value"], "unit": "iter/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": head["ms"] / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32", "bf16": "bf16-values/f32", "fp64": "f64"}[args.precision],
                "data": "synthetic", "config": workload_config(args.workload, P, ws),
                "iteration_form": FORMS[form],
                "tuning": {**head["tuning"], "tiled_index_forms": head["tli"]},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": head["clocks"],
                "gpu_launches": head["launches"] * ws, "time_to_tolerance": ttt, "batched_form": batched,
                ("two_pass_form" if form == "single_pass" else "single_pass_form"): other}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def end_to_end(sgtv, P, args, stream, torch, barrier, ws, flags=0):
    """sgtv_setup from pinned host buffers (H2D inside), K iterations, image D2H."""
    def pin(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        return t.numpy()
    arrs = dict(csr_rowptr=pin(P.csr_rowptr), csr_col=pin(P.csr_col), csr_val=pin(P.csr_val),
                csc_colptr=pin(P.csc_colptr), csc_row=pin(P.csc_row), csc_val=pin(P.csc_val),
                y=pin(P.y), b=pin(P.b))
    h2d = sum(a.nbytes for a in arrs.values())
    img = pin(np.empty(P.J, np.float32))
    opts = sgtv.make_opts(precision=args.precision, stream=stream.cuda_stream, flags=flags)
    barrier()
    t0 = time.perf_counter()
    h = sgtv.setup(P.I, P.J, P.nnz, arrs["csr_rowptr"], arrs["csr_col"], arrs["csr_val"],
                   arrs["csc_colptr"], arrs["csc_row"], arrs["csc_val"], P.Nx, P.Nz, P.Nq,
                   arrs["y"], arrs["b"], P.beta, P.rho, opts)
    sgtv.iterate(h, args.steps)
    sgtv.get_image(h, img)
    t1 = time.perf_counter()
    sgtv.destroy(h)
    dt = t1 - t0
    dt = max_over_ranks(dt, ws, "cuda")
    return {"value": whole_job_rate(ws, args.steps, 1e3 * dt), "unit": "iter/s",
            "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": img.nbytes / args.steps,
            "solve": f"sgtv_setup (host->device copy of CSR+CSC, y, b, validation, init) + "
                     f"{args.steps} iterations + sgtv_get_image, {dt:.3f} s wall"}


def load_phi_star(args):
    """The recorded converged objective of the workload (a long certified solve,
    written by paper_1601_08201_gb300.phistar), or None."""
    # the BF16-values form rounds A, which moves the minimum: it has its own record
    suffix = "_bf16" if args.precision == "bf16" else ""
    path = args.phi_star or os.path.join(ROOT, "profiles", f"phi_star_{args.workload}{suffix}.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    if rec.get("workload") != args.workload or (rec.get("precision") == "bf16") != (args.precision == "bf16"):
        return None
    rec["path"] = os.path.relpath(path, ROOT)
    return rec


def time_to_tolerance(sgtv, P, args, stream, torch, flags=0, tols=(1e-2, 1e-3, 1e-4), rho=None):
    """Wall time of the plain method (flat start, the workload's rho) until the
    relative objective gap (phi - phi*) / phi* stays within tol, with phi* the
    recorded converged objective. The objective is evaluated every
    `every` iterations and that time is included; a tolerance not reached
    within the trace is reported as not reached, with the final gap."""
    every, trace_iters = args.ttt_every, args.ttt_iters
    rec = load_phi_star(args)
    rho = P.rho if rho is None else rho
    h = sgtv.Handle(P, rho=rho, precision=args.precision, stream=stream.cuda_stream, flags=flags)
    phis = [h.objective()[0]]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    times = [0.0]
    for k in range(every, trace_iters + 1, every):
        h.iterate(every)
        phis.append(h.objective()[0])
        times.append(time.perf_counter() - t0)
    h.close()
    phis = np.array(phis)
    if rec is not None:
        phi_star = float(rec["phi_star"])
        src = (f"{rec['path']}: lowest objective of a {rec['iterations']}-iteration {rec['precision']} solve "
               f"at rho = {rec['rho']} (final primal {rec['primal']:.1e}, dual {rec['dual']:.1e}, kkt "
               f"{rec['kkt']:.1e}, last-tenth spread {rec['tail_rel_spread']:.1e})")
    else:
        phi_star = float(phis.min())
        src = "no recorded phi*: the lowest traced value (gaps are lower bounds of the true gaps)"
    gap = (phis - phi_star) / phi_star
    out = {"phi_star": phi_star, "phi_star_from": src, "rho": rho, "trace_iters": trace_iters,
           "objective_every": every, "includes_objective_evals": True, "final_gap": float(gap[-1]),
           "min_gap": float(gap.min())}
    for tol in tols:
        ok = gap <= tol
        idx = None
        for k in range(len(ok)):  # first evaluation from which every later one stays within tol
            if ok[k:].all():
                idx = k
                break
        if idx is None:
            out[f"{tol:g}"] = {"reached": False,
                               "reason": f"gap {gap[-1]:.2e} after {trace_iters} iterations ({times[-1]:.1f} s)"}
        else:
            out[f"{tol:g}"] = {"reached": True, "iters": int(idx * every), "wall_s": times[idx]}
    return out


if __name__ == "__main__":
    sys.exit(main())
