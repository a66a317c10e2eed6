"""The converged objective phi* of a workload, for time-to-tolerance figures.

The relative objective gap (phi(f^k) - phi*) / phi* needs the minimum of
Eq. 4, phi* = min_f D(f) + beta R(w.G f), f >= 0. It does not depend on the
ADMM penalty rho (Eqs. 5-7): every rho > 0 has the same fixed points, where
the KKT conditions of Eq. 4 hold. So phi* can be computed with whichever rho
converges fastest, and certified by the residuals of sgtv_residuals.

  python -m paper_1601_08201_gb300.phistar --sweep 1,4,16,64 --iters 20000 [--n-inner 1,2,4]
      traces of the objective and the residuals for each rho (and number of
      surrogate steps per iteration; the plain method from the flat start),
      to see which converges fastest
  python -m paper_1601_08201_gb300.phistar --rho R --iters N --out FILE.json
      one long solve at rho = R, the objective every --every iterations;
      records phi* = the lowest objective seen, the final residuals and how
      much the objective still moved over the last tenth of the run

Runs on the GPU through the C ABI (sgtv.Handle); every iteration is the
method's own.
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import sys
import time

import numpy as np

from . import sgtv, synth


def trace(P, rho, iters, every, precision="fp32", flags=None, stream=None, n_inner=1):
    """Objective and residuals of the plain method (flat start) at penalty rho,
    every `every` iterations; wall time of the iterations alone. n_inner:
    surrogate steps (f-updates) per ADMM iteration."""
    if flags is None:
        flags = sgtv.FLAG_SINGLE_PASS | sgtv.FLAG_GRAPH
    with sgtv.Handle(P, rho=rho, precision=precision, flags=flags, stream=stream, n_inner=n_inner) as h:
        rows = [(0, h.objective()[0], *h.residuals(), 0.0)]
        t_iter = 0.0
        done = 0
        while done < iters:
            n = min(every, iters - done)
            t0 = time.perf_counter()
            h.iterate(n)
            h.sync()
            t_iter += time.perf_counter() - t0
            done += n
            phi = h.objective()[0]
            rows.append((done, phi, *h.residuals(), t_iter))
    return np.array(rows)  # iteration, phi, primal, dual, kkt, seconds


def summary(tr):
    it, phi = tr[:, 0], tr[:, 1]
    best = float(phi.min())
    tail = phi[int(0.9 * (len(phi) - 1)):]
    return {"iterations": int(it[-1]), "phi_min": best, "phi_last": float(phi[-1]),
            "tail_rel_spread": float((tail.max() - tail.min()) / best),
            "primal": float(tr[-1, 2]), "dual": float(tr[-1, 3]), "kkt": float(tr[-1, 4]),
            "seconds": float(tr[-1, 5])}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="scale_128x128x64")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "bf16"])
    ap.add_argument("--sweep", default=None, help="comma-separated rho values to trace")
    ap.add_argument("--rho", type=float, default=None, help="rho of the long solve")
    ap.add_argument("--iters", type=int, default=20000)
    ap.add_argument("--every", type=int, default=500)
    ap.add_argument("--out", default=None, help="JSON record of the long solve")
    ap.add_argument("--n-inner", default="1",
                    help="surrogate steps per ADMM iteration; with --sweep, a comma-separated list traced at each rho")
    args = ap.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    P = synth.preset(args.workload)
    stream = torch.cuda.Stream()
    inner = [int(v) for v in args.n_inner.split(",")]
    if args.sweep:
        for rho in [float(v) for v in args.sweep.split(",")]:
            for ni in inner:
                tr = trace(P, rho, args.iters, args.every, args.precision, stream=stream.cuda_stream, n_inner=ni)
                print(json.dumps({"rho": rho, "n_inner": ni, **summary(tr),
                                  "phi_at": {int(r[0]): float(r[1]) for r in tr[:: max(1, len(tr) // 10)]}}),
                      flush=True)
        return 0
    rho = P.rho if args.rho is None else args.rho
    tr = trace(P, rho, args.iters, args.every, args.precision, stream=stream.cuda_stream, n_inner=inner[0])
    s = summary(tr)
    rec = {"workload": args.workload, "precision": args.precision, "rho": rho, "n_inner": inner[0], "beta": P.beta,
           "phi_star": s["phi_min"], **s,
           "command": "python -m paper_1601_08201_gb300.phistar " + " ".join(sys.argv[1:] if argv is None else argv),
           "device": torch.cuda.get_device_name(0),
           "date": datetime.datetime.now(datetime.timezone.utc).strftime("%Y-%m-%dT%H:%M:%SZ"),
           "note": "phi* = lowest objective of a long plain-method solve (flat start, single-pass form, CUDA "
                   "graphs) at the rho given; Eq. 4's minimum does not depend on rho"}
    print(json.dumps(rec), flush=True)
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(rec, fh, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
