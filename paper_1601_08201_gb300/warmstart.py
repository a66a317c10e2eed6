"""Learned warm start for SGTV reconstruction: data, training, evaluation.

The network (include/wsnet.h) maps the normalised backprojection A^T y / A^T 1
(q-bins as channels) plus a count-level channel to a starting image and,
with its dual channels, a starting scaled dual; plain ADMM (Sec. III,
Eqs. 5-7) always finishes the solve and its objective judges the result. All numerical work runs in libsgtv.so's kernels (the solver and
the network); this module only sequences calls and moves arrays.

  python -m paper_1601_08201_gb300.warmstart [--train N] [--eval M] ...
prints one JSON line with the cold-versus-warm comparison.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import sgtv, synth, wsnet


def instrument(Nx=64, Nz=64, Nq=64, nnz_col=128, seed=10000):
    """The system matrix shared by every scan (one measurement per hyper-voxel)."""
    return synth.make_problem(Nx, Nz, Nq, Nx * Nz * Nq, nnz_col, n_regions=4, mean_counts=30.0, seed=seed)


def measurements(P, seeds, workers=8, ahead=32):
    """synth.measure(P, s) for each seed, in order, drawn ahead by a thread
    pool (the sparse product and the Poisson draws release the interpreter
    lock), so the GPU does not wait for the host between scans."""
    import collections
    import concurrent.futures as cf

    seeds = list(seeds)
    with cf.ThreadPoolExecutor(workers) as ex:
        pending = collections.deque()
        it = iter(seeds)
        for s in it:
            pending.append(ex.submit(synth.measure, P, s))
            if len(pending) >= ahead:
                break
        for s in it:
            yield pending.popleft().result()
            pending.append(ex.submit(synth.measure, P, s))
        while pending:
            yield pending.popleft().result()


def to_net_layout(f, Nx, Nz, Nq):
    """J-ordered (x, z, q) vector -> [q][x][z]."""
    return np.ascontiguousarray(np.asarray(f, np.float32).reshape(Nx, Nz, Nq).transpose(2, 0, 1))


class Solver:
    """One resident handle for the instrument; scans swap in their counts.
    rho: the ADMM penalty of this handle (default the instrument's)."""

    def __init__(self, P, torch, flags=sgtv.FLAG_GRAPH, rho=None):
        self.P = P
        self.torch = torch
        self.rho = P.rho if rho is None else float(rho)
        self.stream = torch.cuda.Stream()
        self.h = sgtv.Handle(P, rho=self.rho, stream=self.stream.cuda_stream, flags=flags)

    def load(self, M):
        self.h.set_data(M.y, M.b, M.beta)

    def features(self, M, x_dev):
        """Network input of the loaded scan M into x_dev [Q+1, Nx, Nz] (device):
        the normalised backprojection divided by its mean, then the count
        level. Returns the image scale kappa, the value of the method's flat
        initial image (the state right after loading), which the network's
        targets and outputs are measured in."""
        torch = self.torch
        P = self.P
        kappa = float(np.mean(self.h.get_image()))
        kappa = kappa if kappa > 0 else 1.0
        bp = torch.empty(P.J, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        self.h.normalized_backprojection(bp.data_ptr())
        bmean = float(bp.mean().item())
        bmean = bmean if bmean > 0 else 1.0
        level = float(np.log(max(float(np.mean(M.y)), 1e-3)) / 5.0)
        wsnet.pack_input(bp.data_ptr(), P.Nx, P.Nz, P.Nq, bmean, level, x_dev.data_ptr(), self.stream.cuda_stream)
        self.stream.synchronize()  # bp is released on return
        return kappa

    def solve(self, n_iter):
        self.h.iterate(n_iter)
        return self.h.get_image()

    def trace(self, n_iter, every):
        """(objective after 0, every, 2 every, ... iterations; wall seconds at each)."""
        phis, times = [self.h.objective()[0]], [0.0]
        t0 = time.perf_counter()
        for _ in range(n_iter // every):
            self.h.iterate(every)
            phis.append(self.h.objective()[0])
            times.append(time.perf_counter() - t0)
        return np.array(phis), np.array(times)


def dual_to_net_layout(c, Nx, Nz, Nq, n_dirs):
    """Direction-major J-ordered dual [p][(x, z, q)] -> [p * Nq + q][x][z]."""
    c = np.asarray(c, np.float32).reshape(n_dirs, Nx, Nz, Nq).transpose(0, 3, 1, 2)
    return np.ascontiguousarray(c.reshape(n_dirs * Nq, Nx, Nz))


def build_dataset(solver, seeds, n_iter, torch, n_dual=0, target_solver=None):
    """Inputs [n, Q+1, Nx, Nz], targets [n, Q (1 + n_dual), Nx, Nz] (device), scan
    metadata. The targets are the plain method's image after n_iter iterations
    in units of the flat initial image, then (n_dual > 0) its scaled dual in
    units of the shrink threshold tau = beta / rho. Both are invariant in rho
    at the solution of Eq. 4 (the image is the minimiser; the scaled dual
    over tau is the Lagrange multiplier over beta), so target_solver, a
    handle at a larger penalty that converges faster, may produce them; the
    features still come from `solver`."""
    tsolver = solver if target_solver is None else target_solver
    P = solver.P
    n = len(seeds)
    X = torch.empty((n, P.Nq + 1, P.Nx, P.Nz), dtype=torch.float32, device="cuda")
    T = torch.empty((n, P.Nq * (1 + n_dual), P.Nx, P.Nz), dtype=torch.float32, device="cuda")
    meta = []
    torch.cuda.synchronize()
    for k, (s, M) in enumerate(zip(seeds, measurements(P, seeds))):
        solver.load(M)
        scale = solver.features(M, X[k])
        if tsolver is not solver:
            tsolver.load(M)
        f = tsolver.solve(n_iter)
        T[k, :P.Nq].copy_(torch.from_numpy(to_net_layout(f, P.Nx, P.Nz, P.Nq) / scale))
        if n_dual:
            tau = M.beta / tsolver.rho
            c = tsolver.h.get_state_f64()[2]
            T[k, P.Nq:].copy_(torch.from_numpy(dual_to_net_layout(c / tau, P.Nx, P.Nz, P.Nq, n_dual)))
        meta.append(dict(seed=s, scale=scale))
    torch.cuda.synchronize()
    return X, T, meta


def train(net, X, T, epochs, batch, lr, seed=0, log=None):
    import torch

    rng = np.random.default_rng(seed)
    n = X.shape[0]
    losses = []
    for ep in range(epochs):
        order = rng.permutation(n)
        tot = 0.0
        for b0 in range(0, n - batch + 1, batch):
            sel = torch.as_tensor(order[b0:b0 + batch], device=X.device)
            xb = X.index_select(0, sel).contiguous()
            tb = T.index_select(0, sel).contiguous()
            torch.cuda.synchronize()  # the network runs on its own stream
            tot += net.loss_grad(xb.data_ptr(), tb.data_ptr(), batch)
            net.adam_step(lr * (0.5 * (1 + np.cos(np.pi * ep / epochs))) + 1e-5)
        losses.append(tot / max(1, n // batch))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.5f}")
    return losses


def warm_image(solver, net, M, torch, with_dual=False):
    """The network's starting image for scan M (device tensor, J-ordered);
    with_dual: (image, dual [n_dirs * J]) from a network with dual channels."""
    P = solver.P
    x = torch.empty((1, P.Nq + 1, P.Nx, P.Nz), dtype=torch.float32, device="cuda")
    out = torch.empty((1, net.num_outputs, P.Nx, P.Nz), dtype=torch.float32, device="cuda")
    f0 = torch.empty(P.J, dtype=torch.float32, device="cuda")
    scale = solver.features(M, x[0])
    # three streams take part (torch's, the solver's, the network's): order
    # them on the device between the stages
    torch.cuda.synchronize()
    net.forward(x.data_ptr(), 1, out.data_ptr())
    torch.cuda.synchronize()
    wsnet.unpack_output(out.data_ptr(), P.Nx, P.Nz, P.Nq, scale, f0.data_ptr(), solver.stream.cuda_stream)
    if with_dual:
        c0 = torch.empty(P.J * net.n_dual, dtype=torch.float32, device="cuda")
        wsnet.unpack_dual(out.data_ptr(), P.Nx, P.Nz, P.Nq, net.n_dual, M.beta / solver.rho, c0.data_ptr(),
                          solver.stream.cuda_stream)
        torch.cuda.synchronize()
        return f0, c0
    torch.cuda.synchronize()
    return f0


def iters_to_tol(phis, times, phi_star, every, tol=1e-4):
    """First evaluation from which the relative gap stays <= tol (None if never)."""
    gap = (phis - phi_star) / phi_star
    ok = gap <= tol
    for k in range(len(ok)):
        if ok[k:].all():
            return k * every, float(times[k])
    return None, None


def checkpoints(n_iter, every):
    """Iteration counts at which the objective gaps are also reported."""
    return [m for m in (100, 300, 1000, 3000, 10000, 30000) if m <= n_iter and m % every == 0]


def evaluate(solver, net, seeds, n_iter, every, torch, star_iters=20000, starts=(("warm", 1.0),),
             tols=(1e-3, 1e-4), star_solver=None):
    """Flat start ("cold") against the network's start on held-out scans.

    Each entry (name, mode) of `starts` runs plain ADMM from f0 = the
    network's image and d = w.G f0, with c from the dual rule of
    sgtv_warm_start scaled by mode (a number) or, for mode "net", the
    network's own dual channels (sgtv_warm_start_dual; "net:theta" scales
    them by theta). phi* is the lowest objective seen by a long cold solve of
    star_iters iterations (on star_solver, a handle at a larger penalty that
    converges faster to the same minimum, when given) and by every traced run.
    For each tolerance the row holds the iterations (and wall seconds, the
    network's time included for warm starts) after which the relative gap
    stays below it."""
    rows = []
    ssolver = solver if star_solver is None else star_solver
    seeds = list(seeds)
    for s, M in zip(seeds, measurements(solver.P, seeds)):
        ssolver.load(M)
        ssolver.h.iterate(star_iters)
        phi_long = ssolver.h.objective()[0]
        solver.load(M)
        traces = {"cold": solver.trace(n_iter, every) + (0.0,)}
        for name, mode in starts:
            solver.load(M)
            t0 = time.perf_counter()
            if isinstance(mode, str) and mode.startswith("net"):
                f0, c0 = warm_image(solver, net, M, torch, with_dual=True)
                if ":" in mode:  # "net:theta": the network's dual scaled by theta
                    c0.mul_(float(mode.split(":")[1]))
                    torch.cuda.synchronize()
                solver.h.warm_start_dual(f0.data_ptr(), c0.data_ptr())
            else:
                f0 = warm_image(solver, net, M, torch)
                solver.h.warm_start(f0.data_ptr(), mode)
            t_net = time.perf_counter() - t0
            traces[name] = solver.trace(n_iter, every) + (t_net,)
        phi_star = min([phi_long] + [float(tr[0].min()) for tr in traces.values()])
        row = dict(seed=s, phi_star=float(phi_star))
        for name, (phis, times, t_net) in traces.items():
            row[f"{name}_start_gap"] = float((phis[0] - phi_star) / phi_star)
            for m in checkpoints(n_iter, every):
                row[f"{name}_gap@{m}"] = float((phis[m // every] - phi_star) / phi_star)
            row[f"{name}_net_s"] = t_net
            for tol in tols:
                it, sec = iters_to_tol(phis, times, phi_star, every, tol)
                row[f"{name}_iters@{tol:g}"] = it
                row[f"{name}_s@{tol:g}"] = None if sec is None else sec + t_net
        rows.append(row)
    return rows


def summarize(rows, names=("warm",), tols=(1e-3, 1e-4)):
    """Per tolerance and start: scans that reached it, mean iterations and wall
    seconds over the scans where both that start and the cold start did, and
    the ratios to cold."""
    out = dict(n=len(rows))
    for name in ("cold",) + tuple(names):
        out[f"{name}_start_gap_median"] = float(np.median([r[f"{name}_start_gap"] for r in rows]))
    # median objective gap after m iterations, and the median of warm / cold per scan
    ms = sorted({int(k.split("@")[1]) for k in rows[0] if k.startswith("cold_gap@")}) if rows else []
    for m in ms:
        out[f"cold_gap@{m}_median"] = float(np.median([r[f"cold_gap@{m}"] for r in rows]))
        for name in names:
            out[f"{name}_gap@{m}_median"] = float(np.median([r[f"{name}_gap@{m}"] for r in rows]))
            out[f"{name}_over_cold_gap@{m}_median"] = float(np.median(
                [r[f"{name}_gap@{m}"] / max(r[f"cold_gap@{m}"], 1e-300) for r in rows]))
    for tol in tols:
        t = f"{tol:g}"
        for name in names:
            ok = [r for r in rows if r[f"cold_iters@{t}"] is not None and r[f"{name}_iters@{t}"] is not None]
            key = f"{name}@{t}"
            if not ok:
                out[key] = dict(reached=0)
                continue
            ci = np.array([r[f"cold_iters@{t}"] for r in ok], float)
            wi = np.array([r[f"{name}_iters@{t}"] for r in ok], float)
            cs = np.array([r[f"cold_s@{t}"] for r in ok], float)
            ws = np.array([r[f"{name}_s@{t}"] for r in ok], float)
            out[key] = dict(reached=len(ok), cold_reached=sum(r[f"cold_iters@{t}"] is not None for r in rows),
                            warm_reached=sum(r[f"{name}_iters@{t}"] is not None for r in rows),
                            cold_iters_mean=float(ci.mean()), warm_iters_mean=float(wi.mean()),
                            iters_ratio=float(wi.mean() / max(ci.mean(), 1.0)), cold_s_mean=float(cs.mean()),
                            warm_s_mean=float(ws.mean()), wall_ratio=float(ws.mean() / max(cs.mean(), 1e-9)),
                            warm_fewer_frac=float(np.mean(wi < ci)))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--shape", default="64,64,64")
    ap.add_argument("--nnz-col", type=int, default=128)
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--eval", type=int, default=200)
    ap.add_argument("--target-iters", type=int, default=1500)
    ap.add_argument("--eval-iters", type=int, default=3000)
    ap.add_argument("--star-iters", type=int, default=20000)
    ap.add_argument("--with-c0", action="store_true", help="also run the network start with c = 0")
    ap.add_argument("--dual", action="store_true",
                    help="train the dual channels too and start from the network's image and dual")
    ap.add_argument("--dual-scales", type=float, nargs="*", default=[],
                    help="also start from the network's dual scaled by each of these factors")
    ap.add_argument("--target-rho", type=float, default=None,
                    help="ADMM penalty of the target and phi* solves (default: the instrument's); the "
                         "targets and phi* do not depend on it, a larger one converges faster")
    ap.add_argument("--eval-rho", type=float, default=None,
                    help="ADMM penalty of the cold and warm evaluation solves (default: the instrument's)")
    ap.add_argument("--every", type=int, default=10)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    args = ap.parse_args(argv)
    import torch

    torch.cuda.set_device(0)
    Nx, Nz, Nq = (int(v) for v in args.shape.split(","))
    t0 = time.perf_counter()
    P = instrument(Nx, Nz, Nq, args.nnz_col)
    flags = sgtv.FLAG_GRAPH | sgtv.FLAG_SINGLE_PASS
    solver = Solver(P, torch, flags=flags, rho=args.eval_rho)
    tsolver = Solver(P, torch, flags=flags, rho=args.target_rho) if args.target_rho else None
    n_dual = 4 if args.dual else 0
    X, T, _ = build_dataset(solver, range(10000, 10000 + args.train), args.target_iters, torch, n_dual=n_dual,
                            target_solver=tsolver)
    t_data = time.perf_counter() - t0
    net = wsnet.WarmNet(Nx, Nz, Nq, args.batch, seed=0, n_dual=n_dual)
    t1 = time.perf_counter()
    losses = train(net, X, T, args.epochs, args.batch, args.lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    starts = (("warm_c0", 0.0),) if args.dual else (("warm", 1.0),)
    if args.dual:
        starts = (("warm_dual", "net"),) + tuple((f"warm_dual_{t:g}", f"net:{t:g}") for t in args.dual_scales) \
            + starts
    elif args.with_c0:
        starts = starts + (("warm_c0", 0.0),)
    rows = evaluate(solver, net, range(20000, 20000 + args.eval), args.eval_iters, args.every, torch,
                    star_iters=args.star_iters, starts=starts, star_solver=tsolver)
    out = dict(shape=[Nx, Nz, Nq], train=args.train, eval=args.eval, params=net.num_params,
               rho=solver.rho, target_rho=args.target_rho or solver.rho,
               target_iters=args.target_iters, eval_iters=args.eval_iters, star_iters=args.star_iters,
               data_s=round(t_data, 1), train_s=round(t_train, 1), loss_first=losses[0], loss_last=losses[-1],
               summary=summarize(rows, tuple(n for n, _ in starts)))
    print(json.dumps(out), flush=True)
    return out


if __name__ == "__main__":
    main()
