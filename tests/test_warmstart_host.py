"""Host-side helpers of the warm-start driver (no GPU): the layouts between
the solver's hyper-voxel order and the network's channels, the tolerance
crossing and the summary statistics."""
import numpy as np
import pytest

from paper_1601_08201_gb300 import synth, warmstart as WS


def test_image_and_dual_layouts():
    Nx, Nz, Nq, nd = 3, 5, 4, 4
    rng = np.random.default_rng(1)
    f = rng.random(Nx * Nz * Nq)
    c = rng.standard_normal(nd * Nx * Nz * Nq)
    F = WS.to_net_layout(f, Nx, Nz, Nq)
    C = WS.dual_to_net_layout(c, Nx, Nz, Nq, nd)
    assert F.shape == (Nq, Nx, Nz) and C.shape == (nd * Nq, Nx, Nz)
    J = Nx * Nz * Nq
    for x in range(Nx):
        for z in range(Nz):
            for q in range(Nq):
                j = (x * Nz + z) * Nq + q
                assert F[q, x, z] == np.float32(f[j])
                for p in range(nd):
                    assert C[p * Nq + q, x, z] == np.float32(c[p * J + j])


def test_iters_to_tol_needs_the_gap_to_stay_below():
    phis = np.array([10.0, 2.0, 1.0005, 1.02, 1.00005, 1.00001, 1.0])
    times = np.arange(len(phis)) * 0.5
    assert WS.iters_to_tol(phis, times, 1.0, 10, tol=1e-3) == (40, 2.0)  # 1.0005 at 20 does not stay
    assert WS.iters_to_tol(phis, times, 1.0, 10, tol=1e-6) == (60, 3.0)
    assert WS.iters_to_tol(phis + 1.0, times, 1.0, 10, tol=1e-3) == (None, None)


def test_checkpoints_and_summary():
    assert WS.checkpoints(3000, 10) == [100, 300, 1000, 3000]
    assert WS.checkpoints(1000, 300) == [300]
    rows = [dict(seed=s, cold_start_gap=1.0, warm_start_gap=0.5, **{"cold_gap@100": 0.2, "warm_gap@100": 0.1,
             "cold_iters@0.001": 100 * (s + 1), "warm_iters@0.001": 50 * (s + 1),
             "cold_s@0.001": 1.0 * (s + 1), "warm_s@0.001": 0.6 * (s + 1)}) for s in range(3)]
    out = WS.summarize(rows, ("warm",), (1e-3,))
    assert out["warm_over_cold_gap@100_median"] == pytest.approx(0.5)
    assert out["warm_start_gap_median"] == 0.5
    t = out["warm@0.001"]
    assert t["reached"] == 3 and t["iters_ratio"] == pytest.approx(0.5) and t["wall_ratio"] == pytest.approx(0.6)
    assert t["warm_fewer_frac"] == 1.0


def test_measurements_prefetch_keeps_order():
    # the thread-pool prefetch yields exactly synth.measure(P, s) for each seed, in order
    P = synth.make_problem(4, 3, 5, 48, 10, n_regions=2, mean_counts=30.0, seed=3)
    seeds = list(range(100, 137))
    got = list(WS.measurements(P, seeds, workers=4, ahead=5))
    assert len(got) == len(seeds)
    for s, M in zip(seeds, got):
        ref = synth.measure(P, s)
        assert np.array_equal(M.y, ref.y) and M.beta == ref.beta and M.seed == s
