"""Long-run statistics of the channel (the relative viscosity and the
near-wall hematocrit / cell-free layer that Sec. 4 reports for vessels).

Beyond a few hundred steps the cell trajectories of two runs diverge (the
dynamics is chaotic), so long runs are judged on time averages:
  - eta_rel = Q_0 / Q_H, the flow rate of plain plasma over that of the
    suspension at the same uniform drive; the work rate of the drive P =
    G_x sum_x u_x = G_x n_x Q (rbc_stats().power) gives it as P_0 / P_H;
  - the near-wall hematocrit profile: cell-centre counts in 1-lattice-unit
    bins of y (rbc_profile), time-averaged.
Both come out the same, within 1 %, with FP32 populations and with binary16
populations (stochastic rounding) on a reduced channel (32 x 40 x 64, 228
cells in the channel workload's slot lattice, hematocrit 0.28 of the box,
wall shear rate 5e-4, seed 1107_4889 + 2; 6,000 steps, sampled every 50
steps over the second half).  The anchor: over a
short window (200 steps, samples every 20 from step 100) the GPU's FP32
statistics equal the oracle's, the work rate to 1e-5 and the profile to
the count.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1107_4889_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

NX, NY, NZ, NCELLS, RATE = 32, 40, 64, 228, 5e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_4889_gb300 import build
    build.build()


def _channel(cells=True):
    G = 2.0 * (1.0 / 6.0) * RATE / (NY - 2)
    geom, c, params = wl.channel_workload(nx=NX, ny=NY, nz=NZ, ncells=NCELLS, body_force=(G, 0.0, 0.0),
                                          seed=wl.SEED_BASE + 2)
    return geom, (c if cells else None), params


def _gpu_stats(geom, cells, params, steps, every, start):
    from paper_1107_4889_gb300.rbc import Solver
    s = Solver(geom, cells, params)
    powers = []
    done = 0
    while done < steps:
        s.step(every)
        done += every
        if done >= start:
            powers.append(s.stats()["power"])
            if cells is not None:
                s.profile_accumulate(1)
    prof = s.profile()[0] if cells is not None else None
    s.close()
    return float(np.mean(powers)), prof


def test_relative_viscosity_and_wall_profile_fp32_vs_binary16():
    steps, every = 6000, 50
    out = {}
    for prec in ("f32", "f16"):
        g0, _, p = _channel(cells=False)
        P0, _ = _gpu_stats(g0, None, dict(p, precision=prec), steps, every, steps // 2)
        g, c, p = _channel()
        PH, prof = _gpu_stats(g, c, dict(p, precision=prec), steps, every, steps // 2)
        out[prec] = (P0 / PH, prof)
    eta32, prof32 = out["f32"]
    eta16, prof16 = out["f16"]
    l1 = np.abs(prof16 - prof32).sum() / prof32.sum()
    print(f"eta_rel FP32 {eta32:.5f} binary16 {eta16:.5f} ({eta16 / eta32 - 1:+.2e}); profile L1 {l1:.2e}")
    print("near-wall profile (cells per 1-lu bin, y = 0..9):", np.round(prof32[:10], 3))
    assert eta32 > 1.0  # the suspension is more viscous than its plasma
    assert abs(eta16 / eta32 - 1.0) < 0.01
    assert l1 < 0.01
    assert prof32[:2].sum() == 0.0 and prof32[-2:].sum() == 0.0  # no centre inside the wall layers
    assert abs(prof32.sum() - NCELLS) < 1e-9 and abs(prof16.sum() - NCELLS) < 1e-9


def test_statistics_anchor_oracle_short_window():
    g, c, p = _channel()
    steps, every, start = 200, 20, 100
    o = orc.Oracle(g, c, p)
    powers, prof = [], np.zeros(NY)
    done = 0
    while done < steps:
        o.step(every)
        done += every
        if done >= start:
            powers.append(o.budget()["power"])
            y = o.cells()["pos"][:, 1]
            prof += np.bincount(np.floor(y).astype(int), minlength=NY)[:NY]
    o.close()
    P_o, prof_o = float(np.mean(powers)), prof / len(powers)
    P_g, prof_g = _gpu_stats(g, c, p, steps, every, start)
    print(f"work rate GPU {P_g:.8e} oracle {P_o:.8e}; profile diff {np.abs(prof_g - prof_o).sum():.3g}")
    assert abs(P_g / P_o - 1.0) <= 1e-5
    assert np.abs(prof_g - prof_o).sum() * len(powers) <= 1.0
