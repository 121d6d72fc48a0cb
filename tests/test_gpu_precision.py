"""GPU parity of the 16-bit population storage (binary16 / bfloat16 scaled
deviations, FP32 collision) against the oracle.

Two references:
  - the oracle with the same storage step (same format, same rounding, the
    same Philox4x32-10 random bits): the two differ only where FP32 and FP64
    arithmetic put a value on different sides of a rounding threshold, an
    event of probability ~|x32 - x64| / q ~ 1e-4 (binary16) or ~1e-5
    (bfloat16) per stored value that moves it by one format step q (2^-10 or
    2^-7 of the value); over 100 steps that accumulates to ~1e-4 / ~3e-4 of
    the velocity.  Bound: 2e-3;
  - the exact FP64 oracle: the storage error itself.  Stochastic rounding
    adds zero-mean noise of about q / 2.4 per stored value and step; the
    momentum it carries random-walks, ~10x the per-step error after 100
    steps: ~5e-3 (binary16), ~4e-2 (bfloat16) of the velocity.  Bounds 2e-2
    and 1.5e-1, and the measured values are printed.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1107_4889_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SEED = 20110723


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_4889_gb300 import build
    build.build()


def _solver(geom, cells, params):
    from paper_1107_4889_gb300.rbc import Solver
    return Solver(geom, cells, params)


def rel_l2(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


TOL_EMULATED = 2e-3
TOL_EXACT = {"f16": 2e-2, "bf16": 1.5e-1}


def _run(geom, cells, params, prec, rounding, steps):
    stochastic = rounding == "stochastic"
    gp = dict(params, precision=prec, rounding=rounding, seed=SEED)
    s = _solver(geom, cells, gp)
    o = orc.Oracle(geom, cells, params, storage=prec, stochastic=stochastic, seed=SEED)
    e = orc.Oracle(geom, cells, params)
    s.step(steps)
    o.step(steps)
    e.step(steps)
    f = s.fields()
    rho_o, u_o, _ = o.fields()
    rho_e, u_e, _ = e.fields()
    fluid = np.ones(o.N, bool) if geom["solid"] is None else geom["solid"].reshape(-1) == 0
    # rho - 1 is tiny in these flows (~1e-8): its error is measured against
    # the velocity scale (both are Mach-number-sized in lattice units)
    out = dict(u_emul=rel_l2(f["u"][fluid], u_o[fluid]), u_exact=rel_l2(f["u"][fluid], u_e[fluid]),
               rho_emul=rel_l2(f["rho"][fluid], rho_o[fluid]),
               drho_emul=np.linalg.norm(f["rho"][fluid] - rho_o[fluid]) / np.linalg.norm(u_o[fluid]),
               oracle16_vs_exact=rel_l2(u_o[fluid], u_e[fluid]))
    if o.n:
        dg, do = s.cell_diag(), o.diag()
        for k in ("J", "F_mech", "u_s"):
            scale = np.abs(do[k]).max()
            out[k + "_emul"] = np.abs(dg[k] - do[k]).max() / scale if scale > 0 else 0.0
    s.close()
    o.close()
    e.close()
    return out


@pytest.mark.parametrize("prec", ["f16", "bf16"])
@pytest.mark.parametrize("rounding", ["stochastic", "nearest"])
def test_box32_storage_parity(prec, rounding):
    """The 32^3 box with 32 cells, 100 steps, against both references."""
    geom, cells, params = wl.box_workload()
    r = _run(geom, cells, params, prec, rounding, 100)
    print(prec, rounding, r)
    assert r["u_emul"] <= TOL_EMULATED and r["drho_emul"] <= TOL_EMULATED and r["rho_emul"] <= 1e-5
    assert r["J_emul"] <= 5 * TOL_EMULATED and r["u_s_emul"] <= TOL_EMULATED
    assert r["u_exact"] <= TOL_EXACT[prec]


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_ragged_walled_lattice_storage(prec):
    """17 x 19 x 23 with walls and an obstacle (rows of 34 bytes: the
    one-thread-per-node pass) and the 24 x 28 x 32 walled channel with cells
    (the row-staged pass)."""
    geom = wl.plane_channel(17, 19, 23, body_force=(2e-6, 0.0, 1e-6))
    geom["solid"][5:9, 7:10, 6:9] = 1
    r = _run(geom, None, wl.params(), prec, "stochastic", 120)
    print(prec, "ragged", r)
    assert r["u_emul"] <= TOL_EMULATED and r["u_exact"] <= TOL_EXACT[prec]
    geom, cells, params = wl.channel_workload(nx=24, ny=28, nz=32, ncells=12, body_force=(5e-6, 0, 0), seed=33)
    r = _run(geom, cells, params, prec, "stochastic", 80)
    print(prec, "channel", r)
    assert r["u_emul"] <= TOL_EMULATED and r["u_exact"] <= TOL_EXACT[prec]
    assert r["J_emul"] <= 5 * TOL_EMULATED


def test_full_size_channel_binary16_matches_emulating_oracle():
    """The 64 x 64 x 256 channel with 3,650 cells in binary16: the row-staged
    pass stages two nodes per consumer thread on a lattice this size; 4
    steps against the oracle with the same storage step."""
    geom, cells, params = wl.channel_workload()
    r = _run(geom, cells, params, "f16", "stochastic", 4)
    print("f16 full-size channel", r)
    assert r["u_emul"] <= TOL_EMULATED and r["J_emul"] <= 5 * TOL_EMULATED


def test_rest_state_and_uniform_force_storage():
    """A fluid at rest stays exactly at rest in every format; under a
    uniform force the mean velocity of pass n is (n + 1/2) G to within the
    storage noise (momentum is carried by the stored deviations)."""
    geom = wl.periodic_box(16, 8, 24)
    for prec in ("f16", "bf16"):
        s = _solver(geom, None, wl.params(precision=prec, seed=SEED))
        s.step(10)
        f = s.fields()
        assert np.all(f["u"] == 0.0) and np.all(f["rho"] == 1.0)
        s.close()
    G = np.array([1e-5, -2e-5, 5e-6])
    geom = wl.periodic_box(16, 8, 24, body_force=tuple(G))
    for prec, tol in (("f16", 2e-3), ("bf16", 1.5e-2)):
        s = _solver(geom, None, wl.params(precision=prec, seed=SEED))
        s.step(50)
        f = s.fields()
        assert np.allclose(f["u"].mean(axis=0), 49.5 * G, rtol=tol), (prec, f["u"].mean(axis=0) / (49.5 * G))
        s.close()
