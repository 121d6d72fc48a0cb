"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (FP32 storage and arithmetic on the lattice, FP64 cell state):
  - velocity and density: relative L2 <= 1e-5 after up to 100 steps;
  - per-cell force, torque and impulses: relative (to the largest value over
    the cells) <= 1e-5; the rotational quantities (smeared vorticity,
    elongational torque, angular impulse, orientation) relative to the larger
    of their own largest value and the value a velocity gradient |u~| / xi_min
    would give them (see _rotational_floors);
  - positions: relative to how far the cells moved;
  - cell-pair candidate lists: bit-exact.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as orc
from paper_1107_4889_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-5


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


def _rotational_floors(do, params, steps):
    """Floors of the rotational quantities.  They are differences of the
    FP32-stored fluid state (curl of u, non-equilibrium stress), which FP32
    populations resolve only to ~1e-7 of the velocity; in a nearly uniform
    flow their true values sit at that noise.  Each is therefore compared
    with the larger of its own largest value and the value a velocity
    gradient |u~| / xi_min across the support would give it."""
    grad = np.abs(do["u_s"]).max() / min(params["xi"])
    nu0 = (params["tau0"] - 0.5) / 3.0
    return {"omega_s": grad,
            "T_S": params["alpha_tt"] * nu0 * grad * max(params["xi"]),
            "L": params["gamma_R"] * max(params["inertia"]) * grad,
            "angle": steps * grad}


def _compare(geom, cells, params, steps, tol=TOL, check_cells=True, floors=True, schedule=None):
    """Run both for `steps` and compare.  floors=False judges the rotational
    quantities on their own largest value alone (for flows whose gradients
    lift them far above the FP32 noise).  schedule: (split_spread,
    lattice_first) set on the solver before its steps."""
    o = orc.Oracle(geom, cells, params)
    s = _solver(geom, cells, params)
    if schedule is not None:
        s.set_schedule(*schedule)
    o.step(steps)
    s.step(steps)
    rho_o, u_o, _ = o.fields()
    f = s.fields()
    fluid = np.ones(o.N, bool) if geom["solid"] is None else geom["solid"].reshape(-1) == 0
    err_u = rel_l2(f["u"][fluid], u_o[fluid])
    err_rho = rel_l2(f["rho"][fluid], rho_o[fluid])
    assert err_u <= tol, f"u rel-L2 {err_u:.3e}"
    assert err_rho <= tol, f"rho rel-L2 {err_rho:.3e}"
    # rho - 1: the GPU sums 19 FP32 deviations of size ~|u|, so its error is
    # ~1e-7 |u| whatever the size of rho - 1 (in a slow flow rho - 1 ~ u^2
    # sits near that noise); judged against the velocity scale
    drho_err = np.linalg.norm((f["rho"][fluid] - 1.0) - (rho_o[fluid] - 1.0))
    err_drho_u = drho_err / max(np.linalg.norm(u_o[fluid]), 1e-300)
    assert err_drho_u <= tol, f"rho - 1 error / |u| {err_drho_u:.3e}"
    out = dict(err_u=err_u, err_rho=err_rho, err_drho_u=err_drho_u,
               err_drho=rel_l2(f["rho"][fluid] - 1.0, rho_o[fluid] - 1.0))
    if check_cells and o.n:
        dg, do = s.cell_diag(), o.diag()
        fl = _rotational_floors(do, params, steps) if floors else {"angle": 0.0}
        for k in ("J", "L", "F_mech", "tau_mech", "T_S", "u_s", "omega_s"):
            scale = max(np.abs(do[k]).max(), fl.get(k, 0.0))
            out["scale_" + k] = "own" if scale == np.abs(do[k]).max() else "floor"
            if scale == 0:
                assert np.abs(dg[k]).max() == 0, k
                continue
            e = np.abs(dg[k] - do[k]).max() / scale
            assert e <= tol, f"{k}: {e:.3e}"
            out["err_" + k] = e
        co = o.cells()
        dims = np.array([geom["nx"], geom["ny"], geom["nz"]], float)

        def mi(d):
            return d - dims * np.round(d / dims) * np.asarray(geom["periodic"])

        # positions and orientations: error relative to how far the cells moved
        disp = np.abs(mi(co["pos"] - np.asarray(cells["pos"]))).max()
        assert np.abs(mi(f["pos"] - co["pos"])).max() <= tol * disp + 1e-12
        Qg = Rotation.from_quat(f["quat"][:, [1, 2, 3, 0]])
        Qo = Rotation.from_matrix(co["Q"])
        Q0 = Rotation.from_quat(np.asarray(cells["quat"])[:, [1, 2, 3, 0]])
        turned = max((Qo * Q0.inv()).magnitude().max(), fl["angle"])
        assert (Qg * Qo.inv()).magnitude().max() <= tol * turned
        vs = np.abs(co["vel"]).max()
        assert np.abs(f["vel"] - co["vel"]).max() <= tol * max(vs, 1e-30)
        out["err_pos"] = np.abs(mi(f["pos"] - co["pos"])).max() / max(disp, 1e-30)
    s.close()
    o.close()
    return out


def test_fluid_only_uniform_force_matches_closed_form_and_oracle():
    geom = wl.periodic_box(16, 12, 20, body_force=(1e-5, -2e-5, 5e-6))
    s = _solver(geom, None, wl.params())
    s.step(50)
    f = s.fields()
    G = np.array([1e-5, -2e-5, 5e-6])
    # pass n (from 0) reports u = (n + 1/2) G: 49.5 G after 50 passes
    assert np.allclose(f["u"], 49.5 * G, rtol=2e-6)
    s.close()
    _compare(geom, None, wl.params(), 50)


def test_ragged_lattice_and_walls_fluid_only():
    """17 x 19 x 23 nodes (not a multiple of the block size) with solid walls
    and an obstacle, driven flow, 120 steps."""
    geom = wl.plane_channel(17, 19, 23, body_force=(2e-6, 0.0, 1e-6))
    geom["solid"][5:9, 7:10, 6:9] = 1
    _compare(geom, None, wl.params(), 120)


def test_coupled_periodic_box_32_cells_100_steps():
    """The 32^3 box with 32 cells (hematocrit 9.8 %), force 1e-6 along x."""
    geom, cells, params = wl.box_workload()
    r = _compare(geom, cells, params, 100)
    print("box32:", r)


def test_coupled_box_with_cell_velocities_and_contacts():
    """Cells start with velocities towards each other so Gay-Berne forces act."""
    geom, cells, params = wl.box_workload(n=24, ncells=8, body_force=(0, 0, 0), seed=21)
    rng = np.random.default_rng(4)
    cells["vel"] = rng.normal(size=(8, 3)) * 0.01
    cells["omega"] = rng.normal(size=(8, 3)) * 1e-3
    r = _compare(geom, cells, dict(params, eps0=0.01), 60)
    print("contacts:", r)


def test_coupled_walled_channel():
    geom, cells, params = wl.channel_workload(nx=24, ny=28, nz=32, ncells=12, body_force=(5e-6, 0, 0), seed=33)
    rng = np.random.default_rng(5)
    cells["vel"] = rng.normal(size=(12, 3)) * 3e-3  # drive some cells into the walls
    r = _compare(geom, cells, params, 80)
    print("channel:", r)


def test_coupled_sheared_box_rotational_quantities_without_floor():
    """Kolmogorov shear (force A sin(2 pi y / n) along x, peak shear rate
    2e-3) in a 32^3 box with 12 cells: the cells spin and tilt, so the
    smeared vorticity, the elongational torque, the angular impulse and the
    rotation angle are far above the FP32 noise and are judged against
    their own largest value, with no floor."""
    n = 32
    geom, cells, params = wl.box_workload(n=n, ncells=12, body_force=(0, 0, 0), seed=31)
    geom["body_force_wave"] = (wl.kolmogorov_amplitude(n, 2e-3), 0.0, 0.0)
    r = _compare(geom, cells, params, 100, floors=False)
    print("sheared box:", r)
    for k in ("omega_s", "T_S", "L", "u_s", "J"):
        assert r["scale_" + k] == "own"


def test_stats_match_oracle_budget():
    """rbc_stats (FP64 device reductions) against the oracle's budget after
    100 coupled steps of the 32^3 box: mass, fluid and cell momentum, and
    the work rate of the drive."""
    geom, cells, params = wl.box_workload()
    o = orc.Oracle(geom, cells, params)
    s = _solver(geom, cells, params)
    o.step(100)
    s.step(100)
    bo, bg = o.budget(), s.stats()
    s.close()
    o.close()
    assert bg["step"] == 100
    assert abs(bg["mass"] - bo["mass"]) <= 1e-9 * bo["mass"]
    for k in ("p_fluid", "p_cells"):
        sc = np.abs(bo[k]).max()
        assert sc > 0 and np.abs(bg[k] - bo[k]).max() <= TOL * sc, (k, bg[k], bo[k])
    assert abs(bg["power"] - bo["power"]) <= TOL * abs(bo["power"]), (bg["power"], bo["power"])
    # the drive's momentum input: N_fluid G per step, in both
    N = geom["nx"] * geom["ny"] * geom["nz"]
    ptot = bo["p_fluid"][0] + bo["p_cells"][0]
    assert abs(ptot - 100 * N * geom["body_force"][0]) <= 1e-9 * ptot


def test_single_cell_across_periodic_boundary():
    geom = wl.periodic_box(20, body_force=(0, 3e-6, 0))
    cells = wl.cells_dict(np.array([[19.6, 0.3, 10.2]]), np.array([[0.3, 0.8, -0.2, 0.4]]))
    cells["vel"] = np.array([[1e-3, -2e-3, 5e-4]])
    _compare(geom, cells, wl.params(), 60)


def test_no_alpha_and_no_viscosity_contrast():
    geom, cells, params = wl.box_workload(n=24, ncells=6, seed=9)
    _compare(geom, cells, dict(params, alpha_tt=0.0, delta=0.0), 40)


def test_neighbor_lists_bit_exact():
    """Dense random positions plus pairs placed at the candidate radius to
    within rounding; eps0 = 0 so the overlapping cells exert no force."""
    rng = np.random.default_rng(17)
    L = 48
    geom = wl.periodic_box(L)
    n = 400
    pos = rng.random((n, 3)) * L
    rc = wl.PAPER_PARAMS["r_cut"]
    for k in range(20):  # pairs within an ulp or so of r_cut
        dirn = rng.normal(size=3)
        dirn /= np.linalg.norm(dirn)
        pos[2 * k + 1] = np.mod(pos[2 * k] + dirn * rc * (1 + (k % 5 - 2) * 1e-16), L)
    pos[pos >= L] -= L
    cells = wl.cells_dict(pos, wl.random_quaternions(rng, n))
    params = wl.params(eps0=0.0, bin_capacity=64, max_neighbors=128)
    o = orc.Oracle(geom, cells, params)
    ref = {tuple(p) for p in o.neighbor_pairs()}
    s = _solver(geom, cells, params)
    s.step(1)
    lists = s.neighbors(128)
    got = set()
    for i, lst in enumerate(lists):
        assert np.all(np.diff(lst) > 0)
        for j in lst:
            got.add((min(i, j), max(i, j)))
            assert i in lists[j]
    assert got == ref and len(ref) > 100


def test_momentum_budget_on_gpu():
    geom, cells, params = wl.box_workload(n=24, ncells=6, body_force=(0, 0, 0), seed=5)
    rng = np.random.default_rng(1005)
    cells["vel"] = rng.normal(size=(6, 3)) * 1e-3
    s = _solver(geom, cells, params)
    b0 = s.stats()
    P0 = b0["p_fluid"] + b0["p_cells"]
    scale = np.abs(cells["vel"]).sum() * params["mass"]
    s.step(50)
    b = s.stats()
    assert abs(b["mass"] - b0["mass"]) < 1e-6 * b0["mass"]
    assert np.allclose(b["p_fluid"] + b["p_cells"], P0, atol=1e-5 * scale)
    assert np.abs(b["p_fluid"]).max() > 1e-3 * scale


def test_instability_flag_is_reported():
    """A body force far beyond the stability bound (|F| ~ 0.1 of Sec. 3)
    trips the Mach guard; the guard reports on the host, nothing faults."""
    from paper_1107_4889_gb300.rbc import RbcError, RBC_EUNSTABLE
    geom = wl.periodic_box(8, body_force=(0.05, 0, 0))
    s = _solver(geom, None, wl.params())
    s.step(20)
    with pytest.raises(RbcError) as e:
        s.stats()
    assert e.value.code == RBC_EUNSTABLE


def test_full_size_channel_sampled_against_oracle():
    """The 64 x 64 x 256 channel with 3,650 cells in the launch
    configuration the benchmark times: 6 steps compared with the oracle on
    every field and every cell."""
    geom, cells, params = wl.channel_workload()
    cells["vel"] = np.random.default_rng(2).normal(size=(len(cells["pos"]), 3)) * 1e-3
    r = _compare(geom, cells, params, 6)
    print("channel full size:", r)


def test_autotuned_launch_shape_keeps_parity():
    """The autotuner times the lattice pass's launch shapes on the live
    solve; whatever it picks, the results stay those of the oracle (a node's
    update does not depend on which CTA computes it)."""
    geom, cells, params = wl.box_workload()
    s = _solver(geom, cells, params)
    rep = s.autotune(4)
    # every shape in both graph orders, five grids of the side kernels, and
    # the coarser particle-bin grids (32^3: 2 x 2 x 2 and 1 x 1 x 1 bins)
    assert rep["trials"] >= 9
    assert rep["ms_per_step"] <= rep["default_ms_per_step"]
    assert rep["bin_scale"] in (1.0, 1.5, 2.0)
    s.step(6)
    n = s.stats()["step"]
    assert n == 4 * 2 * (rep["trials"] + 1) + 6
    o = orc.Oracle(geom, cells, params)
    o.step(n)
    f = s.fields()
    _, u_o, _ = o.fields()
    assert rel_l2(f["u"], u_o) <= TOL
    s.close()
    o.close()


@pytest.mark.parametrize("lattice_first", [False, True])
def test_split_spread_schedule_matches_oracle(lattice_first):
    """The spread as a kernel of its own, the next step's cell-side kernels
    beside it, in either graph order: the coupled walled channel stays at
    the oracle's results (the schedule moves no arithmetic, only the order
    of the spread's atomics)."""
    geom, cells, params = wl.channel_workload(nx=24, ny=28, nz=32, ncells=12, body_force=(5e-6, 0, 0), seed=33)
    rng = np.random.default_rng(5)
    cells["vel"] = rng.normal(size=(12, 3)) * 3e-3
    r = _compare(geom, cells, params, 80, schedule=(True, lattice_first))
    print("split spread:", r)


def test_non_integer_kappa():
    """kappa = 19.5 takes the general power of Eq. enhance-viscosity (the
    paper's 20 is computed by squaring)."""
    geom, cells, params = wl.box_workload(n=24, ncells=6, seed=9)
    _compare(geom, cells, dict(params, kappa=19.5), 40)


def test_kernel_timing_on_and_off():
    """Per-launch timing through the graphs' event nodes: counts one timed
    launch per step up to the capacity; turning it off (capacity 0) and on
    again leaves the step graphs usable; the results stay the oracle's."""
    geom, cells, params = wl.box_workload(n=24, ncells=6, seed=9)
    s = _solver(geom, cells, params)
    s.set_timing(4)
    s.step(6)
    ms, cnt = s.kernel_times()
    assert list(cnt) == [4, 4] and ms[0] > 0 and ms[1] > 0
    s.set_timing(0)
    s.step(3)
    s.set_timing(2)
    s.step(3)
    ms, cnt = s.kernel_times()
    assert list(cnt) == [2, 2]
    s.set_timing(0)
    s.step(2)
    o = orc.Oracle(geom, cells, params)
    o.step(14)
    _, u_o, _ = o.fields()
    assert rel_l2(s.fields()["u"], u_o) <= TOL
    s.close()
    o.close()


def test_external_force_and_torque_on_cells():
    """Cells pushed by constant external forces and torques (the mobility
    tests of Sec. 3), the counter-force spread uniformly over the fluid."""
    geom, cells, params = wl.box_workload(n=24, ncells=4, body_force=(0, 0, 0), seed=14)
    rng = np.random.default_rng(15)
    F = rng.normal(size=(4, 3)) * 1e-4
    cells["force_ext"] = F
    cells["torque_ext"] = rng.normal(size=(4, 3)) * 5e-3
    geom["body_force"] = tuple(-F.sum(axis=0) / 24 ** 3)
    r = _compare(geom, cells, params, 60)
    print("external push:", r)
