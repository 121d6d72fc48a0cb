"""GPU parity of the compact layout (per lattice row only the span a fluid
node reaches through a link, in lattice order) against the FP64 oracle, and
the library's fluid-node indexing against the oracle's canonical order.

The compact lattice pass, the shape lists that address it, the budgets and
the field read-back are checked on: a tube with cells (rows of every
width, solid rows skipped); a walled lattice whose rows are not a multiple
of the 8-entry alignment (whole-row spans with padding entries); a lattice
whose rows are wider than a stage (the pass cuts them along x); open
boundaries in a tube and a Y-bifurcation; binary16 storage with stochastic
rounding (the random bits are keyed by the lattice index in either layout,
so the oracle with the same storage step is the reference).  Tolerances are
those of the dense path: relative L2 1e-5 on u and rho, per-cell values
1e-5 of their largest (rotational floors as in test_gpu_parity), 2e-3 for
binary16 against the emulating oracle.  Fluid-node indexing: bit-exact.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1107_4889_gb300 import workloads as wl

from .test_gpu_parity import TOL, _compare, rel_l2

pytestmark = pytest.mark.gpu


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


def _small_tube(n=40, radius=17.0, nz=32, ncells=40, seed=3):
    """A short tube (radius 17 in 40 x 40 x 32, periodic along z) with cells
    in the tube workload's slot lattice."""
    geom, cells, params = wl.tube_workload(n=n, radius=radius, ncells=ncells, seed=seed,
                                           body_force=(0.0, 0.0, 4e-6))
    keep = cells["pos"][:, 2] < nz - 2
    geom = wl.tube(n, radius, length=nz, body_force=(0.0, 0.0, 4e-6))
    cells = wl.cells_dict(cells["pos"][keep], cells["quat"][keep])
    return geom, cells, params


def _layout(geom, cells, params):
    s = _solver(geom, cells, params)
    lay = s.layout()
    s.close()
    return lay


def test_tube_with_cells_compact_matches_oracle():
    geom, cells, params = _small_tube()
    lay = _layout(geom, cells, params)
    assert lay["compact"] and lay["entries"] < 0.9 * geom["nx"] * geom["ny"] * geom["nz"]
    rng = np.random.default_rng(6)
    cells["vel"] = rng.normal(size=(len(cells["pos"]), 3)) * 2e-3
    r = _compare(geom, cells, params, 80)
    print("compact tube:", lay, r)


def test_auto_layout_choice():
    """Auto: compact for the tube, dense for a plane channel (nearly every
    row is stored either way) and for a periodic box (no solid nodes)."""
    geom, cells, params = _small_tube()
    assert _layout(geom, cells, params)["compact"]
    geom, cells, params = wl.channel_workload(nx=24, ny=28, nz=32, ncells=12, body_force=(5e-6, 0, 0), seed=33)
    assert not _layout(geom, cells, params)["compact"]
    assert _layout(geom, cells, dict(params, layout="compact"))["compact"]
    geom, cells, params = wl.box_workload(n=24, ncells=6, seed=9)
    assert not _layout(geom, cells, params)["compact"]


def test_ragged_walled_lattice_compact():
    """17 x 19 x 23 plane channel with an obstacle: rows span the whole
    periodic x range and end in padding entries (17 -> 24); fluid only."""
    geom = wl.plane_channel(17, 19, 23, body_force=(2e-6, 0.0, 1e-6))
    geom["solid"][5:9, 7:10, 6:9] = 1
    _compare(geom, None, wl.params(layout="compact"), 120)


def test_coupled_channel_compact():
    geom, cells, params = wl.channel_workload(nx=24, ny=28, nz=32, ncells=12, body_force=(5e-6, 0, 0), seed=33)
    rng = np.random.default_rng(5)
    cells["vel"] = rng.normal(size=(12, 3)) * 3e-3
    r = _compare(geom, cells, dict(params, layout="compact"), 80)
    print("compact channel:", r)


def test_rows_wider_than_a_stage_are_cut():
    """300 x 20 x 20 duct (solid planes x = 0, 299 and y = 0, 19; periodic in
    z) with cells: each row's window (304 entries x 96 bytes with cells) is
    wider than a stage, so the pass cuts the rows along x."""
    nx, ny, nz = 300, 20, 20
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:, :, 0] = solid[:, :, nx - 1] = 1
    solid[:, 0, :] = solid[:, ny - 1, :] = 1
    geom = dict(nx=nx, ny=ny, nz=nz, periodic=(0, 0, 1), solid=solid, body_force=(3e-6, 0.0, 1e-6))
    rng = np.random.default_rng(8)
    pos = np.column_stack([np.linspace(20, 280, 6), np.full(6, 9.7), rng.uniform(4, 16, 6)])
    quat = wl.tilted_quaternions(rng, 6, np.array([1.0, 0.0, 0.0, 0.0]), 0.3)
    cells = wl.cells_dict(pos, quat)
    params = wl.params(layout="compact")
    r = _compare(geom, cells, params, 60)
    print("wide rows:", r)


def test_open_tube_and_ybifurcation_compact_fp32_and_binary16():
    from .test_gpu_open import _compare as open_compare
    geom = wl.open_tube(24, 40, 10.0, 0.02)
    r = open_compare(geom, None, wl.params(layout="compact"), 150)
    print("open tube compact:", r)
    geom = wl.y_bifurcation(48, 9.0, 6.0, umax=0.02)
    r = open_compare(geom, None, wl.params(layout="compact"), 120)
    print("Y compact:", r)
    r = open_compare(geom, None, wl.params(layout="compact", precision="f16", seed=77), 120, storage="f16",
                     tol=2e-3)
    print("Y compact binary16:", r)


def test_binary16_compact_tube_with_cells_matches_emulating_oracle():
    from .test_gpu_precision import TOL_EMULATED, _run
    geom, cells, params = _small_tube()
    out = _run(geom, cells, dict(params, layout="compact"), "f16", "stochastic", 60)
    print("compact f16 tube:", out)
    assert out["u_emul"] <= TOL_EMULATED and out["J_emul"] <= TOL_EMULATED


def test_compact_budgets_match_oracle():
    """rbc_stats over the compact rows against the oracle's budget."""
    geom, cells, params = _small_tube()
    o = orc.Oracle(geom, cells, params)
    s = _solver(geom, cells, params)
    o.step(60)
    s.step(60)
    bo, bg = o.budget(), s.stats()
    s.close()
    o.close()
    assert abs(bg["mass"] - bo["mass"]) <= 1e-9 * bo["mass"]
    for k in ("p_fluid", "p_cells"):
        sc = np.abs(bo[k]).max()
        assert np.abs(bg[k] - bo[k]).max() <= TOL * sc, (k, bg[k], bo[k])
    assert abs(bg["power"] - bo["power"]) <= TOL * abs(bo["power"])


@pytest.mark.parametrize("which", ["tube", "ybif", "channel"])
def test_fluid_node_indexing_is_the_oracles(which):
    """The library's fluid nodes, in the order of its storage entries, equal
    the oracle's canonical list bit for bit (compact and dense layouts)."""
    if which == "tube":
        geom, cells, params = _small_tube()
    elif which == "ybif":
        geom, cells, params = wl.y_bifurcation(64, 12.0, 8.0), None, wl.params()
    else:
        geom, cells, params = wl.channel_workload(nx=24, ny=28, nz=32, ncells=12, seed=33)
    s = _solver(geom, cells, params)
    got = s.fluid_nodes()
    lay = s.layout()
    s.close()
    o = orc.Oracle(geom, cells, params)
    ref = o.fluid_nodes()
    o.close()
    assert lay["fluid"] == len(ref) == wl.fluid_count(geom)
    assert got.dtype == np.int64 and np.array_equal(got, ref)
    if which != "channel":
        assert lay["compact"]
