"""The C-ABI library loads and exports every entry point include/rbc.h
declares; host-only entry points (defaults, workspace sizing, validation)
work without a GPU.  No compute call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1107_4889_gb300 import build as B
from paper_1107_4889_gb300 import rbc
from paper_1107_4889_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return rbc.load()


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(rbc_\w+)\s*\(", txt, re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), name
    assert set(rbc.EXPORTS) == set(declared)


def test_default_params_are_the_papers(lib):
    p = rbc.rbc_default_params()
    assert (p.tau0, p.delta, p.kappa, p.gamma_T, p.gamma_R, p.alpha_tt) == (1.0, 2.0, 20.0, 0.1, 0.1, 0.04)
    assert list(p.xi) == [4.0, 4.0, 1.5] and p.mass == 10.0 and list(p.inertia) == [1000.0] * 3


def test_struct_layouts_match_header(lib):
    # nx..periodic, solid, body_force, body_force_wave, node_type, inlet_center, inlet_radius, inlet_umax
    assert ctypes.sizeof(rbc.rbc_geometry) == 24 + 8 + 24 + 24 + 8 + 16 + 8 + 8
    assert ctypes.sizeof(rbc.rbc_cells) == 8 + 6 * 8  # n, pos, quat, vel, omega_body, force_ext, torque_ext
    assert ctypes.sizeof(rbc.rbc_stats_t) == 8 * 10 + 8 + 8
    assert rbc.rbc_params.stream.offset == ctypes.sizeof(rbc.rbc_params) - 8
    # int precision, int rounding, uint64_t seed, int node_list, int layout, void *stream close the struct
    assert rbc.rbc_params.layout.offset == rbc.rbc_params.stream.offset - 4
    assert rbc.rbc_params.node_list.offset == rbc.rbc_params.stream.offset - 8
    assert rbc.rbc_params.seed.offset == rbc.rbc_params.node_list.offset - 8
    assert rbc.rbc_params.rounding.offset == rbc.rbc_params.seed.offset - 4
    assert rbc.rbc_params.precision.offset == rbc.rbc_params.seed.offset - 8


def test_reduced_precision_halves_population_bytes(lib):
    g, c, p = wl.channel_workload()
    Np = (64 * 64 * 256 + 63) // 64 * 64
    s32 = rbc.rbc_workspace_size(g, c, p)
    for prec in ("f16", "bf16"):
        s16 = rbc.rbc_workspace_size(g, c, dict(p, precision=prec))
        assert abs((s32 - s16) - 2 * 19 * 2 * Np) <= 2 * 256
    with pytest.raises(rbc.RbcError) as e:
        rbc.rbc_workspace_size(g, c, dict(p, precision=3))
    assert e.value.code == rbc.RBC_EINVAL
    with pytest.raises(rbc.RbcError):
        rbc.rbc_workspace_size(g, c, dict(p, precision="f16", rounding=2))


def test_workspace_size_scales_with_problem(lib):
    g, c, p = wl.box_workload()
    s1 = rbc.rbc_workspace_size(g, c, p)
    N = 32 ** 3
    assert s1 > 2 * 19 * 4 * N  # two population copies at least
    g2, c2, p2 = wl.channel_workload()
    s2 = rbc.rbc_workspace_size(g2, c2, p2)
    assert s2 > 2 * 19 * 4 * 64 * 64 * 256


def test_validation_rejects_bad_problems(lib):
    g, c, p = wl.box_workload()
    with pytest.raises(rbc.RbcError) as e:
        rbc.rbc_workspace_size(g, c, dict(p, tau0=0.4))
    assert e.value.code == rbc.RBC_EINVAL
    bad = dict(g, periodic=(1, 0, 1))  # non-periodic y without solid end planes
    with pytest.raises(rbc.RbcError):
        rbc.rbc_workspace_size(bad, c, p)
    tiny = wl.periodic_box(8)
    with pytest.raises(rbc.RbcError):  # support box larger than the lattice
        rbc.rbc_workspace_size(tiny, wl.cells_dict(np.array([[4.0, 4.0, 4.0]]), np.array([[1.0, 0, 0, 0]])), p)
    gch, cch, pch = wl.channel_workload(nx=32, ny=32, nz=32, ncells=10)
    cch["pos"][0, 1] = 40.0  # outside the walled axis
    with pytest.raises(rbc.RbcError):
        rbc.rbc_workspace_size(gch, cch, pch)


def test_missing_library_fails_loudly(tmp_path):
    import importlib
    mod = importlib.reload(rbc)
    mod._lib = None
    with pytest.raises(RuntimeError):
        mod.load(str(tmp_path / "librbc.so"))
    importlib.reload(rbc)


def test_open_boundary_validation(lib):
    g = wl.open_tube(16, 24, 6.0, 0.01)
    p = wl.params()
    dense = rbc.rbc_workspace_size(g, None, dict(p, node_list=-1, layout="dense"))
    # in the dense layout the node-list pass adds one index per fluid node;
    # the default layout of this sparse vessel is the compact one, smaller
    # than both
    nl = rbc.rbc_workspace_size(g, None, dict(p, node_list=1, layout="dense"))
    assert nl > dense and rbc.rbc_workspace_size(g, None, dict(p, layout="dense")) == nl
    assert rbc.rbc_workspace_size(g, None, p) < dense
    bad = dict(g, node_type=np.full_like(g["node_type"], 3))
    with pytest.raises(rbc.RbcError):
        rbc.rbc_workspace_size(bad, None, p)
    bad = dict(g, inlet_radius=0.0)
    with pytest.raises(rbc.RbcError):
        rbc.rbc_workspace_size(bad, None, p)
    bad_nt = g["node_type"].copy()
    bad_nt[0, 0, 0] = 1  # a solid corner node marked as inlet
    with pytest.raises(rbc.RbcError):
        rbc.rbc_workspace_size(dict(g, node_type=bad_nt), None, p)


def test_walled_setup_is_linear_time(lib):
    """Sizing a walled lattice with cells walks the link neighbours of the
    nodes near a wall only (a dilation of the solid mask marks them) and
    wraps coordinates without division: 1.77 M nodes take tens of
    milliseconds.  The earlier all-node walk took 0.8 s here and limited the
    request server, whose one worker thread runs the set-up of every solve."""
    import time

    n = (96, 96, 192)
    solid = np.zeros(n[::-1], np.uint8)
    solid[:, :, 0] = 1
    solid[:, :, -1] = 1
    geom = dict(nx=n[0], ny=n[1], nz=n[2], periodic=(0, 1, 1), solid=solid.reshape(-1), body_force=(0, 0, 1e-6))
    cells = dict(pos=np.array([[n[0] / 2, n[1] / 2, n[2] / 2]]), quat=np.array([[1.0, 0.0, 0.0, 0.0]]))
    rbc.rbc_workspace_size(geom, cells, dict(alpha_tt=0.04))  # warm
    t0 = time.perf_counter()
    rbc.rbc_workspace_size(geom, cells, dict(alpha_tt=0.04))
    assert time.perf_counter() - t0 < 0.4


def test_compact_layout_footprint_follows_the_fluid_nodes(lib):
    """The 512^3 Y-bifurcation (6.67 M fluid nodes of 134 M) with binary16
    populations: the dense layout needs ~18 GB, the compact one stores per
    lattice row only the span its fluid nodes reach, so its workspace is
    within 1.5x of the fluid nodes times the bytes of one stored entry
    (populations 2 x 19 x 2, u 16, sigma 20, rho 4, links 4) plus one byte
    of node flags per lattice node."""
    geom = wl.y_bifurcation(512, 60.0, 45.0)
    p = wl.params(precision="f16")
    dense = rbc.rbc_workspace_size(geom, None, dict(p, layout="dense"))
    compact = rbc.rbc_workspace_size(geom, None, dict(p, layout="compact"))
    auto = rbc.rbc_workspace_size(geom, None, p)
    nf = wl.fluid_count(geom)
    N = 512 ** 3
    per_entry = 2 * 19 * 2 + 16 + 20 + 4 + 4
    assert dense > 15e9 and auto == compact
    assert compact < 1.5 * nf * per_entry + N + 64e6, (compact, nf)
    print(f"Y 512^3 binary16: dense {dense / 1e9:.2f} GB, compact {compact / 1e9:.2f} GB, {nf} fluid nodes")


def test_layout_argument_checks(lib):
    """An unknown layout, and the compact layout of a lattice without solid
    nodes, are rejected on the host."""
    with pytest.raises(rbc.RbcError) as e:
        rbc.rbc_workspace_size(wl.periodic_box(16), None, wl.params(layout=5))
    assert e.value.code == rbc.RBC_EINVAL
    with pytest.raises(rbc.RbcError) as e:
        rbc.rbc_workspace_size(wl.periodic_box(16), None, wl.params(layout="compact"))
    assert e.value.code == rbc.RBC_EINVAL
    # a tube: compact by default, and smaller
    g = wl.tube(64, 28.0, length=32)
    assert rbc.rbc_workspace_size(g, None, wl.params()) < 0.9 * rbc.rbc_workspace_size(g, None, wl.params(layout="dense"))
