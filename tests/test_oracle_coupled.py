"""Pins of the oracle's coupled step and of the seeded workloads.

Total fluid-plus-cell momentum is conserved to rounding in a periodic box
(and grows by exactly N_fluid G_ext h per step under an external force
density), mass is conserved, a dragged cell trails the fluid by a / gamma_T, the
brute-force cell-pair list equals a KD-tree query, and the seeded workloads
place no two cells (or cell and wall) inside the Gay-Berne range.
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from oracle import oracle as orc
from paper_1107_4889_gb300 import workloads as wl


def _small_box(n=24, ncells=6, force=(0.0, 0.0, 0.0), seed=5, **pover):
    geom, cells, params = wl.box_workload(n=n, ncells=ncells, body_force=force, seed=seed, **pover)
    rng = np.random.default_rng(seed + 1000)
    cells["vel"] = rng.normal(size=(ncells, 3)) * 1e-3
    cells["omega"] = rng.normal(size=(ncells, 3)) * 1e-4
    return geom, cells, params


def _total(o):
    b = o.budget()
    return b["mass"], b["p_fluid"] + b["p_cells"]


def test_momentum_conserved_in_periodic_box():
    geom, cells, params = _small_box()
    o = orc.Oracle(geom, cells, params)
    m0, P0 = _total(o)
    scale = np.abs(cells["vel"]).sum() * params["mass"]
    for _ in range(25):
        o.step(1)
        m, P = _total(o)
        assert abs(m - m0) < 1e-11 * m0
        assert np.allclose(P, P0, atol=1e-12 * scale)
    # the fluid did take up momentum: the budget is not trivially static
    assert np.abs(o.budget()["p_fluid"]).max() > 1e-3 * scale


def test_external_force_momentum_budget():
    G = np.array([1e-6, -5e-7, 2e-7])
    geom, cells, params = _small_box(force=G)
    o = orc.Oracle(geom, cells, params)
    N = geom["nx"] * geom["ny"] * geom["nz"]
    _, P0 = _total(o)
    for n in range(1, 11):
        o.step(1)
        _, P = _total(o)
        assert np.allclose(P - P0, n * N * G, rtol=1e-9, atol=1e-14)


def test_dragged_cell_follows_fluid_with_first_order_lag():
    """One cell at rest in fluid accelerated by a uniform force density a:
    the cell obeys dV/dt = gamma_T (u~ - V), so once transients die it trails
    the smeared fluid velocity by a / gamma_T (to O(gamma_T h))."""
    a = 2e-6
    geom = wl.periodic_box(20, body_force=(a, 0.0, 0.0))
    cells = wl.cells_dict(np.array([[10.2, 9.7, 10.4]]), np.array([[0.9, 0.1, 0.3, 0.2]]))
    p = wl.params()
    o = orc.Oracle(geom, cells, p)
    o.step(300)
    V = o.cells()["vel"][0]
    ut = o.diag()["u_s"][0]
    lag = a / p["gamma_T"]
    assert V[0] > 0 and abs((ut[0] - V[0]) - lag) < 0.1 * lag
    # transverse drift only from the anisotropic disturbance of the cell
    assert np.allclose(V[1:], 0.0, atol=2e-2 * lag)


def test_no_force_no_cells_fluid_at_rest():
    geom = wl.periodic_box(8)
    o = orc.Oracle(geom, None, wl.params())
    o.step(5)
    rho, u, s = o.fields()
    assert np.allclose(rho, 1.0, atol=1e-15) and np.allclose(u, 0.0, atol=1e-18)


def test_neighbor_pairs_match_kdtree():
    rng = np.random.default_rng(8)
    geom = wl.periodic_box(40)
    n = 300
    pos = rng.random((n, 3)) * 40.0
    cells = wl.cells_dict(pos, wl.random_quaternions(rng, n))
    o = orc.Oracle(geom, cells, wl.params())
    pairs = o.neighbor_pairs()
    tree = cKDTree(pos, boxsize=40.0)
    ref = np.array(sorted(tree.query_pairs(r=wl.PAPER_PARAMS["r_cut"])))
    got = np.array(sorted(map(tuple, pairs)))
    assert len(ref) > 50 and np.array_equal(got, ref)


def _gb_check(geom, cells, params, max_cells=None, level=0.0):
    """Number of cell-cell and cell-wall pairs whose Gay-Berne energy (via the
    oracle's pair) exceeds ``level`` among the first max_cells cells (level 0:
    any interaction; level eps0: an overlap, reduced distance below 1)."""
    pos = cells["pos"]
    n = len(pos) if max_cells is None else min(max_cells, len(pos))
    Q = np.array([orc.quat_to_Q(q) for q in cells["quat"]])
    a = np.asarray(params["semi_axes"])
    A = np.einsum("nab,b,ncb->nac", Q, a * a, Q)
    dims = np.array([geom["nx"], geom["ny"], geom["nz"]], float)
    box = np.where(np.asarray(geom["periodic"]) == 1, dims, 1e9)
    tree = cKDTree(np.mod(pos, box) if np.all(geom["periodic"]) else pos, boxsize=box)
    smin = np.sqrt(2 * 2 * min(a) ** 2)
    hits = 0
    for i, j in tree.query_pairs(r=params["r_cut"]):
        if i >= n and j >= n:
            continue
        d = pos[i] - pos[j]
        for k in range(3):
            if geom["periodic"][k]:
                d[k] -= dims[k] * np.round(d[k] / dims[k])
        u, F, *_ = orc.gb_pair(d, A[i], A[j], smin, params["eps0"])
        hits += u > level
    # walls: distance to the nearest solid node must exceed the wall range
    if geom["solid"] is not None:
        s = geom["solid"]
        zz, yy, xx = np.nonzero(s)
        wpos = np.stack([xx, yy, zz], axis=1).astype(float)
        wt = cKDTree(wpos, boxsize=box)
        Aw = params["wall_radius"] ** 2 * np.eye(3)
        for i in range(n):
            for w in wt.query_ball_point(pos[i], params["r_cut_wall"]):
                d = pos[i] - wpos[w]
                for k in range(3):
                    if geom["periodic"][k]:
                        d[k] -= dims[k] * np.round(d[k] / dims[k])
                u, *_ = orc.gb_pair(d, A[i], Aw, params["sigma_min_wall"], params["eps0"])
                hits += u > level
    return hits


def test_box_workload_cells_do_not_interact_initially():
    geom, cells, params = wl.box_workload()
    assert abs(wl.hematocrit(geom, 32) - 0.098) < 0.001
    assert _gb_check(geom, cells, params) == 0


def test_channel_workload_cells_do_not_interact_initially():
    geom, cells, params = wl.channel_workload()
    assert len(cells["pos"]) == 3650 and abs(wl.hematocrit(geom, 3650) - 0.35) < 0.001
    assert _gb_check(geom, cells, params, max_cells=3650) == 0
    # every centre stays clear of the walls
    assert cells["pos"][:, 1].min() >= 5.9 and cells["pos"][:, 1].max() <= 57.1


def test_tube_workload_dense_and_without_overlaps():
    """Radius 120 in 256^3: 11,582,464 fluid nodes, 51,846 cells at
    hematocrit 0.45 of the lumen.  The hexagonal slot lattice is denser than
    the Gay-Berne range (neighbours in a cross-section repel weakly at t = 0)
    but no two cells and no cell and wall overlap: every reduced distance
    exceeds 1 (energy below eps0).  Checked on the cells of the first 60
    slot columns, which include the ones next to the wall."""
    geom, cells, params = wl.tube_workload()
    n = len(cells["pos"])
    assert n == 51846 and wl.fluid_count(geom) == 11582464
    assert abs(wl.tube_hematocrit(geom, n) - 0.45) < 1e-3
    r = np.hypot(cells["pos"][:, 0] - 127.5, cells["pos"][:, 1] - 127.5)
    assert r.max() <= 120 - 5.9
    assert _gb_check(geom, cells, params, max_cells=4000, level=params["eps0"]) == 0


def test_candidate_radii_bound_the_interaction_range():
    """r_cut / r_cut_wall enclose every interacting pair: along the direction
    of largest extent (edge to edge) the potential vanishes inside them."""
    p = wl.PAPER_PARAMS
    a = np.asarray(p["semi_axes"])
    A = np.diag(a * a)
    smin = np.sqrt(2 * 2 * min(a) ** 2)
    u, *_ = orc.gb_pair([p["r_cut"], 0, 0], A, A, smin, p["eps0"])
    assert u == 0.0
    u, *_ = orc.gb_pair([p["r_cut"] - 0.05, 0, 0], A, A, smin, p["eps0"])
    assert u > 0.0
    Aw = p["wall_radius"] ** 2 * np.eye(3)
    u, *_ = orc.gb_pair([p["r_cut_wall"], 0, 0], A, Aw, p["sigma_min_wall"], p["eps0"])
    assert u == 0.0
    u, *_ = orc.gb_pair([p["r_cut_wall"] - 0.05, 0, 0], A, Aw, p["sigma_min_wall"], p["eps0"])
    assert u > 0.0
