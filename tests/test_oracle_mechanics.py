"""Pins of the oracle's per-cell mechanical sums, its wall particles and the
first step's hydrodynamic impulses.

- Cells in Gay-Berne contact (Sec. 2.5, App. B): the pair forces sum to zero
  over all cells (Newton's third law applied on the j side of every pair),
  the pair torques and moments of the forces sum to zero (the identity
  tau_i + tau_j = -R_ij x F_ij at the end of App. B, summed over pairs), and
  the total fluid-plus-cell momentum of a periodic box stays constant to
  rounding while the contacts act.  A sign slip on the j side of the force
  or the torque accumulation fails these.
- Wall particles (Sec. 2.5, last paragraph: each wall mesh point a Gay-Berne
  sphere): the set is the solid nodes with a fluid node among their lattice
  links, built here independently of the oracle on a channel with a ledge
  (solid nodes behind the surface and on the ledge's inner corner make the
  set differ from both "all solid nodes" and "solid nodes with a fluid face
  neighbour").  The oracle's wall force equals minus the finite-difference
  gradient of the summed wall energy, its wall torque minus the derivative
  under small rotations, a sphere beside a flat wall feels no tangential
  force and no torque, and at deep overlaps its force is the sum over the
  correct set and not over the two wrong ones.
- First step in quiescent fluid (App. A with the readings of the oracle):
  the fluid and the mechanical forces are zero, so the impulses are the
  friction half step alone, J = M (e^(-gamma_T h/2) - 1) V0 and
  L = Q0 I (e^(-gamma_R h/2) - 1) Omega0 with the orientation Q0 before the
  sub-rotations (anisotropic I and a fast spin make the frame matter).
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as orc
from paper_1107_4889_gb300 import workloads as wl

D3Q19_LINKS = np.array([(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
                        (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1),
                        (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)])


def _A(Q, a):
    return Q @ np.diag(np.asarray(a, float) ** 2) @ Q.T


def _smin_cc(a):
    return np.sqrt(2.0 * 2.0 * min(a) ** 2)


# ---------------------------------------------------------------------------
# cells in contact
# ---------------------------------------------------------------------------

def _contact_partner(rng, Ri, Qi, a, eps0, shell):
    """A partner pose j at a distance where the pair's reduced distance lies
    in `shell` (an interval of rho); contact found by bisection along a
    random direction with the oracle's pinned pair."""
    smin = _smin_cc(a)
    while True:
        Qj = Rotation.random(random_state=rng).as_matrix()
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        Ai, Aj = _A(Qi, a), _A(Qj, a)
        lo, hi = 0.5, 12.0
        for _ in range(80):  # contact distance: u = eps0 (rho = 1)
            mid = 0.5 * (lo + hi)
            u, *_ = orc.gb_pair(mid * n, Ai, Aj, smin, eps0)
            lo, hi = (mid, hi) if u > eps0 else (lo, mid)
        rho = rng.uniform(*shell)
        # rho = (R - sigma + smin) / smin with sigma the contact distance
        R = hi + (rho - 1.0) * smin
        if R > 1.0:
            return Ri - R * n, Qj


def _contact_workload(seed=3, deep=True, eps0=0.01):
    rng = np.random.default_rng(seed)
    L = 40
    a = wl.PAPER_PARAMS["semi_axes"]
    pos, quat = [], []
    centres = [(10, 10, 10), (30, 10, 12), (10, 30, 28), (29, 29, 30), (20, 20, 20)]
    for k, c in enumerate(centres):
        Ri = np.array(c, float) + rng.uniform(-0.5, 0.5, 3)
        Qi = Rotation.random(random_state=rng).as_matrix()
        shell = (0.55, 0.7) if (deep and k == 0) else (0.85, 1.1)  # one pair clamped
        Rj, Qj = _contact_partner(rng, Ri, Qi, a, eps0, shell)
        for R, Q in ((Ri, Qi), (Rj, Qj)):
            pos.append(R)
            q = Rotation.from_matrix(Q).as_quat()  # (x, y, z, w)
            quat.append([q[3], q[0], q[1], q[2]])
    geom = wl.periodic_box(L)
    cells = wl.cells_dict(np.array(pos), np.array(quat))
    cells["vel"] = rng.normal(size=(len(pos), 3)) * 1e-3
    cells["omega"] = rng.normal(size=(len(pos), 3)) * 1e-4
    return geom, cells, wl.params(eps0=eps0)


def test_pair_forces_and_torques_of_contacts_sum_to_zero():
    """Sum of F_mech = 0 and sum of (R x F_mech + tau_mech) = 0 over all
    cells when five pairs are in contact (one of them deep enough to be
    clamped); a slip on the j side of either sum breaks one of them."""
    geom, cells, params = _contact_workload()
    o = orc.Oracle(geom, cells, params)
    R0 = o.cells()["pos"].copy()
    o.step(1)
    d = o.diag()
    F, T = d["F_mech"], d["tau_mech"]
    fscale = np.abs(F).max()
    assert fscale > 1e-3 and np.count_nonzero(np.linalg.norm(F, axis=1) > 1e-4 * fscale) == len(F)
    assert np.abs(T).max() > 1e-3  # the tilted pairs exert torques
    assert o.clamps >= 1  # the deep pair was clamped
    assert np.abs(F.sum(axis=0)).max() <= 1e-14 * fscale * len(F)
    # no pair straddles the periodic boundary, so R_i - R_j is the pair vector
    Ltot = np.cross(R0, F).sum(axis=0) + T.sum(axis=0)
    assert np.abs(Ltot).max() <= 1e-13 * fscale * 40 * len(F)
    o.close()


def test_momentum_conserved_with_contacts():
    """Total fluid-plus-cell momentum in a periodic box without external
    force stays constant to rounding while Gay-Berne contacts push the
    cells apart; the cells do exchange momentum with each other.  eps0 =
    1e-4 keeps the contact forces (the clamped pair's included) inside the
    stability bound |F| < 0.1 that the paper gives for the lattice."""
    geom, cells, params = _contact_workload(seed=11, eps0=1e-4)
    o = orc.Oracle(geom, cells, params)
    b0 = o.budget()
    P0 = b0["p_fluid"] + b0["p_cells"]
    V0 = np.asarray(cells["vel"]).copy()
    fmax = 0.0
    for _ in range(15):
        o.step(1)
        b = o.budget()
        fmax = max(fmax, np.abs(o.diag()["F_mech"]).max())
        # the budget sums 19 x 64,000 populations in plain order: its own
        # rounding is ~1e-11 of the mass
        assert abs(b["mass"] - b0["mass"]) < 1e-10 * b0["mass"]
        # rounding of momenta of this size (the clamped pair's force is O(1))
        scale = params["mass"] * np.abs(o.cells()["vel"]).sum() + np.abs(b["p_fluid"]).sum() + 1e-3
        assert np.allclose(b["p_fluid"] + b["p_cells"], P0, rtol=0, atol=1e-13 * scale)
    dV = np.abs(o.cells()["vel"] - V0).max()
    assert fmax > 1e-3 and dV > 1e-4 and o.clamps >= 1  # the contacts did act
    o.close()


# ---------------------------------------------------------------------------
# wall particles
# ---------------------------------------------------------------------------

def _ledge_geometry(n=32):
    """Channel along x and z (periodic), solid slab y <= 2 and y >= n - 3,
    and a ledge y <= 5 for x < 12 (its inner corner leaves solid nodes with
    only diagonal fluid links)."""
    solid = np.zeros((n, n, n), np.uint8)  # (z, y, x)
    solid[:, :3, :] = 1
    solid[:, n - 3:, :] = 1
    solid[:, 3:6, :12] = 1
    return dict(nx=n, ny=n, nz=n, periodic=(1, 0, 1), solid=solid, body_force=(0.0, 0.0, 0.0))


def _wet_sets(solid):
    """(link-wet, face-wet, all solid) node coordinates (x, y, z): solid
    nodes with a fluid node among their 18 lattice links, among their six
    face neighbours, and every solid node.  The lattice wraps on every axis."""
    fluid = solid == 0
    link = np.zeros_like(fluid)
    face = np.zeros_like(fluid)
    for c in D3Q19_LINKS:
        nb = np.roll(fluid, shift=(-c[2], -c[1], -c[0]), axis=(0, 1, 2))
        link |= nb
        if np.abs(c).sum() == 1:
            face |= nb
    out = []
    for m in (link & ~fluid, face & ~fluid, ~fluid):
        z, y, x = np.nonzero(m)
        out.append(np.stack([x, y, z], axis=1).astype(float))
    return out


def _wall_sum(R, Q, wall, geom, params, what="energy"):
    a = params["semi_axes"]
    Ai = _A(Q, a)
    Aw = params["wall_radius"] ** 2 * np.eye(3)
    dims = np.array([geom["nx"], geom["ny"], geom["nz"]], float)
    per = np.asarray(geom["periodic"], bool)
    d = R - wall
    d[:, per] -= dims[per] * np.round(d[:, per] / dims[per])
    near = np.einsum("ij,ij->i", d, d) < params["r_cut_wall"] ** 2
    E, F, T = 0.0, np.zeros(3), np.zeros(3)
    for dv in d[near]:
        u, f, ti, _, _ = orc.gb_pair(dv, Ai, Aw, params["sigma_min_wall"], params["eps0"], params["rho_floor"])
        E += u
        F += f
        T += ti
    return E if what == "energy" else (F, T)


def _oracle_wall_force(geom, R, Q, params):
    q = Rotation.from_matrix(Q).as_quat()
    cells = wl.cells_dict(np.array([R]), np.array([[q[3], q[0], q[1], q[2]]]))
    o = orc.Oracle(geom, cells, params)
    o.step(1)
    d = o.diag()
    o.close()
    return d["F_mech"][0], d["tau_mech"][0]


def _rot(axis, t):
    v = np.zeros(3)
    v[axis] = t
    return Rotation.from_rotvec(v).as_matrix()


def test_wall_force_and_torque_are_minus_energy_derivatives():
    geom = _ledge_geometry()
    params = wl.params()
    wet, _, _ = _wet_sets(geom["solid"])
    rng = np.random.default_rng(12)
    checked = 0
    while checked < 5:
        R = np.array([rng.uniform(8, 16), rng.uniform(6.5, 10.5), rng.uniform(8, 24)])
        Q = Rotation.random(random_state=rng).as_matrix()
        E = _wall_sum(R, Q, wet, geom, params)
        if not (1e-5 < E):
            continue
        # every wall pair unclamped, so the energy is differentiable
        Ai = _A(Q, params["semi_axes"])
        clamped = False
        for w in wet:
            d = R - w
            d[0] -= 32 * np.round(d[0] / 32)
            d[2] -= 32 * np.round(d[2] / 32)
            if d @ d < params["r_cut_wall"] ** 2:
                clamped |= bool(orc.gb_pair(d, Ai, params["wall_radius"] ** 2 * np.eye(3),
                                            params["sigma_min_wall"], params["eps0"], params["rho_floor"])[4])
        if clamped:
            continue
        F, T = _oracle_wall_force(geom, R, Q, params)
        h = 1e-6
        Ffd = np.zeros(3)
        Tfd = np.zeros(3)
        for ax in range(3):
            e = np.zeros(3)
            e[ax] = h
            Ffd[ax] = -(_wall_sum(R + e, Q, wet, geom, params) - _wall_sum(R - e, Q, wet, geom, params)) / (2 * h)
            Tfd[ax] = -(_wall_sum(R, _rot(ax, h) @ Q, wet, geom, params) -
                        _wall_sum(R, _rot(ax, -h) @ Q, wet, geom, params)) / (2 * h)
        assert np.linalg.norm(F) > 1e-4
        assert np.allclose(F, Ffd, rtol=0, atol=1e-6 * np.linalg.norm(F)), (F, Ffd)
        assert np.allclose(T, Tfd, rtol=0, atol=1e-6 * max(np.linalg.norm(T), np.linalg.norm(F))), (T, Tfd)
        checked += 1


def test_wall_particles_are_the_solid_nodes_with_a_fluid_link():
    """At deep overlaps (clamped pairs, where no energy derivative exists)
    the oracle's wall force is the sum of the pair forces over the solid
    nodes with a fluid link, and differs from the sums over all solid nodes
    and over solid nodes with a fluid face neighbour."""
    geom = _ledge_geometry()
    params = wl.params()
    link, face, allsolid = _wet_sets(geom["solid"])
    assert len(allsolid) > len(link) > len(face)
    rng = np.random.default_rng(7)
    beat_all = beat_face = 0
    for _ in range(30):
        # near the ledge's edge and inner corner, overlapping the surface
        R = np.array([rng.uniform(10, 14), rng.uniform(5.5, 8.0), rng.uniform(8, 24)])
        Q = Rotation.random(random_state=rng).as_matrix()
        F, T = _oracle_wall_force(geom, R, Q, params)
        Fl, Tl = _wall_sum(R, Q, link, geom, params, "force")
        scale = max(np.linalg.norm(Fl), 1e-300)
        assert np.allclose(F, Fl, rtol=0, atol=1e-12 * scale)
        assert np.allclose(T, Tl, rtol=0, atol=1e-12 * max(np.linalg.norm(Tl), scale))
        Fa, _ = _wall_sum(R, Q, allsolid, geom, params, "force")
        Ff, _ = _wall_sum(R, Q, face, geom, params, "force")
        beat_all += np.linalg.norm(Fa - Fl) > 1e-3 * scale
        beat_face += np.linalg.norm(Ff - Fl) > 1e-3 * scale
    assert beat_all >= 3 and beat_face >= 3


def test_sphere_beside_flat_wall_feels_only_normal_force():
    """A spherical cell centred over a lattice node (x) and a half node (z)
    of a flat wall: mirror symmetry leaves no tangential force, an isotropic
    shape no torque; the force pushes away from the wall."""
    n = 24
    solid = np.zeros((n, n, n), np.uint8)
    solid[:, 0, :] = 1
    solid[:, n - 1, :] = 1
    geom = dict(nx=n, ny=n, nz=n, periodic=(1, 0, 1), solid=solid, body_force=(0.0, 0.0, 0.0))
    params = wl.params(semi_axes=(3.0, 3.0, 3.0), xi=(3.0, 3.0, 3.0))
    for y in (3.0, 3.1, 3.2):
        F, T = _oracle_wall_force(geom, np.array([11.0, y, 11.5]), np.eye(3), params)
        assert F[1] > 1e-4
        assert abs(F[0]) <= 1e-14 * F[1] and abs(F[2]) <= 1e-14 * F[1]
        assert np.abs(T).max() <= 1e-14 * F[1]


# ---------------------------------------------------------------------------
# first-step impulses
# ---------------------------------------------------------------------------

def test_first_step_impulses_in_quiescent_fluid():
    geom = wl.periodic_box(24)
    rng = np.random.default_rng(9)
    n = 3
    pos = np.array([[6.2, 7.1, 5.3], [17.4, 8.8, 15.9], [9.6, 18.3, 12.2]])
    quat = wl.random_quaternions(rng, n)
    cells = wl.cells_dict(pos, quat)
    V0 = rng.normal(size=(n, 3)) * 2e-3
    W0 = rng.normal(size=(n, 3)) * 0.05  # fast spin: the sub-rotations turn Q by ~0.05 rad
    cells["vel"], cells["omega"] = V0, W0
    params = wl.params(inertia=(1000.0, 700.0, 400.0), gamma_T=0.1, gamma_R=0.07)
    o = orc.Oracle(geom, cells, params)
    o.step(1)
    d = o.diag()
    Q1 = o.cells()["Q"]
    o.close()
    M, I = params["mass"], np.asarray(params["inertia"])
    eT, eR = np.exp(-params["gamma_T"] / 2), np.exp(-params["gamma_R"] / 2)
    for i in range(n):
        Q0 = orc.quat_to_Q(quat[i])
        J = M * (eT - 1.0) * V0[i]
        L = Q0 @ (I * (eR - 1.0) * W0[i])
        assert np.allclose(d["J"][i], J, rtol=1e-12, atol=0)
        assert np.allclose(d["L"][i], L, rtol=1e-12, atol=0)
        # the frame matters: the orientation after the step gives another L
        assert np.linalg.norm(Q1[i] @ (I * (eR - 1.0) * W0[i]) - L) > 1e-3 * np.linalg.norm(L)
        assert np.abs(d["F_mech"][i]).max() == 0.0 and np.abs(d["u_s"][i]).max() == 0.0


# ---------------------------------------------------------------------------
# external force and torque (the push of the mobility tests of Sec. 3)
# ---------------------------------------------------------------------------

def test_external_push_adds_exactly_its_impulse():
    """A constant external force F on one cell in a periodic box without
    external fluid force: the total fluid-plus-cell momentum grows by exactly
    F per step, (n - 1/2) F after n steps since the first step applies only
    its opening half kick (the push is not returned to the fluid as a
    hydrodynamic impulse, and the impulse the cell does return conserves
    momentum); the
    cell's rotation under a constant torque about a principal axis speeds up
    monotonically.  An external torque acts in the
    lab frame (it enters the combined torque through Q^T)."""
    geom = wl.periodic_box(24)
    cells = wl.cells_dict(np.array([[11.3, 12.2, 12.7]]), np.array([[0.9, 0.2, -0.3, 0.1]]))
    F = np.array([2e-4, -1e-4, 5e-5])
    cells["force_ext"] = F[None, :]
    o = orc.Oracle(geom, cells, wl.params())
    b0 = o.budget()
    P0 = b0["p_fluid"] + b0["p_cells"]
    for n in range(1, 31):
        o.step(1)
        b = o.budget()
        assert np.allclose(b["p_fluid"] + b["p_cells"] - P0, (n - 0.5) * F, rtol=1e-9, atol=1e-15)
    assert np.allclose(o.diag()["F_mech"][0], F)
    o.close()
    # torque about the lab z axis on a cell whose short axis points along z
    cells = wl.cells_dict(np.array([[11.3, 12.2, 12.7]]), np.array([[1.0, 0.0, 0.0, 0.0]]))
    cells["torque_ext"] = np.array([[0.0, 0.0, 0.05]])
    o = orc.Oracle(geom, cells, wl.params(alpha_tt=0.0))
    w = []
    for _ in range(60):
        o.step(1)
        w.append(o.cells()["omega"][0, 2])
    o.close()
    w = np.array(w)
    assert np.all(np.diff(w) > 0) and w[-1] > 0
    # the fluid co-rotates with the cell and adds mobility: the spin passes
    # the bare friction rate tau / (I gamma_R) and keeps growing
    bare = 0.05 / (1000.0 * 0.1)
    assert w[-1] > bare
