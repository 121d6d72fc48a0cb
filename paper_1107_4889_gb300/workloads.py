"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs: geometry masks (periodic boxes, walled plane
channels, straight tubes), cell centres and orientations, and the parameter
set of the paper.  It holds none of the method's arithmetic: cells are placed
by pure geometry (a minimum centre distance, or one cell per slot of a slot
lattice), and the pair-potential check that no two placed cells interact at
t = 0 lives in the tests.  Both the CUDA path and the CPU oracle consume what
it returns, as plain dicts of numpy arrays.

Units are lattice units.  Parameter values follow the paper: tau0 = 1
(nu0 = 1/6), Delta = 2, kappa = 20 (Sec. 2.4); gamma_T = gamma_R = 0.1 and
alpha = 0.04 (Sec. 3); M = 10, I = 1000 (Sec. 3); the cell is an oblate
ellipsoid with semi-axes (4, 4, 1.5) whose shape-function radii equal its
semi-axes.  eps0 (never given in the paper) defaults to 0.01.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 1107_4889

#: parameter set of the paper (lattice units); r_cut / r_cut_wall are the
#: candidate radii of the cell-pair and cell-wall searches, rounded up from the
#: largest Gay-Berne interaction range of this cell shape (8.367 and 5.762).
PAPER_PARAMS = dict(
    tau0=1.0, delta=2.0, kappa=20.0,
    gamma_T=0.1, gamma_R=0.1, alpha_tt=0.04, eps0=0.01,
    xi=(4.0, 4.0, 1.5), semi_axes=(4.0, 4.0, 1.5),
    mass=10.0, inertia=(1000.0, 1000.0, 1000.0),
    sigma_min_wall=0.5, wall_radius=0.5, rho_floor=0.75,
    r_cut=8.4, r_cut_wall=5.8,
)

CELL_VOLUME = 4.0 / 3.0 * math.pi * 4.0 * 4.0 * 1.5  # 100.53 lu^3


def params(**overrides):
    p = dict(PAPER_PARAMS)
    p.update(overrides)
    return p


# ---------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------

def periodic_box(nx, ny=None, nz=None, body_force=(0.0, 0.0, 0.0)):
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return dict(nx=nx, ny=ny, nz=nz, periodic=(1, 1, 1), solid=None,
                body_force=tuple(float(b) for b in body_force))


def plane_channel(nx, ny, nz, body_force=(0.0, 0.0, 0.0)):
    """Solid planes y = 0 and y = ny - 1; periodic along x and z."""
    solid = np.zeros((nz, ny, nx), dtype=np.uint8)
    solid[:, 0, :] = 1
    solid[:, ny - 1, :] = 1
    return dict(nx=nx, ny=ny, nz=nz, periodic=(1, 0, 1), solid=solid,
                body_force=tuple(float(b) for b in body_force))


def tube(n, radius, length=None, body_force=(0.0, 0.0, 0.0)):
    """Straight tube along z centred at ((n-1)/2, (n-1)/2); nodes farther than
    ``radius`` from the axis are solid; periodic along z."""
    nz = n if length is None else length
    c = (n - 1) / 2.0
    y, x = np.mgrid[0:n, 0:n]
    outside = ((x - c) ** 2 + (y - c) ** 2) > radius * radius
    solid = np.broadcast_to(outside.astype(np.uint8), (nz, n, n)).copy()
    return dict(nx=n, ny=n, nz=nz, periodic=(0, 0, 1), solid=solid,
                body_force=tuple(float(b) for b in body_force))


def fluid_count(geom):
    N = geom["nx"] * geom["ny"] * geom["nz"]
    return N if geom["solid"] is None else int(N - int(np.count_nonzero(geom["solid"])))


# ---------------------------------------------------------------------------
# orientations and placement
# ---------------------------------------------------------------------------

def random_quaternions(rng, n):
    """Uniform random unit quaternions (w, x, y, z), Shoemake's method."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    q = np.stack([b * np.cos(2 * np.pi * u3), a * np.sin(2 * np.pi * u2),
                  a * np.cos(2 * np.pi * u2), b * np.sin(2 * np.pi * u3)], axis=1)
    return q


def quat_mul(p, q):
    w1, x1, y1, z1 = np.moveaxis(np.asarray(p, float), -1, 0)
    w2, x2, y2, z2 = np.moveaxis(np.asarray(q, float), -1, 0)
    return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], axis=-1)


def axis_angle_quat(axis, angle):
    axis = np.asarray(axis, float)
    axis = axis / np.linalg.norm(axis, axis=-1, keepdims=True)
    h = 0.5 * np.asarray(angle, float)[..., None]
    return np.concatenate([np.cos(h), np.sin(h) * axis], axis=-1)


def _min_image(d, dims, periodic):
    d = d.copy()
    for a in range(3):
        if periodic[a]:
            L = dims[a]
            d[..., a] -= L * np.round(d[..., a] / L)
    return d


def place_rsa(rng, geom, n, min_dist, lo=None, hi=None, max_tries=200000):
    """Random sequential addition of ``n`` centres at least ``min_dist`` apart
    (minimum image along periodic axes), uniform in the box [lo, hi)."""
    dims = (geom["nx"], geom["ny"], geom["nz"])
    lo = np.zeros(3) if lo is None else np.asarray(lo, float)
    hi = np.asarray(dims, float) if hi is None else np.asarray(hi, float)
    pts = np.zeros((0, 3))
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError(f"placement jammed at {len(pts)} of {n} cells")
        p = lo + rng.random(3) * (hi - lo)
        if len(pts):
            d = _min_image(pts - p, dims, geom["periodic"])
            if np.min(np.einsum("ij,ij->i", d, d)) < min_dist * min_dist:
                continue
        pts = np.vstack([pts, p])
    return pts


def slot_centres(L, spacing, periodic, cmin=None, cmax=None):
    if periodic:
        m = int(math.floor(L / spacing))
        return (np.arange(m) + 0.5) * (L / m)
    m = int(math.floor((cmax - cmin) / spacing)) + 1
    if m == 1:
        return np.array([(cmin + cmax) / 2.0])
    return np.linspace(cmin, cmax, m)


def place_slots(rng, axes_centres, n, jitter):
    """Choose ``n`` distinct slots of the lattice spanned by the per-axis slot
    centres at random and jitter each centre uniformly by +-jitter."""
    X, Y, Z = np.meshgrid(*axes_centres, indexing="ij")
    slots = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    if n > len(slots):
        raise RuntimeError(f"{n} cells do not fit in {len(slots)} slots")
    pick = np.sort(rng.choice(len(slots), size=n, replace=False))
    pos = slots[pick] + (rng.random((n, 3)) * 2.0 - 1.0) * np.asarray(jitter, float)
    return pos


def tilted_quaternions(rng, n, base, tilt_max):
    """Base orientation, a random spin about the body short axis (z), then a
    random tilt of at most ``tilt_max`` radians about a random lab axis."""
    spin = axis_angle_quat(np.tile([0.0, 0.0, 1.0], (n, 1)), rng.random(n) * 2 * np.pi)
    axis = rng.normal(size=(n, 3))
    tilt = axis_angle_quat(axis, rng.random(n) * tilt_max)
    q = quat_mul(tilt, quat_mul(np.tile(base, (n, 1)), spin))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def _wrap(pos, geom):
    dims = np.array([geom["nx"], geom["ny"], geom["nz"]], float)
    pos = pos.copy()
    for a in range(3):
        if geom["periodic"][a]:
            pos[:, a] = np.mod(pos[:, a], dims[a])
    return pos


def cells_dict(pos, quat):
    n = len(pos)
    return dict(pos=np.ascontiguousarray(pos, dtype=np.float64),
                quat=np.ascontiguousarray(quat, dtype=np.float64),
                vel=np.zeros((n, 3)), omega=np.zeros((n, 3)))


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def box_workload(n=32, ncells=32, body_force=(1e-6, 0.0, 0.0), seed=SEED_BASE + 1, **pover):
    """Periodic box with randomly oriented cells whose centres are at least
    8.2 apart (more than twice the largest semi-axis, so no two cells touch).
    Default: the 32^3 box with 32 cells (hematocrit 9.8 %) driven by a
    uniform force density 1e-6 along x."""
    rng = np.random.default_rng(seed)
    geom = periodic_box(n, body_force=body_force)
    pos = place_rsa(rng, geom, ncells, 8.2)
    quat = random_quaternions(rng, ncells)
    return geom, cells_dict(pos, quat), params(**pover)


def channel_workload(nx=64, ny=64, nz=256, ncells=3650, body_force=(5.376e-7, 0.0, 0.0),
                     seed=SEED_BASE + 2, wall_clearance=6.0, tilt_max_deg=5.0, **pover):
    """Walled plane channel (solid planes y = 0 and y = ny-1, periodic in x and
    z) with cells in a slot lattice: short axis along x (slot pitch >= 3.37),
    in-plane pitch >= 8.4 along y and z, centres at least ``wall_clearance``
    from the wall planes, random spin about the short axis and a tilt of at
    most ``tilt_max_deg``.  Default: 64 x 64 x 256 with 3,650 cells
    (hematocrit 0.35 of the box) and the force density 5.376e-7 along x that
    gives a wall shear rate 1e-4 per step in plain plasma (G = 2 nu0 rate / W,
    nu0 = 1/6, W = 62)."""
    rng = np.random.default_rng(seed)
    geom = plane_channel(nx, ny, nz, body_force=body_force)
    xs = slot_centres(nx, 3.37, True)
    ys = slot_centres(ny, 8.4, False, wall_clearance, (ny - 1) - wall_clearance)
    zs = slot_centres(nz, 8.4, True)
    pos = _wrap(place_slots(rng, (xs, ys, zs), ncells, (0.05, 0.04, 0.05)), geom)
    base = axis_angle_quat([0.0, 1.0, 0.0], math.pi / 2.0)  # body z (short axis) -> lab x
    quat = tilted_quaternions(rng, ncells, base, math.radians(tilt_max_deg))
    return geom, cells_dict(pos, quat), params(**pover)


def tube_workload(n=256, radius=120.0, ncells=51846, body_force=(0.0, 0.0, 0.0),
                  seed=SEED_BASE + 3, wall_clearance=6.0, tilt_max_deg=5.0, **pover):
    """Straight tube along z with cells in slots inside radius - clearance;
    short axis along z (slot pitch >= 3.37), in-plane pitch >= 8.4."""
    rng = np.random.default_rng(seed)
    geom = tube(n, radius, body_force=body_force)
    c = (n - 1) / 2.0
    r_in = radius - wall_clearance
    xs = slot_centres(n, 8.4, False, c - r_in, c + r_in)
    zs = slot_centres(n, 3.37, True)
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    inside = (X - c) ** 2 + (Y - c) ** 2 <= r_in * r_in
    xy = np.stack([X[inside], Y[inside]], axis=1)
    slots = np.concatenate([np.column_stack([np.repeat(xy, len(zs), axis=0),
                                             np.tile(zs, len(xy))])])
    if ncells > len(slots):
        raise RuntimeError(f"{ncells} cells do not fit in {len(slots)} tube slots")
    pick = np.sort(rng.choice(len(slots), size=ncells, replace=False))
    pos = slots[pick] + (rng.random((ncells, 3)) * 2.0 - 1.0) * np.array([0.04, 0.04, 0.05])
    pos = _wrap(pos, geom)
    base = np.array([1.0, 0.0, 0.0, 0.0])
    quat = tilted_quaternions(rng, ncells, base, math.radians(tilt_max_deg))
    return geom, cells_dict(pos, quat), params(**pover)


def hematocrit(geom, ncells, semi_axes=(4.0, 4.0, 1.5)):
    V = geom["nx"] * geom["ny"] * geom["nz"]
    a = semi_axes
    return ncells * 4.0 / 3.0 * math.pi * a[0] * a[1] * a[2] / V
