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

def periodic_box(nx, ny=None, nz=None, body_force=(0.0, 0.0, 0.0), body_force_wave=(0.0, 0.0, 0.0)):
    """Fully periodic box; ``body_force_wave`` is the amplitude of a force
    density profile A sin(2 pi y / ny) added to the uniform ``body_force``
    (a Kolmogorov flow)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return dict(nx=nx, ny=ny, nz=nz, periodic=(1, 1, 1), solid=None,
                body_force=tuple(float(b) for b in body_force),
                body_force_wave=tuple(float(b) for b in body_force_wave))


def kolmogorov_amplitude(ny, rate, nu=1.0 / 6.0):
    """Amplitude A of the force A sin(k y), k = 2 pi / ny, whose steady plasma
    flow u_x = A / (nu k^2) sin(k y) has the peak shear rate ``rate``."""
    k = 2.0 * math.pi / ny
    return nu * k * rate


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


NODE_INLET, NODE_OUTLET = 1, 2


def open_tube(n, length, radius, umax):
    """Tube along z (axis at ((n-1)/2, (n-1)/2), nodes farther than
    ``radius`` solid) with a velocity inlet on the plane z = 0 (Poiseuille
    profile umax (1 - r^2/radius^2) along +z) and a pressure outlet on the
    plane z = length - 1; the z index wraps, so the two planes are adjacent
    and neither pulls from the other."""
    g = tube(n, radius, length)
    nt = np.zeros((length, n, n), dtype=np.uint8)
    fluid = g["solid"] == 0
    nt[0][fluid[0]] = NODE_INLET
    nt[length - 1][fluid[length - 1]] = NODE_OUTLET
    c = (n - 1) / 2.0
    g.update(node_type=nt, inlet_center=(c, c), inlet_radius=float(radius), inlet_umax=float(umax))
    return g


def y_bifurcation(n, r_parent, r_daughter, angle_deg=35.0, z_split=None, umax=0.02, nz=None):
    """Y-shaped vessel in an n x n x nz box: a parent tube of radius r_parent
    along z from the inlet plane z = 0 to the branch point ((n-1)/2, (n-1)/2,
    z_split), two daughter tubes of radius r_daughter leaving it at
    +-angle_deg from the z axis in the x-z plane up to the outlet plane
    z = nz - 1, and a sphere of radius r_parent joining them.  Velocity inlet
    (Poiseuille profile of peak umax in the parent) on z = 0, pressure outlets
    on z = nz - 1; solid elsewhere."""
    nz = n if nz is None else nz
    z_split = nz // 2 if z_split is None else z_split
    c = (n - 1) / 2.0
    th = math.radians(angle_deg)
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    dx, dy = x - c, y - c
    rr = dx * dx + dy * dy
    fluid = np.zeros((nz, n, n), dtype=bool)
    for zi in range(nz):  # one plane at a time
        dz = zi - z_split
        f = rr + dz * dz < r_parent ** 2
        if zi <= z_split:
            f |= rr < r_parent ** 2
        for sgn in (-1.0, 1.0):
            t = dx * sgn * math.sin(th) + dz * math.cos(th)
            f |= (t >= 0.0) & (rr + dz * dz - t * t < r_daughter ** 2)
        fluid[zi] = f
    solid = (~fluid).astype(np.uint8)
    nt = np.zeros((nz, n, n), dtype=np.uint8)
    nt[0][fluid[0]] = NODE_INLET
    nt[nz - 1][fluid[nz - 1]] = NODE_OUTLET
    return dict(nx=n, ny=n, nz=nz, periodic=(0, 0, 1), solid=solid, body_force=(0.0, 0.0, 0.0),
                node_type=nt, inlet_center=(c, c), inlet_radius=float(r_parent), inlet_umax=float(umax),
                branch=dict(z_split=z_split, angle=angle_deg, r_parent=r_parent, r_daughter=r_daughter))


def y_bifurcation_cells(rng, geom, hematocrit, wall_clearance=6.0, end_clearance=20.0, pitch=8.3, zpitch=3.3,
                        tilt_max_deg=1.5):
    """Cells in the slots of the tube workload's lattice (hexagonal of pitch
    ``pitch`` across, ``zpitch`` along z; short axis along z) that lie inside
    the Y at least ``wall_clearance`` from its walls and ``end_clearance``
    from the inlet and outlet planes; as many as give ``hematocrit`` of the
    lumen, or all slots if fewer."""
    n, nz = geom["nx"], geom["nz"]
    b = geom["branch"]
    c = (n - 1) / 2.0
    th = math.radians(b["angle"])
    dy = pitch * math.sqrt(3.0) / 2.0
    pts = []
    k = int(math.ceil(n / pitch)) + 1
    for zz in np.arange(end_clearance, nz - 1 - end_clearance, zpitch):
        for i, yy in enumerate(np.arange(0.0, n, dy)):
            xs = np.arange(-k, k + 1) * pitch + c + 0.5 * pitch * (i % 2)
            xs = xs[(xs >= 0) & (xs < n)]
            px, py = xs - c, yy - c
            pz = zz - b["z_split"]
            m = np.full(xs.shape, -np.inf)
            if zz <= b["z_split"]:
                m = np.maximum(m, b["r_parent"] - np.hypot(px, py))
            m = np.maximum(m, b["r_parent"] - np.sqrt(px * px + py * py + pz * pz))
            for sgn in (-1.0, 1.0):
                ax = (sgn * math.sin(th), 0.0, math.cos(th))
                t = px * ax[0] + py * ax[1] + pz * ax[2]
                d = np.sqrt(np.maximum(px * px + py * py + pz * pz - t * t, 0.0))
                m = np.maximum(m, np.where(t >= 0.0, b["r_daughter"] - d, -np.inf))
            for x in xs[m >= wall_clearance]:
                pts.append((x, yy, zz))
    pts = np.array(pts).reshape(-1, 3)
    want = int(round(hematocrit * fluid_count(geom) / CELL_VOLUME))
    ncell = min(want, len(pts))
    pick = np.sort(rng.choice(len(pts), size=ncell, replace=False))
    pos = pts[pick] + (rng.random((ncell, 3)) * 2.0 - 1.0) * np.array([0.04, 0.04, 0.03])
    quat = tilted_quaternions(rng, ncell, np.array([1.0, 0.0, 0.0, 0.0]), math.radians(tilt_max_deg))
    return cells_dict(pos, quat)


def ybif_workload(n=512, r_parent=60.0, r_daughter=45.0, angle_deg=35.0, hematocrit=0.40, umax=0.02,
                  seed=SEED_BASE + 5, **pover):
    """The vascular workload: Y-bifurcation in n^3 (parent radius 60,
    daughters radius 45 at +-35 degrees), velocity inlet / pressure outlets,
    cells at up to ``hematocrit`` of the lumen (slot-limited)."""
    rng = np.random.default_rng(seed)
    geom = y_bifurcation(n, r_parent, r_daughter, angle_deg, umax=umax)
    cells = y_bifurcation_cells(rng, geom, hematocrit)
    return geom, cells, params(**pover)


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


def tube_workload(n=256, radius=120.0, ncells=51846, body_force=None, seed=SEED_BASE + 3,
                  wall_clearance=6.0, pitch=8.3, zpitch=3.3, tilt_max_deg=1.5, **pover):
    """Straight tube of the given radius along z in an n^3 box (periodic in
    z) with cells in the slots of a lattice: hexagonal of pitch ``pitch`` in
    the cross-section, inside radius - ``wall_clearance`` (the Gay-Berne
    contact distance of a cell edge-on to a wall particle is 5.7), and
    n / floor(n / zpitch) along z; short axis along z, a random spin about it
    and a tilt of at most ``tilt_max_deg``.  Default: radius 120 in 256^3 (11,582,464
    fluid nodes) with 51,846 cells, hematocrit 0.45 of the lumen, driven by
    the axial force density 2 nu0 rate / radius that gives a wall shear rate
    1e-4 per step in plain plasma (nu0 = 1/6), the periodic stand-in for a
    pressure drop."""
    rng = np.random.default_rng(seed)
    if body_force is None:
        body_force = (0.0, 0.0, 2.0 * (1.0 / 6.0) * 1e-4 / radius)
    geom = tube(n, radius, body_force=body_force)
    c = (n - 1) / 2.0
    r_in = radius - wall_clearance
    dy = pitch * math.sqrt(3.0) / 2.0
    xy = []
    k = int(math.ceil(r_in / pitch)) + 1
    for i, y in enumerate(np.arange(-r_in, r_in + 1e-9, dy)):
        xs = np.arange(-k, k + 1) * pitch + 0.5 * pitch * (i % 2)  # odd rows shifted half a pitch
        for x in xs[xs * xs + y * y <= r_in * r_in]:
            xy.append((c + x, c + y))
    xy = np.array(xy)
    zs = slot_centres(n, zpitch, True)
    slots = np.column_stack([np.repeat(xy, len(zs), axis=0), np.tile(zs, len(xy))])
    if ncells > len(slots):
        raise RuntimeError(f"{ncells} cells do not fit in {len(slots)} tube slots")
    pick = np.sort(rng.choice(len(slots), size=ncells, replace=False))
    pos = slots[pick] + (rng.random((ncells, 3)) * 2.0 - 1.0) * np.array([0.04, 0.04, 0.03])
    pos = _wrap(pos, geom)
    base = np.array([1.0, 0.0, 0.0, 0.0])
    quat = tilted_quaternions(rng, ncells, base, math.radians(tilt_max_deg))
    return geom, cells_dict(pos, quat), params(**pover)


def tube_slab(nz=20, **kw):
    """A slab of the tube workload: its cross-section (radius 120 in 256 x
    256, the same drive) over nz planes, periodic along z, with the cells
    of the slot layers whose centres lie below nz - 1.65 (the first six at
    nz = 20, each layer's slots as in the full tube; the layers across the
    periodic seam stay more than a face-to-face contact apart).  The same
    geometry and cell density at 1/12.8 of the size: a bounded sample of
    the tube for timing the oracle."""
    geom, cells, params = tube_workload(**kw)
    keep = cells["pos"][:, 2] < nz - 1.65
    slab = tube(geom["nx"], 120.0 if "radius" not in kw else kw["radius"], length=nz,
                body_force=geom["body_force"])
    return slab, cells_dict(cells["pos"][keep], cells["quat"][keep]), params


def tube_hematocrit(geom, ncells, semi_axes=(4.0, 4.0, 1.5)):
    """Cell volume fraction of the fluid nodes (the lumen)."""
    a = semi_axes
    return ncells * 4.0 / 3.0 * math.pi * a[0] * a[1] * a[2] / fluid_count(geom)


def hematocrit(geom, ncells, semi_axes=(4.0, 4.0, 1.5)):
    V = geom["nx"] * geom["ny"] * geom["nz"]
    a = semi_axes
    return ncells * 4.0 / 3.0 * math.pi * a[0] * a[1] * a[2] / V


# ---------------------------------------------------------------------------
# request stream of the batched-serving workload
# ---------------------------------------------------------------------------

SERVING_BOXES = ((32, 32, 32), (48, 48, 48), (64, 64, 128), (96, 96, 96))


def slot_lattice_cells(rng, geom, ncells, dense, wall_clearance=6.0, tilt_max_deg=None):
    """Cells in the slots of a lattice, short axis along x: pitches (3.37,
    8.4, 8.4) leave every pair out of the Gay-Berne range (tilt up to 5
    degrees), (3.05, 8.05, 8.05) hold up to hematocrit 0.5 with neighbours
    inside the range but not overlapping (tilt up to 0.5 degrees, which
    moves a rim by 0.035 of the 0.05 gap).  Centres stay ``wall_clearance``
    from solid y planes.  Returns as many cells as there are slots when
    ``ncells`` is larger."""
    if tilt_max_deg is None:
        tilt_max_deg = 0.5 if dense else 5.0
    px, pyz = (3.05, 8.05) if dense else (3.37, 8.4)
    nx, ny, nz = geom["nx"], geom["ny"], geom["nz"]
    xs = slot_centres(nx, px, True)
    if geom["periodic"][1]:
        ys = slot_centres(ny, pyz, True)
    else:
        ys = slot_centres(ny, pyz, False, wall_clearance, (ny - 1) - wall_clearance)
    zs = slot_centres(nz, pyz, True)
    n = min(ncells, len(xs) * len(ys) * len(zs))
    pos = _wrap(place_slots(rng, (xs, ys, zs), n, (0.02, 0.02, 0.02)), geom)
    base = axis_angle_quat([0.0, 1.0, 0.0], math.pi / 2.0)
    quat = tilted_quaternions(rng, n, base, math.radians(tilt_max_deg))
    return cells_dict(pos, quat)


def serving_request(rng, box=None, walled=None, hematocrit=None, rate=None, steps=None,
                    precision="f16", step_scale=1.0):
    """One request of the serving stream: a periodic box driven by the
    Kolmogorov force (peak shear rate ``rate``) or a walled channel along x
    driven by a uniform force (wall shear rate ``rate``); hematocrit of the
    fluid volume; 2,000-10,000 steps (times ``step_scale``).  Unset fields
    are drawn: box from SERVING_BOXES, walled with probability 1/2,
    hematocrit U[0.1, 0.5], rate log-uniform in [1e-5, 1e-3]."""
    if box is None:
        box = SERVING_BOXES[int(rng.integers(len(SERVING_BOXES)))]
    if walled is None:
        walled = bool(rng.random() < 0.5)
    if hematocrit is None:
        hematocrit = float(rng.uniform(0.1, 0.5))
    if rate is None:
        rate = float(10.0 ** rng.uniform(-5.0, -3.0))
    if steps is None:
        steps = int(rng.integers(2000, 10001))
    steps = max(2, int(round(steps * step_scale / 2.0)) * 2)
    nx, ny, nz = box
    nu = 1.0 / 6.0
    if walled:
        geom = plane_channel(nx, ny, nz, body_force=(2.0 * nu * rate / (ny - 2), 0.0, 0.0))
    else:
        geom = periodic_box(nx, ny, nz, body_force_wave=(kolmogorov_amplitude(ny, rate, nu), 0.0, 0.0))
    ncells = int(round(hematocrit * fluid_count(geom) / CELL_VOLUME))
    cells = slot_lattice_cells(rng, geom, ncells, dense=hematocrit > 0.35)
    info = dict(box=box, walled=walled, hematocrit=len(cells["pos"]) * CELL_VOLUME / fluid_count(geom),
                rate=rate, steps=steps, ncells=len(cells["pos"]))
    return geom, cells, params(precision=precision), steps, info


def serving_stream(n, seed=SEED_BASE + 4, precision="f16", step_scale=1.0):
    """The first n requests of the seeded serving stream."""
    rng = np.random.default_rng(seed)
    return [serving_request(rng, precision=precision, step_scale=step_scale) for _ in range(n)]
