"""Pins of the oracle's shape function, sampling and spreading (Sec. 2.2, 2.4).

Checked against properties that hold independently of the oracle's code:
Peskin's four-point kernel identities (partition of unity, zero first moment,
sum of squares 3/8), the support size the paper prints, the normalisation and
summation-by-parts identities the paper states, body coordinates computed by
scipy's rotation routine, exactness of the smeared fields on uniform and
rigid-rotation flows, and the momentum / angular-momentum content of the
reaction force density.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as orc
from tests.golden import load_golden


def _Q(q):
    return orc.quat_to_Q(q)


def test_peskin_kernel_identities():
    rng = np.random.default_rng(1)
    assert orc.peskin(0.0) == 0.5
    assert abs(orc.peskin(1.0) - 0.25) < 1e-15
    assert abs(orc.peskin(1.0 + 1e-12) - 0.25) < 1e-10  # continuous at r = 1
    assert orc.peskin(2.0) == 0.0 and orc.peskin(2.5) == 0.0
    for r in rng.random(50):
        js = np.arange(-3, 5)
        ph = np.array([orc.peskin(r - j) for j in js])
        assert np.all(ph >= 0)
        assert abs(ph.sum() - 1.0) < 1e-14             # partition of unity
        assert abs(((js - r) * ph).sum()) < 1e-14      # zero first moment
        assert abs((ph * ph).sum() - 3.0 / 8.0) < 1e-14  # Peskin's sum of squares


def test_printed_kernel_is_not_normalised():
    """The branches as printed in Sec. 2.2 (s = |y|/xi) are discontinuous at
    s = 1/2 and do not sum to one on the lattice at xi = 2, which contradicts
    the normalisation the paper states right after; hence the reading of
    Peskin's kernel."""
    def printed(y, xi=2.0):
        s = abs(y) / xi
        if s <= 0.5:
            return (5 - 4 * s - np.sqrt(1 + 8 * s - 16 * s * s)) / 8
        if s <= 1.0:
            return (3 - 4 * s - np.sqrt(max(-7 + 24 * s - 16 * s * s, 0.0))) / 8
        return 0.0
    assert abs(printed(0.999) - printed(1.001)) > 0.2
    sums = [sum(printed(r - j) for j in range(-3, 5)) for r in (0.0, 0.3, 0.5)]
    assert all(abs(s - 1.0) > 0.4 for s in sums)


def test_xi2_axis_aligned_partition_of_unity_and_support():
    g = load_golden("paper_numbers.txt")
    rng = np.random.default_rng(2)
    dims = (12, 12, 12)
    for _ in range(5):
        R = 3.0 + 6.0 * rng.random(3)
        S, w, d, D = orc.shape_field(dims, None, R, np.eye(3), (2.0, 2.0, 2.0))
        assert abs(S - 1.0) < 1e-14 and abs(w.sum() - 1.0) < 1e-14
        zz, yy, xx = np.mgrid[0:12, 0:12, 0:12]
        X = np.stack([xx, yy, zz], axis=-1).astype(float)
        assert np.allclose(np.einsum("zyx,zyxa->a", w, X - R), 0.0, atol=1e-13)
        assert np.count_nonzero(w) == int(g["support_nodes_xi2"])


def _lattice_coords(dims):
    nx, ny, nz = dims
    zz, yy, xx = np.mgrid[0:nz, 0:ny, 0:nx]
    return np.stack([xx, yy, zz], axis=-1).astype(float)


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_normalisation_and_summation_by_parts(seed):
    """sum delta = 1 for any pose (normalised reading) and the identity the
    paper states, sum_x (x - T)_a d_b delta = -delta_ab, plus sum_x d delta = 0,
    both exact under the lattice central difference."""
    rng = np.random.default_rng(seed)
    dims = (20, 20, 20)
    q = rng.normal(size=4)
    R = 8.0 + 4.0 * rng.random(3)
    S, w, d, D = orc.shape_field(dims, None, R, _Q(q), (4.0, 4.0, 1.5))
    X = _lattice_coords(dims)
    assert abs(d.sum() - 1.0) < 1e-13
    M = np.einsum("zyxa,zyxb->ab", X - R, D)
    assert np.allclose(M, -np.eye(3), atol=1e-12)
    assert np.allclose(D.sum(axis=(0, 1, 2)), 0.0, atol=1e-14)


def test_support_matches_body_coordinates_from_scipy():
    rng = np.random.default_rng(6)
    dims = (20, 20, 20)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    R = np.array([9.3, 10.1, 9.7])
    xi = np.array([4.0, 4.0, 1.5])
    S, w, d, D = orc.shape_field(dims, None, R, _Q(q), xi)
    rot = Rotation.from_quat([q[1], q[2], q[3], q[0]])  # scipy: (x, y, z, w), body -> lab
    X = _lattice_coords(dims).reshape(-1, 3)
    y = rot.inv().apply(X - R)
    inside = np.all(np.abs(y) < xi, axis=1)
    assert np.array_equal(w.reshape(-1) > 0, inside)
    # the product of Peskin factors, evaluated independently through scipy's
    # body coordinates at a few support nodes
    idx = np.flatnonzero(inside)[::37]
    for n in idx:
        ref = np.prod([orc.peskin(2 * y[n, b] / xi[b]) for b in range(3)])
        assert abs(w.reshape(-1)[n] - ref) < 1e-14


def test_theta_peak_of_paper_kappa():
    """theta = 1 - (1 - w)^kappa with the raw product w (peak phi(0)^3 = 1/8):
    theta ~ 0.93 at the centre for kappa = 20 and theta in [0, 1) elsewhere."""
    dims = (16, 16, 16)
    G, th = orc.spread_cell(dims, None, (8.0, 8.0, 8.0), np.eye(3), (4.0, 4.0, 1.5), 20.0,
                            np.zeros(3), np.zeros(3))
    assert abs(th.max() - (1.0 - (7.0 / 8.0) ** 20)) < 1e-14
    assert np.all(th >= 0) and np.all(th < 1)


def _rand_pose(rng, lo=8.0, span=4.0):
    q = rng.normal(size=4)
    return lo + span * rng.random(3), _Q(q)


@pytest.mark.parametrize("seed", [7, 8])
def test_sampling_uniform_and_rigid_rotation(seed):
    """Uniform u0: u~ = u0, omega~ = 0.  Rigid rotation u = W x (x - c):
    curl = 2 W exactly under central differences, so omega~ = 2 W, and
    u~ = W x (sum_x delta x - c)."""
    rng = np.random.default_rng(seed)
    dims = (24, 24, 24)
    N = 24 ** 3
    R, Q = _rand_pose(rng)
    u0 = rng.normal(size=3) * 1e-3
    ut, wt, TS = orc.sample_cell(dims, None, np.tile(u0, (N, 1)), None, R, Q, (4, 4, 1.5), 0.0)
    assert np.allclose(ut, u0, rtol=1e-13) and np.allclose(wt, 0.0, atol=1e-17)
    Wv = rng.normal(size=3) * 1e-3
    c = np.array([12.0, 12.0, 12.0])
    X = _lattice_coords(dims).reshape(-1, 3)
    u = np.cross(Wv, X - c)
    ut, wt, _ = orc.sample_cell(dims, None, u, None, R, Q, (4, 4, 1.5), 0.0)
    assert np.allclose(wt, 2 * Wv, rtol=1e-12)
    S, w, d, D = orc.shape_field(dims, None, R, Q, (4, 4, 1.5))
    centroid = np.einsum("n,na->a", d.reshape(-1), X)
    assert np.allclose(ut, np.cross(Wv, centroid - c), rtol=1e-12, atol=1e-18)


def test_vorticity_sample_equals_summation_by_parts_form():
    """Sum_x delta (curl u) computed by the oracle equals -sum_x D delta x u,
    evaluated here from the oracle's gradient (the two are equal by summation
    by parts on a periodic lattice)."""
    rng = np.random.default_rng(9)
    dims = (18, 16, 14)
    N = 18 * 16 * 14
    R, Q = _rand_pose(rng, lo=6.0)
    u = rng.normal(size=(N, 3)) * 1e-3
    ut, wt, _ = orc.sample_cell(dims, None, u, None, R, Q, (4, 4, 1.5), 0.0)
    S, w, d, D = orc.shape_field(dims, None, R, Q, (4, 4, 1.5))
    sbp = -np.cross(D.reshape(-1, 3), u).sum(axis=0)
    assert np.allclose(wt, sbp, rtol=1e-11, atol=1e-17)
    assert np.allclose(ut, (d.reshape(-1)[:, None] * u).sum(0), rtol=1e-12)


def _sym(rng):
    A = rng.normal(size=(3, 3))
    A = A + A.T
    return np.array([A[0, 0], A[1, 1], A[2, 2], A[0, 1], A[0, 2], A[1, 2]])


def test_elongational_torque_vanishes_for_a_sphere():
    """A spherical diffused particle (xi equal on all axes, centred on a node)
    has cubic lattice symmetry; the sum of (sigma n) x r then vanishes for any
    uniform symmetric stress (Sec. 2.2: zero for spherical solutes)."""
    rng = np.random.default_rng(10)
    dims = (16, 16, 16)
    N = 16 ** 3
    for _ in range(3):
        s6 = _sym(rng)
        sig = np.tile(s6, (N, 1))
        _, _, TS = orc.sample_cell(dims, None, np.zeros((N, 3)), sig, (8.0, 8.0, 8.0), np.eye(3),
                                   (3.0, 3.0, 3.0), 0.04)
        # rounding level only: the terms are of size alpha |sigma| xi
        assert np.allclose(TS, 0.0, atol=1e-14 * 0.04 * np.abs(s6).max() * 3.0)


def test_elongational_torque_turns_flat_cell_towards_extension():
    """Simple shear u = g y x (g > 0): sigma_xy > 0, extensional axis at +45
    degrees, vorticity clockwise.  The elongational torque must turn a flat
    cell towards the extensional axis (Sec. 2.3): counter-clockwise (T_z > 0)
    when its long axes lie along the flow (short axis along y), clockwise when
    its short axis lies along the flow; it is linear in alpha and in sigma."""
    dims = (16, 16, 16)
    N = 16 ** 3
    sig = np.zeros((N, 6))
    sig[:, 3] = 1e-5
    R = (8.0, 8.0, 8.0)
    Q_flat = Rotation.from_euler("x", -90, degrees=True).as_matrix()   # body z -> lab y
    Q_edge = Rotation.from_euler("y", 90, degrees=True).as_matrix()    # body z -> lab x
    _, _, T1 = orc.sample_cell(dims, None, np.zeros((N, 3)), sig, R, Q_flat, (4, 4, 1.5), 0.04)
    _, _, T2 = orc.sample_cell(dims, None, np.zeros((N, 3)), sig, R, Q_edge, (4, 4, 1.5), 0.04)
    assert T1[2] > 0 and T2[2] < 0
    assert np.allclose(T1[:2], 0.0, atol=1e-12 * abs(T1[2]))
    _, _, T3 = orc.sample_cell(dims, None, np.zeros((N, 3)), 2 * sig, R, Q_flat, (4, 4, 1.5), 0.02)
    assert np.allclose(T3, T1, rtol=1e-13)


@pytest.mark.parametrize("seed", [11, 12])
def test_spread_momentum_and_angular_momentum(seed):
    """Reaction force density of one cell: sum_x G = -J/h, sum_x (x - R) x
    G_torque = -L/h with zero net force from the torque term, and adjointness
    with sampling: sum_x G_F . u = -(J/h) . u~ for any u."""
    rng = np.random.default_rng(seed)
    dims = (22, 22, 22)
    N = 22 ** 3
    R, Q = _rand_pose(rng, lo=9.0)
    J = rng.normal(size=3) * 1e-4
    L = rng.normal(size=3) * 1e-3
    X = _lattice_coords(dims).reshape(-1, 3)
    G, th = orc.spread_cell(dims, None, R, Q, (4, 4, 1.5), 20.0, J, np.zeros(3))
    assert np.allclose(G.sum(0), -J, rtol=1e-12)
    u = rng.normal(size=(N, 3))
    ut, _, _ = orc.sample_cell(dims, None, u, None, R, Q, (4, 4, 1.5), 0.0)
    assert abs(np.einsum("na,na->", G, u) + J @ ut) < 1e-12 * np.abs(J).sum() * np.abs(u).max()
    Gt, _ = orc.spread_cell(dims, None, R, Q, (4, 4, 1.5), 20.0, np.zeros(3), L)
    assert np.allclose(Gt.sum(0), 0.0, atol=1e-16)
    assert np.allclose(np.cross(X - R, Gt).sum(0), -L, rtol=1e-11)


def test_shape_renormalises_over_fluid_nodes():
    """A support cut by a solid wall: delta = 0 at solid nodes and sums to 1
    over the fluid ones."""
    dims = (16, 16, 16)
    solid = np.zeros((16, 16, 16), dtype=np.uint8)
    solid[:, 0:6, :] = 1
    S, w, d, D = orc.shape_field(dims, solid, (8.0, 7.2, 8.0), np.eye(3), (4, 4, 1.5))
    assert np.all(d[solid == 1] == 0) and abs(d.sum() - 1.0) < 1e-14
