"""Pins of the oracle's Gay-Berne pair (Sec. 2.5, App. B).

Arbiters: the textbook WCA potential (equal spheres reduce the pair to it),
the contact distances the paper states (face-to-face 2 a_min), finite
differences of the oracle's own energy for the force (-grad u) and for both
torques (-du/dtheta under small rotations), Newton's third law and the
angular-momentum identity the paper states at the end of App. B.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as orc

EPS0 = 0.01
A_CELL = np.array([4.0, 4.0, 1.5])
SMIN = np.sqrt(2 * (1.5 ** 2 + 1.5 ** 2))  # sigma_min of two identical cells (Sec. 2.5)


def _A(Q, a):
    return Q @ np.diag(np.asarray(a) ** 2) @ Q.T


def _wca(R, sigma, eps):
    rc = 2 ** (1 / 6) * sigma
    return np.where(R <= rc, 4 * eps * ((sigma / R) ** 12 - (sigma / R) ** 6) + eps, 0.0)


def test_equal_spheres_reduce_to_wca():
    a = 2.0
    A = _A(np.eye(3), (a, a, a))
    smin = np.sqrt(2 * (a * a + a * a))  # = 2a
    rng = np.random.default_rng(0)
    for R in np.linspace(3.2, 4.6, 15):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        u, F, ti, tj, _ = orc.gb_pair(R * n, A, A, smin, EPS0)
        assert abs(u - _wca(R, 2 * a, EPS0)) < 1e-13
        assert np.allclose(ti, 0.0, atol=1e-15) and np.allclose(tj, 0.0, atol=1e-15)


def test_contact_distances_of_identical_oblate_cells():
    """Face-to-face: contact (rho = 1, u = eps0) at 2 a_min; edge-to-edge at
    2 a_max; sigma_min is the face-to-face contact distance (Sec. 2.5)."""
    A = _A(np.eye(3), A_CELL)
    u, *_ = orc.gb_pair([0, 0, 3.0], A, A, SMIN, EPS0)
    assert abs(u - EPS0) < 1e-14
    u, *_ = orc.gb_pair([8.0, 0, 0], A, A, SMIN, EPS0)
    assert abs(u - EPS0) < 1e-14
    # range: u vanishes continuously at rho = 2^(1/6)
    Rc = 8.0 + (2 ** (1 / 6) - 1) * SMIN
    u1, F1, *_ = orc.gb_pair([Rc - 1e-7, 0, 0], A, A, SMIN, EPS0)
    u2, F2, *_ = orc.gb_pair([Rc + 1e-7, 0, 0], A, A, SMIN, EPS0)
    assert u1 < 1e-12 and u2 == 0.0 and np.linalg.norm(F1) < 1e-6


def _random_interacting(rng):
    while True:
        Qi = Rotation.random(random_state=rng).as_matrix()
        Qj = Rotation.random(random_state=rng).as_matrix()
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        Ai, Aj = _A(Qi, A_CELL), _A(Qj, A_CELL)
        # bisect for the contact distance along n, then back off into the shell
        lo, hi = 0.5, 12.0
        for _ in range(80):
            mid = 0.5 * (lo + hi)
            u, *_ = orc.gb_pair(mid * n, Ai, Aj, SMIN, EPS0)
            if u > EPS0:
                lo = mid
            else:
                hi = mid
        R = hi + rng.uniform(0.02, 0.3)
        u, *_ = orc.gb_pair(R * n, Ai, Aj, SMIN, EPS0)
        if 1e-6 < u < EPS0:
            return R * n, Ai, Aj, Qi, Qj


@pytest.mark.parametrize("seed", range(6))
def test_force_is_minus_energy_gradient(seed):
    rng = np.random.default_rng(100 + seed)
    d, Ai, Aj, *_ = _random_interacting(rng)
    u, F, *_ = orc.gb_pair(d, Ai, Aj, SMIN, EPS0)
    h = 1e-6
    Ffd = np.zeros(3)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        up, *_ = orc.gb_pair(d + e, Ai, Aj, SMIN, EPS0)
        um, *_ = orc.gb_pair(d - e, Ai, Aj, SMIN, EPS0)
        Ffd[a] = -(up - um) / (2 * h)
    assert np.allclose(F, Ffd, rtol=1e-6, atol=1e-9 * np.abs(F).max())


@pytest.mark.parametrize("seed", range(6))
def test_torques_are_minus_energy_derivative_under_rotation(seed):
    rng = np.random.default_rng(200 + seed)
    d, Ai, Aj, Qi, Qj = _random_interacting(rng)
    u, F, ti, tj, _ = orc.gb_pair(d, Ai, Aj, SMIN, EPS0)
    h = 1e-6
    for which, tau in (("i", ti), ("j", tj)):
        tfd = np.zeros(3)
        for a in range(3):
            vals = []
            for s in (+1, -1):
                Rm = Rotation.from_rotvec(s * h * np.eye(3)[a]).as_matrix()
                if which == "i":
                    up, *_ = orc.gb_pair(d, _A(Rm @ Qi, A_CELL), Aj, SMIN, EPS0)
                else:
                    up, *_ = orc.gb_pair(d, Ai, _A(Rm @ Qj, A_CELL), SMIN, EPS0)
                vals.append(up)
            tfd[a] = -(vals[0] - vals[1]) / (2 * h)
        assert np.allclose(tau, tfd, rtol=1e-6, atol=1e-9 * np.abs(tau).max())


@pytest.mark.parametrize("seed", range(4))
def test_third_law_and_angular_momentum_identity(seed):
    """F_ji = -F_ij and tau_i + tau_j = -R_ij x F_ij (end of App. B)."""
    rng = np.random.default_rng(300 + seed)
    d, Ai, Aj, *_ = _random_interacting(rng)
    u, F, ti, tj, _ = orc.gb_pair(d, Ai, Aj, SMIN, EPS0)
    u2, F2, tj2, ti2, _ = orc.gb_pair(-d, Aj, Ai, SMIN, EPS0)
    assert abs(u - u2) < 1e-15 and np.allclose(F2, -F, rtol=1e-12)
    assert np.allclose(ti2, ti, rtol=1e-10) and np.allclose(tj2, tj, rtol=1e-10)
    assert np.allclose(ti + tj, -np.cross(d, F), rtol=1e-10, atol=1e-14 * np.abs(F).max())


def test_clamp_bounds_deep_overlap():
    A = _A(np.eye(3), A_CELL)
    u, F, ti, tj, cl = orc.gb_pair([0, 0, 1.0], A, A, SMIN, EPS0, rho_floor=0.75)
    assert cl == 1 and np.all(np.isfinite(F))
    u2, F2, *_ = orc.gb_pair([0, 0, 2.25], A, A, SMIN, EPS0, rho_floor=0.75)  # rho = 0.75
    # face to face the force depends on rho only: clamped at R = 1 it equals the
    # force at R = 2.25, where rho = 0.75 unclamped
    assert np.allclose(F, F2, rtol=1e-12) and F[2] > 0


def test_wall_particle_pair():
    """A wall particle is a sphere of radius 1/2 with sigma_min = 1/2
    (Sec. 2.5, last paragraph): for a spherical cell of radius a the pair is
    WCA-shaped with contact at sqrt(2 (a^2 + 1/4))."""
    a = 3.0
    A = _A(np.eye(3), (a, a, a))
    Aw = 0.25 * np.eye(3)
    s = np.sqrt(2 * (a * a + 0.25))
    u, F, ti, tj, _ = orc.gb_pair([0.0, s, 0.0], A, Aw, 0.5, EPS0)
    assert abs(u - EPS0) < 1e-13 and F[1] > 0
