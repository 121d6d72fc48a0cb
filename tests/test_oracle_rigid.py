"""Pins of the oracle's rigid-body integrator (App. A).

Closed forms of the scheme: exponential friction, the geometric approach to
the terminal velocity hF / (2 M sinh(gamma h / 2)) under a constant force,
exact rotation about a principal axis, the right-hand sense of dQ/dt =
Q [Omega]x, exact conservation of the lab angular momentum, and an energy
error that stays bounded and scales as h^2 (DLM splitting, cited in App. A).
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as orc

M = 10.0
I_ISO = np.array([1000.0, 1000.0, 1000.0])


def _run(nsteps, R, Q, V, Om, F, T, M, I, gT, gR):
    """The cached velocity-Verlet sequence of the coupled step: close the
    previous step (not on the first), then open the next."""
    Q = np.asarray(Q, float).reshape(9)
    hist = []
    for n in range(nsteps):
        if n > 0:
            V, Om = orc.rigid_close(V, Om, F, T, M, I, gT, gR)
        R, Qm, V, Om = orc.rigid_open(R, Q, V, Om, F, T, M, I, gT, gR)
        Q = Qm.reshape(9)
        hist.append((R.copy(), Qm.copy(), V.copy(), Om.copy()))
    return hist


def test_friction_only_decay():
    g = 0.1
    V0 = np.array([1e-3, -2e-3, 5e-4])
    Om0 = np.array([1e-4, 2e-4, -3e-4])
    hist = _run(20, np.zeros(3), np.eye(3), V0, Om0, np.zeros(3), np.zeros(3), M, I_ISO, g, 2 * g)
    for n, (R, Q, V, Om) in enumerate(hist, start=1):
        # first step: only the opening half; every later step a full one
        assert np.allclose(V, V0 * np.exp(-g * (n - 0.5)), rtol=1e-13)
        assert np.allclose(Om, Om0 * np.exp(-2 * g * (n - 0.5)), rtol=1e-12)


def test_constant_force_terminal_velocity():
    g = 0.1
    F = np.array([2e-4, 0.0, -1e-4])
    hist = _run(400, np.zeros(3), np.eye(3), np.zeros(3), np.zeros(3), F, np.zeros(3), M, I_ISO, g, g)
    Vinf = F / (2 * M * np.sinh(g / 2))
    # recursion V_{n+1} = e^{-g} V_n + e^{-g/2} F/M from V_1 = e^{-g/2} F/(2M)
    V = np.exp(-g / 2) * F / (2 * M)
    for n, (_, _, Vn, _) in enumerate(hist, start=1):
        assert np.allclose(Vn, V, rtol=1e-12, atol=1e-20)
        V = np.exp(-g) * V + np.exp(-g / 2) * F / M
    assert np.allclose(hist[-1][2], Vinf, rtol=1e-10)
    # drift: R_n = sum of the velocities after each opening half
    assert np.allclose(hist[-1][0], sum(h[2] for h in hist), rtol=1e-12)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_rotation_about_principal_axis_is_exact(axis):
    I = np.array([1000.0, 700.0, 1300.0])
    w = 0.013
    Om0 = np.zeros(3)
    Om0[axis] = w
    Q0 = Rotation.random(random_state=axis).as_matrix()
    hist = _run(50, np.zeros(3), Q0, np.zeros(3), Om0, np.zeros(3), np.zeros(3), M, I, 0.0, 0.0)
    for n, (_, Q, _, Om) in enumerate(hist, start=1):
        ref = Q0 @ Rotation.from_rotvec(n * w * np.eye(3)[axis]).as_matrix()
        assert np.allclose(Q, ref, atol=1e-13) and np.allclose(Om, Om0, atol=1e-16)


def test_right_hand_sense_of_rotation():
    """Positive body Omega_z turns the body x axis towards +y (dQ/dt = Q [Omega]x)."""
    hist = _run(10, np.zeros(3), np.eye(3), np.zeros(3), np.array([0, 0, 0.05]), np.zeros(3),
                np.zeros(3), M, I_ISO, 0.0, 0.0)
    Q = hist[-1][1]
    assert Q[1, 0] > 0 and abs(Q[1, 0] - np.sin(0.5)) < 1e-13


def _energy_and_L(Q, Om, I):
    return 0.5 * np.sum(I * Om * Om), Q @ (I * Om)


@pytest.mark.parametrize("seed", [0, 1])
def test_free_asymmetric_top_conserves_angular_momentum_and_energy(seed):
    rng = np.random.default_rng(seed)
    I = np.array([1000.0, 1500.0, 2300.0])
    Q0 = Rotation.random(random_state=rng).as_matrix()
    errs = []
    for s in (0.02, 0.01):
        Om0 = s * np.array([0.6, -0.3, 0.74])
        E0, L0 = _energy_and_L(Q0, Om0, I)
        hist = _run(2000, np.zeros(3), Q0, np.zeros(3), Om0, np.zeros(3), np.zeros(3), M, I, 0.0, 0.0)
        worst = 0.0
        for _, Q, _, Om in hist:
            E, L = _energy_and_L(Q, Om, I)
            assert np.allclose(L, L0, rtol=1e-11, atol=1e-14 * np.linalg.norm(L0))
            assert abs(np.linalg.det(Q) - 1) < 1e-12
            worst = max(worst, abs(E / E0 - 1))
        errs.append(worst)
    assert errs[0] < 1e-3
    # bounded energy error of a second-order splitting: ~ (Omega h)^2
    assert 3.0 < errs[0] / errs[1] < 5.0
