"""Pins of the oracle's lattice-Boltzmann pass (Sec. 2.1) against closed forms.

None of these re-types the oracle's formulas: they check what the paper and
the mathematics fix -- the isotropy of the D3Q19 set, exact conservation,
Galilean fixed points, the closed-form response to a uniform force, the
shear-wave decay rate nu k^2 with nu = c^2 (T - h/2), the Poiseuille profile
between halfway walls and the sign of the stress it carries.
"""
import numpy as np
import pytest

from oracle import oracle as orc


def _rest(N):
    c, w = orc.lattice()
    return np.ascontiguousarray(np.repeat(w[:, None], N, axis=1))


def test_d3q19_isotropy():
    c, w = orc.lattice()
    assert len({tuple(v) for v in c}) == 19
    assert np.isclose(w.sum(), 1.0, atol=1e-15)
    assert np.allclose(np.einsum("p,pa->a", w, c), 0.0, atol=1e-15)
    # second and fourth moments of an isotropic lattice with c^2 = 1/3
    assert np.allclose(np.einsum("p,pa,pb->ab", w, c, c), np.eye(3) / 3.0, atol=1e-15)
    d = np.eye(3)
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
            + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(np.einsum("p,pa,pb,pc,pd->abcd", w, c, c, c, c), iso4, atol=1e-15)
    # paper Sec. 2.1: weights 1/3, 1/18 (first neighbours), 1/36 (second)
    c2 = (c * c).sum(1)
    assert np.allclose(w[c2 == 0], 1 / 3) and np.allclose(w[c2 == 1], 1 / 18)
    assert np.allclose(w[c2 == 2], 1 / 36) and (c2 == 1).sum() == 6 and (c2 == 2).sum() == 12


def test_rest_state_is_fixed_point():
    dims = (5, 4, 3)
    N = 60
    f = _rest(N)
    tau = np.full(N, 0.9)
    rho, u, sig = orc.lb_pass(dims, None, f, None, tau)
    assert np.allclose(f, _rest(N), atol=1e-16)
    assert np.allclose(rho, 1.0, atol=1e-15) and np.allclose(u, 0.0, atol=1e-16)
    assert np.allclose(sig, 0.0, atol=1e-16)


@pytest.mark.parametrize("tau", [0.7, 1.0, 1.6])
def test_uniform_force_closed_form(tau):
    """Uniform force density G in a periodic box: the fluid gains exactly h G
    of momentum per pass and the velocity of pass n (counted from 0) is
    (n + 1/2) G, with rho = 1 throughout.  A missing half-force shift of
    Eq. vel gives n G; a forcing term without the (1 - h/2T) factor gives a
    tau-dependent (1 + 1/2T) gain per pass."""
    dims = (4, 3, 5)
    N = 60
    f = _rest(N)
    G = np.tile([1e-4, -2e-4, 5e-5], (N, 1))
    for n in range(40):
        rho, u, _ = orc.lb_pass(dims, None, f, G, np.full(N, tau))
        assert np.allclose(u, (n + 0.5) * G, rtol=1e-12, atol=0)
        assert np.allclose(rho, 1.0, atol=1e-13)
        c, _w = orc.lattice()
        j = np.einsum("pn,pa->na", f, c)
        assert np.allclose(j, (n + 1) * G, rtol=1e-12, atol=0)


def test_mass_and_momentum_conservation_variable_tau():
    rng = np.random.default_rng(0)
    dims = (6, 5, 7)
    N = 210
    c, w = orc.lattice()
    f = np.ascontiguousarray(w[:, None] * (1.0 + 0.02 * rng.standard_normal((19, N))))
    tau = 0.6 + 2.0 * rng.random(N)
    m0 = f.sum()
    p0 = np.einsum("pn,pa->a", f, c)
    for _ in range(12):
        orc.lb_pass(dims, None, f, None, tau)
    assert abs(f.sum() - m0) < 1e-12 * m0
    assert np.allclose(np.einsum("pn,pa->a", f, c), p0, atol=1e-13)


def _shear_wave_rate(L, tau, steps=(40, 140)):
    """u_x(y) = U sin(2 pi y / L) in a 1 x L x 1 periodic box; returns the
    measured exponential decay rate of the mode between the two step counts."""
    dims = (1, L, 1)
    N = L
    c, w = orc.lattice()
    y = np.arange(L)
    k = 2 * np.pi / L
    ux = 1e-4 * np.sin(k * y)
    # first-order start f = w (1 + 3 c.u); the mode relaxes onto the
    # hydrodynamic branch long before the measurement window
    f = np.ascontiguousarray(w[:, None] * (1.0 + 3.0 * c[:, 0][:, None] * ux[None, :]))
    amp = {}
    for n in range(1, steps[1] + 1):
        _, u, _ = orc.lb_pass(dims, None, f, None, np.full(N, tau))
        if n in steps:
            amp[n] = 2.0 / L * np.sum(u[:, 0] * np.sin(k * y))
    rate = np.log(amp[steps[0]] / amp[steps[1]]) / (steps[1] - steps[0])
    return rate, k


@pytest.mark.parametrize("tau", [0.8, 1.0])
def test_shear_wave_decay_rate(tau):
    """Decay rate nu k^2 with nu = c^2 (T - h/2) = (T - 1/2)/3 (Sec. 2.1); the
    relative error is a lattice artefact O(k^2): it must be small and shrink
    about fourfold when L doubles."""
    nu = (tau - 0.5) / 3.0
    errs = []
    for L in (16, 32, 64):
        steps = (int(0.05 * L * L), int(0.3 * L * L))
        rate, k = _shear_wave_rate(L, tau, steps)
        errs.append(abs(rate / (nu * k * k) - 1.0))
    assert errs[1] < 5e-3 and errs[2] < 2e-3
    assert errs[2] < errs[1] / 2.5 and errs[1] < errs[0] / 2.5


def test_viscosity_ratio_of_paper():
    """Sec. 2.4: nu0 = 1/6 (T0 = 1) and Delta = 2 give an inner (theta = 1,
    T = T0 + Delta) to outer viscosity ratio of 5."""
    from tests.golden import load_golden
    g = load_golden("paper_numbers.txt")
    r_out, _ = _shear_wave_rate(128, g["tau0"], (800, 4800))
    r_in, _ = _shear_wave_rate(128, g["tau0"] + g["delta"], (160, 960))
    assert abs(r_in / r_out - g["viscosity_ratio"]) < 0.01 * g["viscosity_ratio"]


def _poiseuille(ny, tau, G, steps):
    dims = (1, ny, 1)
    N = ny
    solid = np.zeros(N, dtype=np.uint8)
    solid[0] = solid[-1] = 1
    f = _rest(N)
    f[:, solid == 1] = 0.0
    Gf = np.zeros((N, 3))
    Gf[solid == 0, 0] = G
    for _ in range(steps):
        rho, u, sig = orc.lb_pass(dims, solid, f, Gf, np.full(N, tau))
    return solid, rho, u, sig


def test_poiseuille_between_halfway_walls():
    """Steady channel flow driven by a uniform force density G between solid
    planes y = 0 and y = ny-1 (walls half way, at y = 0.5 and ny-1.5):
    the profile is a parabola of curvature -G/nu; shear stress
    sigma_xy = +rho nu du/dy = -G (y - y_c) (this fixes the sign of
    Eq. stresstensorLB); the wall drag balances the injected force."""
    ny, tau, G = 20, 1.0, 1e-6
    nu = (tau - 0.5) / 3.0
    solid, rho, u, sig = _poiseuille(ny, tau, G, 6000)
    y = np.arange(ny, dtype=float)
    fl = solid == 0
    ux = u[:, 0]
    yc = (ny - 1) / 2.0
    # exact parabola in the bulk: constant second difference -G/nu
    d2 = ux[3:-1] - 2 * ux[2:-2] + ux[1:-3]
    assert np.allclose(d2, -G / nu, rtol=1e-8)
    # close to the no-slip parabola with walls half way
    W = ny - 2
    exact = G / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
    umax = G * W * W / (8 * nu)
    assert np.max(np.abs(ux[fl] - exact[fl])) < 0.02 * umax
    # stress
    assert np.allclose(sig[fl, 3], -G * (y[fl] - yc), rtol=1e-6, atol=1e-12)
    # normal stresses are O(u G) forcing terms, negligible beside the shear
    smax = np.max(np.abs(sig[fl, 3]))
    assert np.allclose(sig[fl][:, [0, 1, 2, 4, 5]], 0.0, atol=1e-4 * smax)
    assert np.allclose(u[:, 1:], 0.0, atol=1e-13) and np.all(u[~fl] == 0.0)


def test_walls_conserve_mass():
    rng = np.random.default_rng(3)
    dims = (5, 7, 4)
    N = 140
    solid = np.zeros((4, 7, 5), dtype=np.uint8)
    solid[:, 0, :] = solid[:, 6, :] = 1
    solid[1, 3, 2] = 1  # an obstacle
    solid = solid.reshape(-1)
    c, w = orc.lattice()
    f = np.ascontiguousarray(w[:, None] * (1.0 + 0.05 * rng.standard_normal((19, N))))
    f[:, solid == 1] = 0.0
    m0 = f.sum()
    for _ in range(15):
        orc.lb_pass(dims, solid, f, None, np.full(N, 0.8))
    assert abs(f.sum() - m0) < 1e-12 * m0


def _kolmogorov(L, A, steps):
    from paper_1107_4889_gb300 import workloads as wl
    geom = wl.periodic_box(1, L, 1, body_force_wave=(A, 0.0, 0.0))
    o = orc.Oracle(geom, None, wl.params())
    o.step(steps)
    _, u, _ = o.fields()
    b = o.budget()
    o.close()
    return u, b


def test_kolmogorov_steady_state_and_work_rate():
    """Force A sin(k y) x in a periodic box (k = 2 pi / L): the steady
    Navier-Stokes flow is u_x = A / (nu k^2) sin(k y) with nu = (T - 1/2)/3;
    the lattice error of this mode at tau = 1 falls faster than k^2 (1e-4 at
    L = 16, 6e-6 at L = 32).  The work rate of the force, sum_x G(x).u(x),
    is A^2 L / (2 nu k^2) there."""
    nu = (1.0 - 0.5) / 3.0
    A = 1e-6
    errs = []
    for L in (16, 32):
        k = 2 * np.pi / L
        U = A / (nu * k * k)
        u, b = _kolmogorov(L, A, 30 * int(1.0 / (nu * k * k)))
        prof = U * np.sin(k * np.arange(L))
        err = np.abs(u[:, 0] - prof).max() / U
        errs.append(err)
        assert np.abs(u[:, 1:]).max() < 1e-9 * U
        assert abs(b["power"] / (A * A * L / (2 * nu * k * k)) - 1.0) < 2 * err + 1e-6
        assert abs(b["p_fluid"][0]) < 1e-9 * U * L
    assert errs[0] < 3e-4 and errs[1] < errs[0] / 8.0
