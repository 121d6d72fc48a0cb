"""Python driver of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` use this module; the product package never
imports it.  It compiles ``oracle.c`` with gcc (``-ffp-contract=off`` so that no
multiply-add is fused and the cell-pair distance test is bit-reproducible) and
marshals numpy arrays through ctypes.

Inputs are plain dicts / numpy arrays (geometry, cells, params) so the oracle
shares nothing with the CUDA package but the seeded input generators.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_U8 = ctypes.POINTER(ctypes.c_ubyte)


class _Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("periodic", ctypes.c_int * 3),
        ("solid", _U8),
        ("body_force", ctypes.c_double * 3),
        ("tau0", ctypes.c_double), ("delta", ctypes.c_double), ("kappa", ctypes.c_double),
        ("gamma_T", ctypes.c_double), ("gamma_R", ctypes.c_double),
        ("alpha", ctypes.c_double), ("eps0", ctypes.c_double),
        ("xi", ctypes.c_double * 3), ("semi_axes", ctypes.c_double * 3),
        ("mass", ctypes.c_double), ("inertia", ctypes.c_double * 3),
        ("sigma_min_wall", ctypes.c_double), ("wall_radius", ctypes.c_double),
        ("rho_floor", ctypes.c_double),
        ("r_cut", ctypes.c_double), ("r_cut_wall", ctypes.c_double),
        ("ncells", ctypes.c_int),
        ("pos", _D), ("quat", _D), ("vel", _D), ("omega", _D),
        ("storage", ctypes.c_int), ("stochastic", ctypes.c_int),
        ("seed", ctypes.c_ulonglong),
        ("body_force_wave", ctypes.c_double * 3),
        ("node_type", _U8), ("inlet_center", ctypes.c_double * 2), ("inlet_radius", ctypes.c_double),
        ("inlet_umax", ctypes.c_double), ("force_ext", _D), ("torque_ext", _D),
    ]


#: population storage of the reduced-precision variants (orc_round_storage)
STORAGE = {"f64": 0, "f32": 0, "f16": 1, "bf16": 2}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (idempotent)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                   "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.POINTER(_Config)]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
        L.orc_step_count.restype = ctypes.c_long
        L.orc_step_count.argtypes = [ctypes.c_void_p]
        L.orc_clamps.restype = ctypes.c_long
        L.orc_clamps.argtypes = [ctypes.c_void_p]
        L.orc_fields.argtypes = [ctypes.c_void_p, _D, _D, _D]
        L.orc_cells.argtypes = [ctypes.c_void_p, _D]
        L.orc_diag.argtypes = [ctypes.c_void_p, _D]
        L.orc_budget.argtypes = [ctypes.c_void_p, _D]
        L.orc_neighbor_pairs.restype = ctypes.c_long
        L.orc_neighbor_pairs.argtypes = [ctypes.c_void_p, _I, ctypes.c_long]
        L.orc_set_sampled_fields.argtypes = [ctypes.c_void_p, _D, _D]
        L.orc_fluid_nodes.restype = ctypes.c_long
        L.orc_fluid_nodes.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_long), ctypes.c_long]
        L.orc_peskin.restype = ctypes.c_double
        L.orc_peskin.argtypes = [ctypes.c_double]
        L.orc_quat_to_Q.argtypes = [_D, _D]
        L.orc_shape_field.restype = ctypes.c_double
        L.orc_shape_field.argtypes = [ctypes.c_int] * 3 + [_U8, _D, _D, _D, _D, _D, _D]
        L.orc_sample_cell.argtypes = [ctypes.c_int] * 3 + [_U8, _D, _D, _D, _D, _D,
                                                           ctypes.c_double, _D, _D, _D]
        L.orc_spread_cell.argtypes = [ctypes.c_int] * 3 + [_U8, _D, _D, _D, ctypes.c_double,
                                                           _D, _D, _D, _D]
        L.orc_gb_pair.restype = ctypes.c_int
        L.orc_gb_pair.argtypes = [_D, _D, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  _D, _D, _D, _D]
        L.orc_rigid_close.argtypes = [_D, _D, _D, _D, ctypes.c_double, _D, ctypes.c_double,
                                      ctypes.c_double]
        L.orc_rigid_open.argtypes = [_D, _D, _D, _D, _D, _D, ctypes.c_double, _D,
                                     ctypes.c_double, ctypes.c_double]
        L.orc_lb_pass.argtypes = [ctypes.c_int] * 3 + [_U8, _D, _D, _D, _D, _D, _D]
        L.orc_lattice.argtypes = [_I, _D]
        L.orc_round_storage.restype = ctypes.c_double
        L.orc_round_storage.argtypes = [ctypes.c_int, ctypes.c_double]
        L.orc_round_storage_sr.restype = ctypes.c_double
        L.orc_round_storage_sr.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_uint, ctypes.c_int]
        L.orc_philox4x32.argtypes = [ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(ctypes.c_uint),
                                     ctypes.POINTER(ctypes.c_uint)]
        L.orc_storage_bits.restype = ctypes.c_uint
        L.orc_storage_bits.argtypes = [ctypes.c_ulonglong, ctypes.c_long, ctypes.c_long, ctypes.c_int]
        L.orc_storage_scale.restype = ctypes.c_double
        L.orc_storage_scale.argtypes = [ctypes.c_int]
        L.orc_populations.argtypes = [ctypes.c_void_p, _D]
        L.orc_set_populations.argtypes = [ctypes.c_void_p, _D]
        L.orc_wall_shear.restype = ctypes.c_long
        L.orc_wall_shear.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_long), _D, ctypes.c_long]
        _lib = L
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _u8(a):
    if a is None:
        return None
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint8))


def _u8p(a):
    return None if a is None else a.ctypes.data_as(_U8)


# ---------------------------------------------------------------------------
# building blocks
# ---------------------------------------------------------------------------

def lattice():
    c = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    lib().orc_lattice(c.ctypes.data_as(_I), _dp(w))
    return c, w


def round_storage(kind, v):
    """orc_round_storage elementwise: kind 'f16' or 'bf16' (or 'f64')."""
    k = STORAGE[kind]
    v = np.asarray(v, dtype=np.float64)
    return np.array([lib().orc_round_storage(k, float(x)) for x in v.ravel()]).reshape(v.shape)


def round_storage_sr(kind, v, r, bits=6):
    """orc_round_storage_sr elementwise with random integers r (same shape)."""
    k = STORAGE[kind]
    v = np.asarray(v, dtype=np.float64)
    r = np.broadcast_to(np.asarray(r, dtype=np.int64), v.shape)
    return np.array([lib().orc_round_storage_sr(k, float(x), int(ri), int(bits))
                     for x, ri in zip(v.ravel(), r.ravel())]).reshape(v.shape)


def philox4x32(ctr, key):
    c = (ctypes.c_uint * 4)(*[int(x) & 0xffffffff for x in ctr])
    k = (ctypes.c_uint * 2)(*[int(x) & 0xffffffff for x in key])
    o = (ctypes.c_uint * 4)()
    lib().orc_philox4x32(c, k, o)
    return [int(x) for x in o]


def storage_bits(seed, step, n, slot):
    return int(lib().orc_storage_bits(int(seed), int(step), int(n), int(slot)))


def storage_scale(kind):
    return float(lib().orc_storage_scale(STORAGE[kind]))


def peskin(r):
    return float(lib().orc_peskin(float(r)))


def quat_to_Q(q):
    q = _f64(q, (4,))
    Q = np.zeros(9)
    lib().orc_quat_to_Q(_dp(q), _dp(Q))
    return Q.reshape(3, 3)


def shape_field(dims, solid, R, Q, xi):
    """Raw weight w, normalised delta and gradient Ddelta on the full lattice.

    Arrays are node-major with node n = x + nx*(y + ny*z); returned reshaped to
    (nz, ny, nx) and (nz, ny, nx, 3)."""
    nx, ny, nz = dims
    N = nx * ny * nz
    solid = _u8(solid)
    R, Q, xi = _f64(R, (3,)), _f64(Q, (9,)), _f64(xi, (3,))
    w, d, D = np.zeros(N), np.zeros(N), np.zeros(3 * N)
    S = lib().orc_shape_field(nx, ny, nz, _u8p(solid), _dp(R), _dp(Q), _dp(xi), _dp(w), _dp(d), _dp(D))
    return S, w.reshape(nz, ny, nx), d.reshape(nz, ny, nx), D.reshape(nz, ny, nx, 3)


def sample_cell(dims, solid, u, sigma, R, Q, xi, alpha):
    nx, ny, nz = dims
    N = nx * ny * nz
    solid = _u8(solid)
    u = _f64(u, (3 * N,))
    sigma = _f64(sigma if sigma is not None else np.zeros(6 * N), (6 * N,))
    R, Q, xi = _f64(R, (3,)), _f64(Q, (9,)), _f64(xi, (3,))
    ut, wt, TS = np.zeros(3), np.zeros(3), np.zeros(3)
    lib().orc_sample_cell(nx, ny, nz, _u8p(solid), _dp(u), _dp(sigma), _dp(R), _dp(Q), _dp(xi),
                          float(alpha), _dp(ut), _dp(wt), _dp(TS))
    return ut, wt, TS


def spread_cell(dims, solid, R, Q, xi, kappa, J, L):
    nx, ny, nz = dims
    N = nx * ny * nz
    solid = _u8(solid)
    R, Q, xi = _f64(R, (3,)), _f64(Q, (9,)), _f64(xi, (3,))
    J, L = _f64(J, (3,)), _f64(L, (3,))
    G, th = np.zeros(3 * N), np.zeros(N)
    lib().orc_spread_cell(nx, ny, nz, _u8p(solid), _dp(R), _dp(Q), _dp(xi), float(kappa),
                          _dp(J), _dp(L), _dp(G), _dp(th))
    return G.reshape(N, 3), th


def gb_pair(d, Ai, Aj, sigma_min, eps0, rho_floor=-1e300):
    d, Ai, Aj = _f64(d, (3,)), _f64(Ai, (9,)), _f64(Aj, (9,))
    u = np.zeros(1)
    F, ti, tj = np.zeros(3), np.zeros(3), np.zeros(3)
    cl = lib().orc_gb_pair(_dp(d), _dp(Ai), _dp(Aj), float(sigma_min), float(eps0), float(rho_floor),
                           _dp(u), _dp(F), _dp(ti), _dp(tj))
    return float(u[0]), F, ti, tj, int(cl)


def rigid_close(V, Om, Fc, Tc, M, I, gT, gR):
    V, Om = _f64(V, (3,)).copy(), _f64(Om, (3,)).copy()
    Fc, Tc, I = _f64(Fc, (3,)), _f64(Tc, (3,)), _f64(I, (3,))
    lib().orc_rigid_close(_dp(V), _dp(Om), _dp(Fc), _dp(Tc), float(M), _dp(I), float(gT), float(gR))
    return V, Om


def rigid_open(R, Q, V, Om, Fc, Tc, M, I, gT, gR):
    R, Q = _f64(R, (3,)).copy(), _f64(Q, (9,)).copy()
    V, Om = _f64(V, (3,)).copy(), _f64(Om, (3,)).copy()
    Fc, Tc, I = _f64(Fc, (3,)), _f64(Tc, (3,)), _f64(I, (3,))
    lib().orc_rigid_open(_dp(R), _dp(Q), _dp(V), _dp(Om), _dp(Fc), _dp(Tc), float(M), _dp(I),
                         float(gT), float(gR))
    return R, Q.reshape(3, 3), V, Om


def lb_pass(dims, solid, f, G, tau):
    """One streaming + collision pass; f (19, N) is updated in place."""
    nx, ny, nz = dims
    N = nx * ny * nz
    assert f.dtype == np.float64 and f.flags.c_contiguous and f.size == 19 * N
    solid = _u8(solid)
    G = _f64(G, (3 * N,)) if G is not None else None
    tau = _f64(tau, (N,))
    rho, u, sig = np.zeros(N), np.zeros(3 * N), np.zeros(6 * N)
    lib().orc_lb_pass(nx, ny, nz, _u8p(solid), _dp(f), _dp(G), _dp(tau), _dp(rho), _dp(u), _dp(sig))
    return rho, u.reshape(N, 3), sig.reshape(N, 6)


# ---------------------------------------------------------------------------
# coupled solver
# ---------------------------------------------------------------------------

class Oracle:
    """FP64 coupled solver.  ``geometry``: dict(nx, ny, nz, periodic, solid,
    body_force); ``cells``: dict(pos (n,3), quat (n,4), vel, omega);
    ``params``: dict with the keys of orc_config.  ``storage``: population
    storage of the reduced-precision variants ('f64' exact, 'f16', 'bf16';
    'f32' is taken as exact); ``stochastic``: stochastic rounding of the
    16-bit store (else to nearest) keyed by ``seed``."""

    def __init__(self, geometry, cells, params, storage="f64", stochastic=True, seed=0):
        L = lib()
        nx, ny, nz = int(geometry["nx"]), int(geometry["ny"]), int(geometry["nz"])
        self.dims = (nx, ny, nz)
        self.N = nx * ny * nz
        solid = geometry.get("solid")
        self._solid = _u8(solid.reshape(-1)) if solid is not None else None
        n = 0 if cells is None else int(np.asarray(cells["pos"]).shape[0])
        self.n = n
        self._pos = _f64(cells["pos"], (3 * n,)) if n else np.zeros(3)
        self._quat = _f64(cells["quat"], (4 * n,)) if n else np.zeros(4)
        self._vel = _f64(cells.get("vel"), (3 * n,)) if n and cells.get("vel") is not None else None
        self._om = _f64(cells.get("omega"), (3 * n,)) if n and cells.get("omega") is not None else None
        self._fext = _f64(cells.get("force_ext"), (3 * n,)) if n and cells.get("force_ext") is not None else None
        self._text = _f64(cells.get("torque_ext"), (3 * n,)) if n and cells.get("torque_ext") is not None else None
        c = _Config()
        c.nx, c.ny, c.nz = nx, ny, nz
        for a in range(3):
            c.periodic[a] = int(geometry.get("periodic", (1, 1, 1))[a])
            c.body_force[a] = float(geometry.get("body_force", (0.0, 0.0, 0.0))[a])
            c.body_force_wave[a] = float(geometry.get("body_force_wave", (0.0, 0.0, 0.0))[a])
            c.xi[a] = float(params["xi"][a])
            c.semi_axes[a] = float(params["semi_axes"][a])
            c.inertia[a] = float(params["inertia"][a])
        c.solid = _u8p(self._solid)
        for k in ("tau0", "delta", "kappa", "gamma_T", "gamma_R", "eps0", "mass",
                  "sigma_min_wall", "wall_radius", "rho_floor", "r_cut", "r_cut_wall"):
            setattr(c, k, float(params[k]))
        c.alpha = float(params["alpha_tt"])
        c.ncells = n
        c.pos, c.quat = _dp(self._pos), _dp(self._quat)
        c.vel, c.omega = _dp(self._vel), _dp(self._om)
        c.force_ext, c.torque_ext = _dp(self._fext), _dp(self._text)
        nt = geometry.get("node_type")
        self._nt = _u8(np.asarray(nt).reshape(-1)) if nt is not None else None
        c.node_type = _u8p(self._nt)
        ic = geometry.get("inlet_center", (0.0, 0.0))
        c.inlet_center[0], c.inlet_center[1] = float(ic[0]), float(ic[1])
        c.inlet_radius = float(geometry.get("inlet_radius", 1.0))
        c.inlet_umax = float(geometry.get("inlet_umax", 0.0))
        c.storage = STORAGE[storage]
        c.stochastic = 1 if stochastic else 0
        c.seed = int(seed) & 0xffffffffffffffff
        self._cfg = c
        self._h = L.orc_create(ctypes.byref(c))
        if not self._h:
            raise RuntimeError("orc_create failed")

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        lib().orc_step(self._h, int(n))

    @property
    def step_count(self):
        return int(lib().orc_step_count(self._h))

    @property
    def clamps(self):
        return int(lib().orc_clamps(self._h))

    def fields(self):
        rho, u, s = np.zeros(self.N), np.zeros(3 * self.N), np.zeros(6 * self.N)
        lib().orc_fields(self._h, _dp(rho), _dp(u), _dp(s))
        return rho, u.reshape(self.N, 3), s.reshape(self.N, 6)

    def populations(self):
        """Post-collision populations f (19, N) in the oracle's speed order."""
        f = np.zeros(19 * self.N)
        lib().orc_populations(self._h, _dp(f))
        return f.reshape(19, self.N)

    def wall_shear(self):
        """(nodes, tau (n, 3)) of the wall-adjacent fluid nodes (orc_wall_shear)."""
        cap = self.N
        nodes = np.zeros(cap, dtype=np.int64)
        tau = np.zeros(3 * cap)
        n = lib().orc_wall_shear(self._h, nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _dp(tau), cap)
        return nodes[:n].copy(), tau[: 3 * n].reshape(n, 3).copy()

    def set_populations(self, f):
        f = _f64(f, (19 * self.N,))
        lib().orc_set_populations(self._h, _dp(f))

    def set_sampled_fields(self, u=None, sigma=None):
        u = _f64(u, (3 * self.N,)) if u is not None else None
        s = _f64(sigma, (6 * self.N,)) if sigma is not None else None
        lib().orc_set_sampled_fields(self._h, _dp(u), _dp(s))

    def cells(self):
        out = np.zeros(18 * max(self.n, 1))
        lib().orc_cells(self._h, _dp(out))
        out = out[: 18 * self.n].reshape(self.n, 18)
        return dict(pos=out[:, 0:3], Q=out[:, 3:12].reshape(self.n, 3, 3),
                    vel=out[:, 12:15], omega=out[:, 15:18])

    def diag(self):
        out = np.zeros(21 * max(self.n, 1))
        lib().orc_diag(self._h, _dp(out))
        out = out[: 21 * self.n].reshape(self.n, 21)
        return dict(F_mech=out[:, 0:3], tau_mech=out[:, 3:6], u_s=out[:, 6:9], omega_s=out[:, 9:12],
                    T_S=out[:, 12:15], J=out[:, 15:18], L=out[:, 18:21])

    def budget(self):
        out = np.zeros(8)
        lib().orc_budget(self._h, _dp(out))
        return dict(mass=out[0], p_fluid=out[1:4].copy(), p_cells=out[4:7].copy(), power=out[7])

    def fluid_nodes(self):
        """Lattice indices of the fluid nodes in canonical order (orc_fluid_nodes)."""
        out = np.zeros(self.N, dtype=np.int64)
        n = lib().orc_fluid_nodes(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), self.N)
        return out[:n].copy()

    def neighbor_pairs(self):
        cap = max(16, self.n * 64)
        pairs = np.zeros(2 * cap, dtype=np.int32)
        npairs = lib().orc_neighbor_pairs(self._h, pairs.ctypes.data_as(_I), cap)
        if npairs > cap:
            raise RuntimeError("pair buffer too small")
        return pairs[: 2 * npairs].reshape(npairs, 2)
