"""Thin Python binding of the C ABI in include/rbc.h (ctypes).

Argument marshalling only: every step of the coupled time step runs in the
CUDA kernels of ``lib/librbc.so``.  PyTorch supplies the device workspace
(one uint8 tensor from its caching allocator) and the CUDA stream.  There is
no CPU fallback: if the library is missing or no GPU is present, the calls
raise.

The functions carry the C names (``rbc_init``, ``rbc_step``, ``rbc_fields``,
``rbc_stats`` ...); :class:`Solver` bundles them with the workspace it owns.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "librbc.so")

RBC_OK, RBC_EINVAL, RBC_ENOMEM, RBC_ECUDA, RBC_EUNSTABLE, RBC_ETIMEOUT = 0, -1, -2, -3, -4, -5
_NAMES = {RBC_EINVAL: "EINVAL", RBC_ENOMEM: "ENOMEM", RBC_ECUDA: "ECUDA",
          RBC_EUNSTABLE: "EUNSTABLE", RBC_ETIMEOUT: "ETIMEOUT"}

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U8 = ctypes.POINTER(ctypes.c_uint8)


class rbc_geometry(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("periodic", ctypes.c_int * 3), ("solid", _U8), ("body_force", ctypes.c_double * 3),
                ("body_force_wave", ctypes.c_double * 3), ("node_type", _U8),
                ("inlet_center", ctypes.c_double * 2), ("inlet_radius", ctypes.c_double),
                ("inlet_umax", ctypes.c_double)]


class rbc_cells(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("pos", _D), ("quat", _D), ("vel", _D), ("omega_body", _D),
                ("force_ext", _D), ("torque_ext", _D)]


class rbc_params(ctypes.Structure):
    _fields_ = [("tau0", ctypes.c_double), ("delta", ctypes.c_double), ("kappa", ctypes.c_double),
                ("gamma_T", ctypes.c_double), ("gamma_R", ctypes.c_double),
                ("alpha_tt", ctypes.c_double), ("eps0", ctypes.c_double),
                ("xi", ctypes.c_double * 3), ("semi_axes", ctypes.c_double * 3),
                ("mass", ctypes.c_double), ("inertia", ctypes.c_double * 3),
                ("sigma_min_wall", ctypes.c_double), ("wall_radius", ctypes.c_double),
                ("rho_floor", ctypes.c_double), ("r_cut", ctypes.c_double),
                ("r_cut_wall", ctypes.c_double), ("mach_max", ctypes.c_double),
                ("bin_capacity", ctypes.c_int), ("max_neighbors", ctypes.c_int),
                ("precision", ctypes.c_int), ("rounding", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("node_list", ctypes.c_int), ("layout", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


#: rbc_params.precision / rounding values (include/rbc.h)
PRECISION = {"f32": 0, "f16": 1, "bf16": 2}
ROUNDING = {"stochastic": 0, "nearest": 1}
LAYOUT = {"auto": 0, "dense": 1, "compact": 2}


class rbc_stats_t(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("mass", ctypes.c_double),
                ("p_fluid", ctypes.c_double * 3), ("p_cells", ctypes.c_double * 3),
                ("max_u", ctypes.c_double), ("gb_clamps", ctypes.c_int64),
                ("unstable", ctypes.c_int32), ("overflow", ctypes.c_int32), ("power", ctypes.c_double)]


class rbc_request(ctypes.Structure):
    _fields_ = [("geom", rbc_geometry), ("cells", rbc_cells), ("params", rbc_params),
                ("steps", ctypes.c_int64), ("average_from", ctypes.c_int64), ("tag", ctypes.c_uint64),
                ("out_rho", _D), ("out_u", _D), ("out_cells", _D), ("out_diag", _D)]


class rbc_result(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("steps", ctypes.c_int64), ("samples", ctypes.c_int64), ("mean_power", ctypes.c_double),
                ("mean_p_fluid", ctypes.c_double * 3), ("max_u", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("workspace_bytes", ctypes.c_uint64)]


class rbc_tune_report(ctypes.Structure):
    _fields_ = [("stages", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("ms_per_step", ctypes.c_double),
                ("default_ms_per_step", ctypes.c_double), ("trials", ctypes.c_int),
                ("lattice_first", ctypes.c_int), ("wt_blocks_per_sm", ctypes.c_int),
                ("gb_blocks_per_sm", ctypes.c_int), ("bin_scale", ctypes.c_double), ("split_spread", ctypes.c_int)]


#: symbols include/rbc.h declares
EXPORTS = ["rbc_default_params", "rbc_workspace_size", "rbc_init", "rbc_step", "rbc_fields",
           "rbc_stats", "rbc_cell_diag", "rbc_neighbors", "rbc_set_timing", "rbc_kernel_times",
           "rbc_autotune", "rbc_set_schedule", "rbc_wss_accumulate", "rbc_wss", "rbc_launches_per_step", "rbc_layout", "rbc_fluid_nodes",
           "rbc_profile_accumulate", "rbc_profile", "rbc_set_wait_limit",
           "rbc_checkpoint_size", "rbc_save", "rbc_load",
           "rbc_neighbors_noalloc", "rbc_server_create", "rbc_server_submit",
           "rbc_server_poll", "rbc_server_results", "rbc_server_clock", "rbc_server_free", "rbc_free",
           "rbc_last_error"]

_lib = None


class RbcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    """Load librbc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_1107_4889_gb300.build` (nvcc, sm_103a)")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    L.rbc_default_params.argtypes = [P(rbc_params)]
    L.rbc_default_params.restype = None
    L.rbc_workspace_size.argtypes = [P(rbc_geometry), P(rbc_cells), P(rbc_params), P(ctypes.c_size_t)]
    L.rbc_init.argtypes = [P(rbc_geometry), P(rbc_cells), P(rbc_params), ctypes.c_void_p, ctypes.c_size_t,
                           P(ctypes.c_void_p)]
    L.rbc_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    L.rbc_fields.argtypes = [ctypes.c_void_p, _D, _D, _D]
    L.rbc_stats.argtypes = [ctypes.c_void_p, P(rbc_stats_t)]
    L.rbc_cell_diag.argtypes = [ctypes.c_void_p, _D]
    L.rbc_neighbors.argtypes = [ctypes.c_void_p, _I, _I, ctypes.c_int]
    L.rbc_set_timing.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.rbc_kernel_times.argtypes = [ctypes.c_void_p, _D, _I64]
    L.rbc_launches_per_step.argtypes = [ctypes.c_void_p]
    L.rbc_checkpoint_size.argtypes = [ctypes.c_void_p, P(ctypes.c_size_t)]
    L.rbc_save.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
    L.rbc_load.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
    for name in ("rbc_checkpoint_size", "rbc_save", "rbc_load"):
        getattr(L, name).restype = ctypes.c_int
    L.rbc_set_wait_limit.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]
    L.rbc_set_wait_limit.restype = ctypes.c_int
    L.rbc_profile_accumulate.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.rbc_profile_accumulate.restype = ctypes.c_int
    L.rbc_profile.argtypes = [ctypes.c_void_p, _D, ctypes.c_int, _I, _I64]
    L.rbc_profile.restype = ctypes.c_int
    L.rbc_layout.argtypes = [ctypes.c_void_p, _I, _I64, _I64]
    L.rbc_layout.restype = ctypes.c_int
    L.rbc_fluid_nodes.argtypes = [ctypes.c_void_p, _I64, ctypes.c_int64, _I64]
    L.rbc_fluid_nodes.restype = ctypes.c_int
    L.rbc_autotune.argtypes = [ctypes.c_void_p, ctypes.c_int, P(rbc_tune_report)]
    L.rbc_set_schedule.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    L.rbc_set_schedule.restype = ctypes.c_int
    L.rbc_autotune.restype = ctypes.c_int
    L.rbc_wss_accumulate.argtypes = [ctypes.c_void_p]
    L.rbc_wss_accumulate.restype = ctypes.c_int
    L.rbc_wss.argtypes = [ctypes.c_void_p, _I64, _D, ctypes.c_int64, _I64, _I64]
    L.rbc_wss.restype = ctypes.c_int
    L.rbc_neighbors_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        _I, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_void_p]
    L.rbc_neighbors_noalloc.restype = ctypes.c_int
    L.rbc_server_create.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                    P(ctypes.c_void_p)]
    L.rbc_server_submit.argtypes = [ctypes.c_void_p, P(rbc_request)]
    L.rbc_server_poll.argtypes = [ctypes.c_void_p, _I, _I]
    L.rbc_server_results.argtypes = [ctypes.c_void_p, P(rbc_result), ctypes.c_int, _I]
    L.rbc_server_clock.argtypes = [ctypes.c_void_p]
    L.rbc_server_clock.restype = ctypes.c_double
    L.rbc_server_free.argtypes = [ctypes.c_void_p]
    L.rbc_server_free.restype = None
    for name in ("rbc_server_create", "rbc_server_submit", "rbc_server_poll", "rbc_server_results"):
        getattr(L, name).restype = ctypes.c_int
    L.rbc_free.argtypes = [ctypes.c_void_p]
    L.rbc_free.restype = None
    L.rbc_last_error.argtypes = [ctypes.c_void_p]
    L.rbc_last_error.restype = ctypes.c_char_p
    for name in ("rbc_workspace_size", "rbc_init", "rbc_step", "rbc_fields", "rbc_stats", "rbc_cell_diag",
                 "rbc_neighbors", "rbc_set_timing", "rbc_kernel_times", "rbc_launches_per_step"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(code, handle=None):
    if code != RBC_OK:
        msg = load().rbc_last_error(handle)
        raise RbcError(code, msg.decode() if msg else "")


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


class _Inputs:
    """Keeps the numpy buffers the ctypes structs point into alive."""

    def __init__(self, geometry, cells, params, stream):
        nx, ny, nz = int(geometry["nx"]), int(geometry["ny"]), int(geometry["nz"])
        self.N = nx * ny * nz
        g = rbc_geometry()
        g.nx, g.ny, g.nz = nx, ny, nz
        per = geometry.get("periodic", (1, 1, 1))
        bf = geometry.get("body_force", (0.0, 0.0, 0.0))
        bw = geometry.get("body_force_wave", (0.0, 0.0, 0.0))
        for a in range(3):
            g.periodic[a] = int(per[a])
            g.body_force[a] = float(bf[a])
            g.body_force_wave[a] = float(bw[a])
        solid = geometry.get("solid")
        self.solid = None if solid is None else np.ascontiguousarray(np.asarray(solid, np.uint8).reshape(-1))
        g.solid = None if self.solid is None else self.solid.ctypes.data_as(_U8)
        nt = geometry.get("node_type")
        self.node_type = None if nt is None else np.ascontiguousarray(np.asarray(nt, np.uint8).reshape(-1))
        g.node_type = None if self.node_type is None else self.node_type.ctypes.data_as(_U8)
        ic = geometry.get("inlet_center", (0.0, 0.0))
        g.inlet_center[0], g.inlet_center[1] = float(ic[0]), float(ic[1])
        g.inlet_radius = float(geometry.get("inlet_radius", 1.0))
        g.inlet_umax = float(geometry.get("inlet_umax", 0.0))
        self.geom = g
        c = rbc_cells()
        n = 0 if cells is None else int(np.asarray(cells["pos"]).shape[0])
        self.n = n
        c.n = n
        if n:
            self.pos = np.ascontiguousarray(np.asarray(cells["pos"], np.float64).reshape(n, 3))
            self.quat = np.ascontiguousarray(np.asarray(cells["quat"], np.float64).reshape(n, 4))
            v, w = cells.get("vel"), cells.get("omega")
            self.vel = None if v is None else np.ascontiguousarray(np.asarray(v, np.float64).reshape(n, 3))
            self.om = None if w is None else np.ascontiguousarray(np.asarray(w, np.float64).reshape(n, 3))
            c.pos, c.quat, c.vel, c.omega_body = _dp(self.pos), _dp(self.quat), _dp(self.vel), _dp(self.om)
            fe, te = cells.get("force_ext"), cells.get("torque_ext")
            self.fext = None if fe is None else np.ascontiguousarray(np.asarray(fe, np.float64).reshape(n, 3))
            self.text = None if te is None else np.ascontiguousarray(np.asarray(te, np.float64).reshape(n, 3))
            c.force_ext, c.torque_ext = _dp(self.fext), _dp(self.text)
        self.cells = c
        p = rbc_params()
        load().rbc_default_params(ctypes.byref(p))
        for k, v in (params or {}).items():
            if k in ("xi", "semi_axes", "inertia"):
                arr = getattr(p, k)
                for a in range(3):
                    arr[a] = float(v[a])
            elif k in ("bin_capacity", "max_neighbors", "node_list"):
                setattr(p, k, int(v))
            elif k == "layout":
                p.layout = LAYOUT[v] if isinstance(v, str) else int(v)
            elif k == "precision":
                p.precision = PRECISION[v] if isinstance(v, str) else int(v)
            elif k == "rounding":
                p.rounding = ROUNDING[v] if isinstance(v, str) else int(v)
            elif k == "seed":
                p.seed = int(v) & 0xffffffffffffffff
            elif k == "stream":
                continue
            else:
                setattr(p, k, float(v))
        p.stream = stream
        self.params = p


def rbc_default_params():
    p = rbc_params()
    load().rbc_default_params(ctypes.byref(p))
    return p


def rbc_workspace_size(geometry, cells, params) -> int:
    ins = _Inputs(geometry, cells, params, None)
    nb = ctypes.c_size_t(0)
    _check(load().rbc_workspace_size(ctypes.byref(ins.geom), ctypes.byref(ins.cells), ctypes.byref(ins.params),
                                     ctypes.byref(nb)))
    return int(nb.value)


def rbc_init(geometry, cells, params, workspace_ptr: int, workspace_bytes: int, stream: int | None):
    ins = _Inputs(geometry, cells, params, stream)
    h = ctypes.c_void_p()
    _check(load().rbc_init(ctypes.byref(ins.geom), ctypes.byref(ins.cells), ctypes.byref(ins.params),
                           ctypes.c_void_p(workspace_ptr), ctypes.c_size_t(workspace_bytes), ctypes.byref(h)))
    return h


def rbc_step(h, n: int = 1):
    _check(load().rbc_step(h, int(n)), h)


def rbc_fields(h, N: int, n: int, want_rho=True, want_u=True, want_cells=True):
    rho = np.zeros(N) if want_rho else None
    u = np.zeros(3 * N) if want_u else None
    cs = np.zeros(13 * max(n, 1)) if want_cells else None
    _check(load().rbc_fields(h, _dp(rho), _dp(u), _dp(cs)), h)
    out = {}
    if want_rho:
        out["rho"] = rho
    if want_u:
        out["u"] = u.reshape(N, 3)
    if want_cells:
        cs = cs[: 13 * n].reshape(n, 13)
        out.update(pos=cs[:, 0:3], quat=cs[:, 3:7], vel=cs[:, 7:10], omega=cs[:, 10:13])
    return out


def rbc_stats(h):
    s = rbc_stats_t()
    code = load().rbc_stats(h, ctypes.byref(s))
    out = dict(step=int(s.step), mass=s.mass, p_fluid=np.array(s.p_fluid[:]), p_cells=np.array(s.p_cells[:]),
               max_u=s.max_u, gb_clamps=int(s.gb_clamps), unstable=int(s.unstable), overflow=int(s.overflow),
               power=s.power)
    _check(code, h)
    return out


def rbc_cell_diag(h, n: int):
    out = np.zeros(21 * max(n, 1))
    _check(load().rbc_cell_diag(h, _dp(out)), h)
    out = out[: 21 * n].reshape(n, 21)
    return dict(F_mech=out[:, 0:3], tau_mech=out[:, 3:6], u_s=out[:, 6:9], omega_s=out[:, 9:12],
                T_S=out[:, 12:15], J=out[:, 15:18], L=out[:, 18:21])


def rbc_neighbors(h, n: int, max_per_cell: int = 128):
    counts = np.zeros(max(n, 1), dtype=np.int32)
    lists = np.zeros(max(n, 1) * max_per_cell, dtype=np.int32)
    _check(load().rbc_neighbors(h, counts.ctypes.data_as(_I), lists.ctypes.data_as(_I), max_per_cell), h)
    lists = lists.reshape(-1, max_per_cell)
    return [lists[i, : counts[i]].copy() for i in range(n)]


def rbc_set_timing(h, capacity: int):
    _check(load().rbc_set_timing(h, int(capacity)), h)


def rbc_kernel_times(h):
    ms = np.zeros(2)
    cnt = np.zeros(2, dtype=np.int64)
    _check(load().rbc_kernel_times(h, _dp(ms), cnt.ctypes.data_as(_I64)), h)
    return ms, cnt


def rbc_autotune(h, steps_per_trial: int = 20):
    r = rbc_tune_report()
    _check(load().rbc_autotune(h, int(steps_per_trial), ctypes.byref(r)), h)
    return dict(stages=r.stages, ctas_per_sm=r.ctas_per_sm, ms_per_step=r.ms_per_step,
                default_ms_per_step=r.default_ms_per_step, trials=r.trials,
                lattice_first=bool(r.lattice_first), wt_blocks_per_sm=r.wt_blocks_per_sm,
                gb_blocks_per_sm=r.gb_blocks_per_sm, bin_scale=r.bin_scale, split_spread=bool(r.split_spread))


def rbc_set_schedule(h, split_spread: bool, lattice_first: bool):
    _check(load().rbc_set_schedule(h, int(bool(split_spread)), int(bool(lattice_first))), h)


def rbc_wss_accumulate(h):
    _check(load().rbc_wss_accumulate(h), h)


def rbc_wss(h, max_nodes: int):
    node = np.zeros(max(max_nodes, 1), dtype=np.int64)
    tau = np.zeros(3 * max(max_nodes, 1))
    n, samples = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load().rbc_wss(h, node.ctypes.data_as(_I64), _dp(tau), int(max_nodes), ctypes.byref(n),
                          ctypes.byref(samples)), h)
    k = min(n.value, max_nodes)
    return node[:k].copy(), tau[: 3 * k].reshape(k, 3).copy(), int(samples.value)


def rbc_launches_per_step(h) -> int:
    return int(load().rbc_launches_per_step(h))


def rbc_save(h) -> bytes:
    """The handle's checkpoint (rbc_checkpoint_size bytes) as a bytes object."""
    nb = ctypes.c_size_t(0)
    _check(load().rbc_checkpoint_size(h, ctypes.byref(nb)), h)
    buf = ctypes.create_string_buffer(nb.value)
    _check(load().rbc_save(h, buf, nb.value), h)
    return buf.raw


def rbc_load(h, data: bytes):
    buf = ctypes.create_string_buffer(data, len(data))
    _check(load().rbc_load(h, buf, len(data)), h)


def rbc_set_wait_limit(h, cycles: int, starve_batch: int = -1):
    _check(load().rbc_set_wait_limit(h, int(cycles), int(starve_batch)), h)


def rbc_profile_accumulate(h, axis: int = 1):
    _check(load().rbc_profile_accumulate(h, int(axis)), h)


def rbc_profile(h, nbins: int):
    counts = np.zeros(max(nbins, 1))
    axis, samples = ctypes.c_int(-1), ctypes.c_int64(0)
    _check(load().rbc_profile(h, _dp(counts), int(nbins), ctypes.byref(axis), ctypes.byref(samples)), h)
    return counts[:nbins], int(axis.value), int(samples.value)


def rbc_layout(h):
    c, e, f = ctypes.c_int(0), ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load().rbc_layout(h, ctypes.byref(c), ctypes.byref(e), ctypes.byref(f)), h)
    return dict(compact=bool(c.value), entries=int(e.value), fluid=int(f.value))


def rbc_fluid_nodes(h, max_nodes: int):
    nodes = np.zeros(max(max_nodes, 1), dtype=np.int64)
    cnt = ctypes.c_int64(0)
    _check(load().rbc_fluid_nodes(h, nodes.ctypes.data_as(_I64), int(max_nodes), ctypes.byref(cnt)), h)
    return nodes[: min(cnt.value, max_nodes)].copy()


def rbc_neighbors_noalloc(pos_ptr: int, n: int, dims, periodic, r_cut: float, counts_ptr: int, lists_ptr: int,
                          max_per_cell: int, stream: int | None):
    """Candidate-partner lists without device allocation (device pointers in
    and out; see include/rbc.h).  For callers that cannot allocate device
    memory: the scratch is a static device array inside the library."""
    per = (ctypes.c_int * 3)(*[int(p) for p in periodic])
    _check(load().rbc_neighbors_noalloc(ctypes.c_void_p(pos_ptr), int(n), int(dims[0]), int(dims[1]), int(dims[2]),
                                        per, float(r_cut), ctypes.c_void_p(counts_ptr), ctypes.c_void_p(lists_ptr),
                                        int(max_per_cell), ctypes.c_void_p(stream)))


def rbc_free(h):
    if h:
        load().rbc_free(h)


class Solver:
    """One coupled LB + RBC solve on the current CUDA device.

    ``geometry``: dict(nx, ny, nz, periodic, solid, body_force); ``cells``:
    dict(pos, quat, vel, omega) or None; ``params``: dict of rbc_params
    fields (missing keys take the paper's values)."""

    def __init__(self, geometry, cells, params=None, device=None, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the RBC solver needs a CUDA GPU")
        load()
        self.device = torch.device("cuda" if device is None else device)
        self.dims = (int(geometry["nx"]), int(geometry["ny"]), int(geometry["nz"]))
        self.N = self.dims[0] * self.dims[1] * self.dims[2]
        self.n = 0 if cells is None else int(np.asarray(cells["pos"]).shape[0])
        with torch.cuda.device(self.device):
            # a stream of its own: the legacy default stream cannot be
            # captured into CUDA graphs, and events recorded on self.stream
            # then time exactly the solver's work
            self.stream = torch.cuda.Stream(self.device) if stream is None else stream
            self.workspace_bytes = rbc_workspace_size(geometry, cells, params)
            self.workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
            self.handle = rbc_init(geometry, cells, params, self.workspace.data_ptr(), self.workspace_bytes,
                                   self.stream.cuda_stream)

    def step(self, n=1):
        rbc_step(self.handle, n)

    def fields(self, rho=True, u=True, cells=True):
        return rbc_fields(self.handle, self.N, self.n, rho, u, cells)

    def stats(self):
        return rbc_stats(self.handle)

    def cell_diag(self):
        return rbc_cell_diag(self.handle, self.n)

    def neighbors(self, max_per_cell=128):
        return rbc_neighbors(self.handle, self.n, max_per_cell)

    def set_timing(self, capacity):
        rbc_set_timing(self.handle, capacity)

    def kernel_times(self):
        return rbc_kernel_times(self.handle)

    def launches_per_step(self):
        return rbc_launches_per_step(self.handle)

    def autotune(self, steps_per_trial=20):
        return rbc_autotune(self.handle, steps_per_trial)

    def set_schedule(self, split_spread=False, lattice_first=False):
        rbc_set_schedule(self.handle, split_spread, lattice_first)

    def layout(self):
        return rbc_layout(self.handle)

    def save(self) -> bytes:
        return rbc_save(self.handle)

    def load(self, data: bytes):
        rbc_load(self.handle, data)

    def set_wait_limit(self, cycles, starve_batch=-1):
        rbc_set_wait_limit(self.handle, cycles, starve_batch)

    def profile_accumulate(self, axis=1):
        rbc_profile_accumulate(self.handle, axis)

    def profile(self):
        """(time-averaged cell-centre count per 1-lu bin, axis, samples)."""
        counts, axis, samples = rbc_profile(self.handle, max(self.dims))
        n = self.dims[axis] if axis >= 0 else 0
        return (counts[:n] / max(samples, 1)), axis, samples

    def fluid_nodes(self):
        """Lattice indices of the fluid nodes in the library's storage order."""
        return rbc_fluid_nodes(self.handle, self.N)

    def wss_accumulate(self):
        rbc_wss_accumulate(self.handle)

    def wss(self):
        """(nodes, time-averaged wall shear stress vectors (n, 3), samples)."""
        return rbc_wss(self.handle, self.N)

    def close(self):
        if getattr(self, "handle", None):
            rbc_free(self.handle)
            self.handle = None
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# request server
# ---------------------------------------------------------------------------

def rbc_server_create(arena_ptr: int, arena_bytes: int, max_active: int, tick_steps: int):
    h = ctypes.c_void_p()
    _check(load().rbc_server_create(ctypes.c_void_p(arena_ptr), ctypes.c_size_t(arena_bytes), int(max_active),
                                    int(tick_steps), ctypes.byref(h)))
    return h


def rbc_server_submit(srv, geometry, cells, params, steps: int, average_from: int = 0, tag: int = 0, out=None):
    """Queue a request.  ``out``: optional dict of float64 numpy buffers
    (rho (N,), u (N, 3), cells (n, 13), diag (n, 21)) the server fills with
    the final state; the caller keeps them alive until the result is out."""
    ins = _Inputs(geometry, cells, params, None)
    r = rbc_request()
    r.geom, r.cells, r.params = ins.geom, ins.cells, ins.params
    r.steps, r.average_from, r.tag = int(steps), int(average_from), int(tag)
    if out:
        r.out_rho, r.out_u = _dp(out.get("rho")), _dp(out.get("u"))
        r.out_cells, r.out_diag = _dp(out.get("cells")), _dp(out.get("diag"))
    _check(load().rbc_server_submit(srv, ctypes.byref(r)))  # inputs are copied by the server


def rbc_server_poll(srv):
    a, q = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().rbc_server_poll(srv, ctypes.byref(a), ctypes.byref(q)))
    return a.value, q.value


def rbc_server_results(srv, max_results: int = 256):
    buf = (rbc_result * max_results)()
    n = ctypes.c_int(0)
    _check(load().rbc_server_results(srv, buf, max_results, ctypes.byref(n)))
    out = []
    for k in range(n.value):
        r = buf[k]
        out.append(dict(tag=int(r.tag), status=int(r.status), steps=int(r.steps), samples=int(r.samples),
                        mean_power=r.mean_power, mean_p_fluid=np.array(r.mean_p_fluid[:]), max_u=r.max_u,
                        t_submit=r.t_submit, t_admit=r.t_admit, t_done=r.t_done,
                        workspace_bytes=int(r.workspace_bytes)))
    return out


def rbc_server_clock(srv) -> float:
    return float(load().rbc_server_clock(srv))


def rbc_server_free(srv):
    if srv:
        load().rbc_server_free(srv)


class Server:
    """Continuous-batching request server on the current CUDA device.

    The arena (``arena_bytes`` of device memory from PyTorch's allocator) is
    lent to the server, which carves each admitted solve's workspace from it.
    ``submit`` queues a solve; ``poll`` advances the server one round (never
    blocks); ``results`` drains finished solves."""

    def __init__(self, arena_bytes, max_active=32, tick_steps=100, device=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the RBC server needs a CUDA GPU")
        load()
        self.device = torch.device("cuda" if device is None else device)
        self._out = {}  # tag -> result buffers the server fills when the solve finishes
        with torch.cuda.device(self.device):
            self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=self.device)
            self.handle = rbc_server_create(self.arena.data_ptr(), int(arena_bytes), max_active, tick_steps)

    def submit(self, geometry, cells, params, steps, average_from=0, tag=0, fields=False):
        """Queue a solve.  fields=True: its result carries the final rho,
        u, cell state and per-cell diagnostics (rbc_fields /
        rbc_cell_diag layout), read back when it finishes."""
        out = None
        if fields:
            N = int(geometry["nx"]) * int(geometry["ny"]) * int(geometry["nz"])
            n = 0 if cells is None else int(np.asarray(cells["pos"]).shape[0])
            out = dict(rho=np.zeros(N), u=np.zeros((N, 3)), cells=np.zeros((max(n, 1), 13)),
                       diag=np.zeros((max(n, 1), 21)), n=n)
            self._out[int(tag)] = out
        rbc_server_submit(self.handle, geometry, cells, params, steps, average_from, tag, out)

    def poll(self):
        return rbc_server_poll(self.handle)

    def results(self, max_results=256):
        res = rbc_server_results(self.handle, max_results)
        for r in res:
            out = self._out.pop(r["tag"], None)
            if out is None:
                continue
            n = out["n"]
            cs, dg = out["cells"][:n], out["diag"][:n]
            r["fields"] = dict(rho=out["rho"], u=out["u"], pos=cs[:, 0:3], quat=cs[:, 3:7], vel=cs[:, 7:10],
                               omega=cs[:, 10:13])
            r["diag"] = dict(F_mech=dg[:, 0:3], tau_mech=dg[:, 3:6], u_s=dg[:, 6:9], omega_s=dg[:, 9:12],
                             T_S=dg[:, 12:15], J=dg[:, 15:18], L=dg[:, 18:21])
        return res

    def clock(self):
        return rbc_server_clock(self.handle)

    def drain(self, sleep_s=0.0):
        """Poll until nothing is active or queued; returns all results."""
        import time
        out = []
        while True:
            a, q = self.poll()
            out += self.results()
            if a == 0 and q == 0:
                break
            if sleep_s:
                time.sleep(sleep_s)
        return out + self.results()

    def close(self):
        if getattr(self, "handle", None):
            rbc_server_free(self.handle)
            self.handle = None
        self.arena = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
