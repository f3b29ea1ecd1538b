"""ctypes binding of include/heat.h (argument marshalling only).

Function names match the C ABI. Device arrays are torch CUDA tensors (their
``data_ptr()`` is passed through); host arrays are numpy float64 arrays.
Every non-OK status raises HeatError with the library's message.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libheatgb.so")

HEAT_OK = 0
HEAT_ERR_ARG = 1
HEAT_ERR_NOMEM = 2
HEAT_ERR_CUDA = 3
HEAT_ERR_NOT_CONVERGED = 4
HEAT_ERR_NONFINITE = 5
HEAT_ERR_TIMEOUT = 6
HEAT_ERR_BUSY = 7
HEAT_ERR_BREAKDOWN = 8

HEAT_FP64 = 0
HEAT_FP32_REFINED = 1
HEAT_FP32_PLAIN = 2
PRECISIONS = {"fp64": HEAT_FP64, "fp32_refined": HEAT_FP32_REFINED, "fp32_plain": HEAT_FP32_PLAIN}
HEAT_ELEM_Q1 = 0
HEAT_ELEM_P1 = 1
ELEMENTS = {"q1": HEAT_ELEM_Q1, "p1": HEAT_ELEM_P1}


class HeatError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"heat status {status}: {message}")
        self.status = status


class heat_params(C.Structure):
    _fields_ = [("theta", C.c_double), ("dt", C.c_double), ("rtol", C.c_double),
                ("max_iter", C.c_int), ("resid_period", C.c_int), ("poll_period", C.c_int),
                ("precision", C.c_int), ("inner_rtol", C.c_double), ("max_outer", C.c_int),
                ("inner_max_iter", C.c_int), ("cheb_degree", C.c_int), ("cheb_ratio", C.c_double),
                ("element", C.c_int)]


class heat_bc(C.Structure):
    _fields_ = [("dirichlet_faces", C.c_uint32), ("dirichlet_value", C.c_double * 6),
                ("flux", C.c_double * 6), ("flux_steps", C.c_int)]


class heat_step_stats(C.Structure):
    _fields_ = [("steps", C.c_int), ("status", C.c_int), ("iters", C.c_longlong),
                ("outer", C.c_longlong), ("max_iters_step", C.c_int),
                ("last_rel_residual", C.c_double), ("kernel_launches", C.c_longlong)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class heat_request(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("origin", C.c_double * 3), ("extent", C.c_double * 3),
                ("rho_c", C.c_void_p), ("k", C.c_void_p), ("u0", C.c_void_p),
                ("bc", heat_bc), ("params", heat_params), ("nsteps", C.c_int)]


class heat_corrosion(C.Structure):
    _fields_ = [("z0", C.c_double), ("half_width", C.c_double), ("rho_c_sound", C.c_double),
                ("k_sound", C.c_double), ("rho_c_corr", C.c_double), ("k_corr", C.c_double)]


class heat_mh_config(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("origin", C.c_double * 3), ("extent", C.c_double * 3),
                ("bc", heat_bc), ("params", heat_params), ("nsteps", C.c_int), ("u0", C.c_double),
                ("flux_face", C.c_int), ("flux_q", C.c_void_p), ("geom", heat_corrosion),
                ("obs_face", C.c_int), ("data", C.c_void_p), ("sigma", C.c_double),
                ("depth_max", C.c_double), ("nchains", C.c_int)]


class heat_tuning(C.Structure):
    _fields_ = [("variant", C.c_int * 3), ("seg_nodes", C.c_int * 3), ("pw_quads", C.c_int * 3),
                ("open_w", C.c_int * 3), ("loop", C.c_int * 3)]

    def as_dict(self):
        return {"variant": list(self.variant), "seg_nodes": list(self.seg_nodes), "pw_quads": list(self.pw_quads),
                "open_w": list(self.open_w), "loop": list(self.loop)}


class heat_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("completed", C.c_longlong), ("failed", C.c_longlong),
                ("active", C.c_int), ("pending", C.c_int), ("hbm_in_use", C.c_size_t),
                ("hbm_budget", C.c_size_t), ("kernel_launches", C.c_longlong),
                ("dof_cg_iters", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None

# (name, restype, argtypes); heat_status functions return c_int
_VP = C.c_void_p
_DP = C.POINTER(C.c_double)
_SIGS = [
    ("heat_params_default", None, [C.POINTER(heat_params)]),
    ("heat_create_mesh", C.c_int, [C.c_int, C.c_int, C.c_int, _DP, _DP, C.POINTER(_VP)]),
    ("heat_destroy_mesh", None, [_VP]),
    ("heat_mesh_sizes", C.c_int, [_VP, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    ("heat_sim_create", C.c_int, [_VP, C.POINTER(heat_bc), C.POINTER(heat_params), _VP, C.POINTER(_VP)]),
    ("heat_destroy_sim", None, [_VP]),
    ("heat_set_coeffs", C.c_int, [_VP, _VP, _VP, C.c_int]),
    ("heat_set_params", C.c_int, [_VP, C.POINTER(heat_params)]),
    ("heat_set_state", C.c_int, [_VP, _VP, C.c_int]),
    ("heat_get_state", C.c_int, [_VP, _VP, C.c_int]),
    ("heat_get_history", C.c_int, [_VP, _VP, _VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int]),
    ("heat_set_history", C.c_int, [_VP, _VP, _VP, C.c_int, C.c_int]),
    ("heat_step", C.c_int, [_VP, C.c_int, C.POINTER(heat_step_stats)]),
    ("heat_solve_transient", C.c_int, [_VP, C.c_int, _VP, C.POINTER(heat_step_stats)]),
    ("heat_step_iterations", C.c_int, [_VP, C.c_int, C.POINTER(C.c_int)]),
    ("heat_apply", C.c_int, [_VP, _VP, _VP]),
    ("heat_apply_f32", C.c_int, [_VP, _VP, _VP]),
    ("heat_apply_general", C.c_int, [_VP, C.c_double, C.c_double, _VP, _VP]),
    ("heat_diagonal", C.c_int, [_VP, _VP]),
    ("heat_rhs", C.c_int, [_VP, C.c_int, _VP, _VP]),
    ("heat_flux_vector", C.c_int, [_VP, _VP]),
    ("heat_server_create", C.c_int, [C.c_size_t, C.c_int, _VP, C.POINTER(_VP)]),
    ("heat_submit", C.c_int, [_VP, C.POINTER(heat_request), C.POINTER(C.c_uint64)]),
    ("heat_poll", C.c_int, [_VP, C.c_uint64, C.POINTER(C.c_int)]),
    ("heat_wait", C.c_int, [_VP, C.c_uint64, C.c_double, _VP, C.POINTER(heat_step_stats), _DP]),
    ("heat_server_get_stats", C.c_int, [_VP, C.POINTER(heat_server_stats)]),
    ("heat_destroy_server", None, [_VP]),
    ("heat_batch_create", C.c_int, [C.POINTER(_VP), C.c_int, _VP, C.POINTER(_VP)]),
    ("heat_batch_step", C.c_int, [_VP, C.c_int, C.POINTER(heat_step_stats)]),
    ("heat_destroy_batch", None, [_VP]),
    ("heat_profile_iteration", C.c_int, [_VP, C.c_int, _VP, C.c_size_t, _DP, _DP, _DP, _DP]),
    ("heat_batch_profile_iteration", C.c_int, [_VP, C.c_int, _VP, C.c_size_t, _DP, _DP, _DP, _DP]),
    ("heat_apply_dot_noalloc", C.c_int, [C.c_int, C.c_int, C.c_int, _DP, C.c_double, C.c_double, C.c_uint32,
                                         _VP, _VP, _VP, _VP, _VP]),
    ("heat_tuning_num_variants", C.c_int, []),
    ("heat_tuning_variant", C.c_int, [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                      C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("heat_tuning_get", C.c_int, [C.POINTER(heat_tuning)]),
    ("heat_tuning_set", C.c_int, [C.POINTER(heat_tuning)]),
    ("heat_autotune", C.c_int, [_VP, C.c_int, C.POINTER(heat_tuning), _DP]),
    ("heat_batch_autotune", C.c_int, [_VP, C.c_int, C.POINTER(heat_tuning), _DP]),
    ("heat_get_coeffs", C.c_int, [_VP, _VP, _VP, C.c_int]),
    ("heat_cheb_interval", C.c_int, [_VP, _DP, _DP]),
    ("heat_set_face_flux", C.c_int, [_VP, C.c_int, _VP, C.c_int]),
    ("heat_set_coeffs_corrosion", C.c_int, [_VP, C.POINTER(heat_corrosion), C.c_double]),
    ("heat_face_loglik", C.c_int, [_VP, C.c_int, _VP, C.c_double, _VP]),
    ("heat_mh_create", C.c_int, [C.POINTER(heat_mh_config), _VP, C.POINTER(_VP)]),
    ("heat_mh_destroy", None, [_VP]),
    ("heat_mh_loglik", C.c_int, [_VP, _VP, _VP]),
    ("heat_mh_run", C.c_int, [_VP, C.c_int, C.c_double, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("heat_mh_stats", C.c_int, [_VP, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    ("heat_slab_plan", C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_int)]),
    ("heat_slab_create", C.c_int, [_VP, C.POINTER(heat_bc), C.POINTER(heat_params), C.c_int, C.c_int, _VP,
                                   C.POINTER(_VP)]),
    ("heat_slab_set_coeffs", C.c_int, [_VP, _VP, _VP]),
    ("heat_slab_set_state", C.c_int, [_VP, _VP]),
    ("heat_slab_get_state", C.c_int, [_VP, _VP]),
    ("heat_slab_step", C.c_int, [_VP, C.c_int, C.POINTER(heat_step_stats)]),
    ("heat_slab_step_iterations", C.c_int, [_VP, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int)]),
    ("heat_slab_info", C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_longlong)]),
    ("heat_destroy_slab", None, [_VP]),
    ("heat_probe_fma_rate", C.c_int, [C.c_int, C.c_int, _DP]),
    ("heat_debug_fail_engine_builds", C.c_int, [C.c_int]),
    ("heat_debug_loop_wait", C.c_int, [C.c_uint, C.c_double]),
    ("heat_probe_grid_barrier", C.c_int, [C.c_int, C.c_int, _DP]),
    ("heat_checks_compiled", C.c_int, []),
    ("heat_check_violations", C.c_int, [_VP, C.POINTER(C.c_uint)]),
    ("heat_last_error", C.c_char_p, []),
    ("heat_status_string", C.c_char_p, [C.c_int]),
]

EXPORTED = [name for name, _, _ in _SIGS]


def load_library(path: str = None):
    """Load libheatgb.so, or the library HEATGB_LIBRARY names (for example
    the index-checked build lib/libheatgb_check.so); raises if it has not
    been built: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("HEATGB_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1905_07622_gb300.build.build() "
                          "(the solver has no CPU fallback)")
    lib = C.CDLL(path)
    for name, res, args in _SIGS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st: int):
    if st != HEAT_OK:
        raise HeatError(st, _lib.heat_last_error().decode())


def _dev_ptr(t) -> int:
    """Device pointer of a contiguous torch CUDA tensor."""
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _host_f64(a, n: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _arg(a, n):
    """(pointer, on_device, keepalive) for a numpy host array or a CUDA tensor."""
    if hasattr(a, "is_cuda") and a.is_cuda:
        if a.numel() != n:
            raise ValueError(f"expected {n} values, got {a.numel()}")
        return _dev_ptr(a), 1, a
    h = _host_f64(a, n)
    return h.ctypes.data, 0, h


# ------------------------------------------------------------------ meshes

def heat_params_default(**overrides) -> heat_params:
    load_library()
    p = heat_params()
    _lib.heat_params_default(C.byref(p))
    for k, v in overrides.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "element" and isinstance(v, str):
            v = ELEMENTS[v]
        setattr(p, k, v)
    return p


def heat_create_mesh(nx, ny, nz, origin=(0.0, 0.0, 0.0), extent=(1.0, 1.0, 1.0)):
    load_library()
    o = (C.c_double * 3)(*origin)
    e = (C.c_double * 3)(*extent)
    out = C.c_void_p()
    _check(_lib.heat_create_mesh(int(nx), int(ny), int(nz), o, e, C.byref(out)))
    return out


def heat_destroy_mesh(mesh):
    if mesh:
        _lib.heat_destroy_mesh(mesh)


def heat_mesh_sizes(mesh):
    nn, ne = C.c_longlong(), C.c_longlong()
    _check(_lib.heat_mesh_sizes(mesh, C.byref(nn), C.byref(ne)))
    return nn.value, ne.value


def make_bc(dirichlet=None, flux=None, flux_steps=-1) -> heat_bc:
    bc = heat_bc()
    for f, v in (dirichlet or {}).items():
        bc.dirichlet_faces |= 1 << int(f)
        bc.dirichlet_value[int(f)] = float(v)
    for f, q in (flux or {}).items():
        bc.flux[int(f)] = float(q)
    bc.flux_steps = int(flux_steps)
    return bc


def heat_sim_create(mesh, bc: heat_bc, params: heat_params, stream=None):
    load_library()
    out = C.c_void_p()
    s = C.c_void_p(int(stream) if stream else 0)
    _check(_lib.heat_sim_create(mesh, C.byref(bc), C.byref(params), s, C.byref(out)))
    return out


def heat_destroy_sim(sim):
    if sim:
        _lib.heat_destroy_sim(sim)


def heat_set_coeffs(sim, rho_c, k, n_elems):
    pr, dr, keep1 = _arg(rho_c, n_elems)
    pk, dk, keep2 = _arg(k, n_elems)
    if dr != dk:
        raise ValueError("rho_c and k must both be host arrays or both CUDA tensors")
    _check(_lib.heat_set_coeffs(sim, C.c_void_p(pr), C.c_void_p(pk), dr))


def heat_set_params(sim, params: heat_params):
    _check(_lib.heat_set_params(sim, C.byref(params)))


def heat_set_state(sim, u, n_nodes):
    p, dev, keep = _arg(u, n_nodes)
    _check(_lib.heat_set_state(sim, C.c_void_p(p), dev))


def heat_get_state(sim, n_nodes, out=None):
    if out is not None and hasattr(out, "is_cuda") and out.is_cuda:
        _check(_lib.heat_get_state(sim, C.c_void_p(_dev_ptr(out)), 1))
        return out
    u = np.empty(n_nodes, dtype=np.float64)
    _check(_lib.heat_get_state(sim, C.c_void_p(u.ctypes.data), 0))
    return u


def heat_get_history(sim, n_nodes):
    """Checkpoint: (U^n, U^{n-1} or None, completed steps) as host arrays."""
    u1 = np.empty(n_nodes, dtype=np.float64)
    u2 = np.empty(n_nodes, dtype=np.float64)
    step, hp = C.c_int(), C.c_int()
    _check(_lib.heat_get_history(sim, C.c_void_p(u1.ctypes.data), C.c_void_p(u2.ctypes.data), C.byref(step),
                                 C.byref(hp), 0))
    return u1, (u2 if hp.value else None), step.value


def heat_set_history(sim, u_prev, u_prev2, step: int, n_nodes: int):
    """Resume from heat_get_history's output."""
    a = _host_f64(u_prev, n_nodes)
    b = _host_f64(u_prev2, n_nodes) if u_prev2 is not None else None
    _check(_lib.heat_set_history(sim, C.c_void_p(a.ctypes.data), C.c_void_p(b.ctypes.data if b is not None else 0),
                                 int(step), 0))


def heat_step(sim, nsteps: int) -> dict:
    st = heat_step_stats()
    _check(_lib.heat_step(sim, int(nsteps), C.byref(st)))
    return st.as_dict()


def heat_step_nocheck(sim, nsteps: int):
    """heat_step returning (status, stats) instead of raising."""
    st = heat_step_stats()
    rc = _lib.heat_step(sim, int(nsteps), C.byref(st))
    return rc, st.as_dict()


def heat_solve_transient(sim, nsteps: int, n_nodes: int):
    st = heat_step_stats()
    u = np.empty(n_nodes, dtype=np.float64)
    _check(_lib.heat_solve_transient(sim, int(nsteps), C.c_void_p(u.ctypes.data), C.byref(st)))
    return u, st.as_dict()


def heat_solve_transient_into(sim, nsteps: int, u_out: np.ndarray) -> dict:
    """heat_solve_transient into a caller-owned (e.g. pinned) float64 host array."""
    if u_out.dtype != np.float64 or not u_out.flags["C_CONTIGUOUS"]:
        raise ValueError("u_out must be a contiguous float64 array")
    st = heat_step_stats()
    _check(_lib.heat_solve_transient(sim, int(nsteps), C.c_void_p(u_out.ctypes.data), C.byref(st)))
    return st.as_dict()


def heat_step_iterations(sim, step: int) -> int:
    it = C.c_int()
    _check(_lib.heat_step_iterations(sim, int(step), C.byref(it)))
    return it.value


def heat_apply(sim, x, y):
    _check(_lib.heat_apply(sim, C.c_void_p(_dev_ptr(x)), C.c_void_p(_dev_ptr(y))))


def heat_apply_f32(sim, x, y):
    _check(_lib.heat_apply_f32(sim, C.c_void_p(_dev_ptr(x)), C.c_void_p(_dev_ptr(y))))


def heat_apply_general(sim, sa, sb, x, y):
    _check(_lib.heat_apply_general(sim, float(sa), float(sb), C.c_void_p(_dev_ptr(x)), C.c_void_p(_dev_ptr(y))))


def heat_diagonal(sim, p):
    _check(_lib.heat_diagonal(sim, C.c_void_p(_dev_ptr(p))))


def heat_rhs(sim, n, u_prev, b):
    _check(_lib.heat_rhs(sim, int(n), C.c_void_p(_dev_ptr(u_prev)), C.c_void_p(_dev_ptr(b))))


def heat_flux_vector(sim, f):
    _check(_lib.heat_flux_vector(sim, C.c_void_p(_dev_ptr(f))))


def heat_profile_iteration(sim, reps: int, flush=None):
    """Mean ms per launch and algorithmic bytes of the two CG-iteration kernels."""
    ma, mu, ba, bu = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    fp = C.c_void_p(_dev_ptr(flush)) if flush is not None else C.c_void_p(0)
    fb = flush.numel() * flush.element_size() if flush is not None else 0
    _check(_lib.heat_profile_iteration(sim, int(reps), fp, fb, C.byref(ma), C.byref(mu), C.byref(ba), C.byref(bu)))
    return {"ms_apply": ma.value, "ms_update": mu.value, "bytes_apply": ba.value, "bytes_update": bu.value}


def heat_server_create(hbm_budget_bytes: int, max_active: int, stream=None):
    load_library()
    out = C.c_void_p()
    st = C.c_void_p(int(stream) if stream else 0)
    _check(_lib.heat_server_create(int(hbm_budget_bytes), int(max_active), st, C.byref(out)))
    return out


def make_request(p, precision="fp32_refined", **param_overrides):
    """heat_request for a workloads.Problem-like object; keep the returned
    arrays alive until heat_submit returns (it copies them)."""
    rc = np.ascontiguousarray(p.rho_c, dtype=np.float64)
    kk = np.ascontiguousarray(p.k, dtype=np.float64)
    u0 = np.ascontiguousarray(p.u0, dtype=np.float64) if p.u0 is not None else None
    req = heat_request()
    req.nx, req.ny, req.nz = p.nx, p.ny, p.nz
    req.origin = (C.c_double * 3)(*p.origin)
    req.extent = (C.c_double * 3)(*p.extent)
    req.rho_c = rc.ctypes.data
    req.k = kk.ctypes.data
    req.u0 = u0.ctypes.data if u0 is not None else None
    req.bc = make_bc(p.dirichlet, p.flux, p.flux_steps)
    kw = dict(theta=p.theta, dt=p.dt, rtol=p.rtol, precision=precision, element=getattr(p, "element", "q1"))
    kw.update(param_overrides)
    req.params = heat_params_default(**kw)
    req.nsteps = int(p.nsteps)
    return req, (rc, kk, u0)


def heat_submit(server, req) -> int:
    t = C.c_uint64()
    _check(_lib.heat_submit(server, C.byref(req), C.byref(t)))
    return t.value


def heat_poll(server, ticket: int) -> bool:
    d = C.c_int()
    _check(_lib.heat_poll(server, C.c_uint64(ticket), C.byref(d)))
    return bool(d.value)


def heat_wait(server, ticket: int, n_nodes: int, timeout_s: float = 600.0):
    """(u, stats, latency_s); raises HeatError on failure or timeout."""
    u = np.empty(n_nodes, dtype=np.float64)
    st = heat_step_stats()
    lat = C.c_double()
    _check(_lib.heat_wait(server, C.c_uint64(ticket), float(timeout_s), C.c_void_p(u.ctypes.data), C.byref(st),
                          C.byref(lat)))
    return u, st.as_dict(), lat.value


def heat_server_get_stats(server) -> dict:
    s = heat_server_stats()
    _check(_lib.heat_server_get_stats(server, C.byref(s)))
    return s.as_dict()


def heat_destroy_server(server):
    if server:
        _lib.heat_destroy_server(server)


def heat_batch_create(sims, stream=None):
    """A batch over simulation handles (c_void_p); the sims stay the caller's."""
    load_library()
    arr = (C.c_void_p * len(sims))(*[s.value if isinstance(s, C.c_void_p) else s for s in sims])
    out = C.c_void_p()
    st = C.c_void_p(int(stream) if stream else 0)
    _check(_lib.heat_batch_create(arr, len(sims), st, C.byref(out)))
    return out


def heat_batch_step(batch, nsteps: int, nsims: int):
    """Advance every member; returns (status, [per-member stats dicts])."""
    stats = (heat_step_stats * nsims)()
    rc = _lib.heat_batch_step(batch, int(nsteps), stats)
    return rc, [s.as_dict() for s in stats]


def heat_destroy_batch(batch):
    if batch:
        _lib.heat_destroy_batch(batch)


def _check_noalloc_args(nx, ny, nz, coef, x, y, xdoty):
    """The C entry point cannot see device buffer sizes: check them here, with
    dtype and device, before any pointer reaches it."""
    nx, ny, nz = int(nx), int(ny), int(nz)
    if nx < 1 or ny < 1 or nz < 1:
        raise ValueError("heat_apply_dot_noalloc: mesh sizes must be >= 1")
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    need = {"coef": 2 * nx * ny * nz, "x": nn, "y": nn, "xdoty": 1}
    tens = {"coef": coef, "x": x, "y": y, "xdoty": xdoty}
    import torch
    for name, t in tens.items():
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"heat_apply_dot_noalloc: {name} must be a torch tensor")
        if t.dtype != torch.float64:
            raise ValueError(f"heat_apply_dot_noalloc: {name} must be float64, got {t.dtype}")
        if name == "xdoty" and t.numel() < 1 or name != "xdoty" and t.numel() != need[name]:
            raise ValueError(f"heat_apply_dot_noalloc: {name} needs {need[name]} values, got {t.numel()}")
    for name, t in tens.items():
        if not t.is_cuda:
            raise ValueError(f"heat_apply_dot_noalloc: {name} must be a CUDA tensor")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"heat_apply_dot_noalloc: {name} is on cuda:{t.device.index}, "
                             f"the current device is cuda:{torch.cuda.current_device()}")


def heat_apply_dot_noalloc(nx, ny, nz, extent, dt, theta, dirichlet_faces, coef, x, y, xdoty, stream=None):
    """Allocation-free y = A' x and x.A'x on caller-owned CUDA tensors (see include/heat.h).
    Raises ValueError/TypeError for tensors of the wrong dtype, length or device."""
    _check_noalloc_args(nx, ny, nz, coef, x, y, xdoty)
    load_library()
    ext = (C.c_double * 3)(*extent)
    s = C.c_void_p(int(stream) if stream else 0)
    _check(_lib.heat_apply_dot_noalloc(int(nx), int(ny), int(nz), ext, float(dt), float(theta),
                                       int(dirichlet_faces), C.c_void_p(_dev_ptr(coef)), C.c_void_p(_dev_ptr(x)),
                                       C.c_void_p(_dev_ptr(y)), C.c_void_p(_dev_ptr(xdoty)), s))


def heat_batch_profile_iteration(batch, reps: int, flush=None):
    """heat_profile_iteration over every member of a batch."""
    ma, mu, ba, bu = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    fp = C.c_void_p(_dev_ptr(flush)) if flush is not None else C.c_void_p(0)
    fb = flush.numel() * flush.element_size() if flush is not None else 0
    _check(_lib.heat_batch_profile_iteration(batch, int(reps), fp, fb, C.byref(ma), C.byref(mu), C.byref(ba),
                                             C.byref(bu)))
    return {"ms_apply": ma.value, "ms_update": mu.value, "bytes_apply": ba.value, "bytes_update": bu.value}


def heat_debug_fail_engine_builds(n: int):
    """Testing hook: the next n engine builds or membership updates fail (HEAT_ERR_NOMEM)."""
    load_library()
    _check(_lib.heat_debug_fail_engine_builds(int(n)))


def heat_debug_loop_wait(extra_arrivals: int, limit_s: float):
    """Testing hook: engines built afterwards expect extra_arrivals (0 or 1) more
    arrivals at each persistent-iteration barrier and bound one wait by
    limit_s seconds (0: the default bound)."""
    load_library()
    _check(_lib.heat_debug_loop_wait(int(extra_arrivals), float(limit_s)))


def heat_probe_grid_barrier(blocks_per_sm: int, reps: int = 2000) -> float:
    """Microseconds per grid barrier of the persistent iteration, measured alone."""
    load_library()
    us = C.c_double()
    _check(_lib.heat_probe_grid_barrier(int(blocks_per_sm), int(reps), C.byref(us)))
    return us.value


def heat_probe_fma_rate(fp64: bool, reps: int = 5) -> float:
    """Measured FMA throughput of the current GPU in TFLOP/s (FP64 or FP32)."""
    load_library()
    t = C.c_double()
    _check(_lib.heat_probe_fma_rate(1 if fp64 else 0, int(reps), C.byref(t)))
    return t.value


def heat_tuning_num_variants() -> int:
    load_library()
    return int(_lib.heat_tuning_num_variants())


def heat_tuning_variant(v: int) -> dict:
    load_library()
    a, b, c, d, e, f = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
    _check(_lib.heat_tuning_variant(int(v), C.byref(a), C.byref(b), C.byref(c), C.byref(d), C.byref(e), C.byref(f)))
    return {"seg_width": a.value, "rows": b.value, "warps": c.value, "has_fp64": bool(d.value), "stages": e.value,
            "fused": bool(f.value)}


def heat_tuning_get() -> dict:
    load_library()
    t = heat_tuning()
    _check(_lib.heat_tuning_get(C.byref(t)))
    return t.as_dict()


def heat_tuning_set(variant, seg_nodes, pw_quads=None, open_w=None, loop=None):
    """Set the table; pw_quads=None / open_w=None / loop=None keep the current
    pointwise item sizes / open-pass forms / iteration forms."""
    load_library()
    cur = heat_tuning_get()
    if pw_quads is None:
        pw_quads = cur["pw_quads"]
    if open_w is None:
        open_w = cur["open_w"]
    if loop is None:
        loop = cur["loop"]
    t = heat_tuning((C.c_int * 3)(*variant), (C.c_int * 3)(*seg_nodes), (C.c_int * 3)(*pw_quads),
                    (C.c_int * 3)(*open_w), (C.c_int * 3)(*loop))
    _check(_lib.heat_tuning_set(C.byref(t)))


def heat_autotune(sim, reps: int):
    """Tune the table for this sim's precision and size; returns (table, best ms per CG iteration)."""
    t = heat_tuning()
    ms = C.c_double()
    _check(_lib.heat_autotune(sim, int(reps), C.byref(t), C.byref(ms)))
    return t.as_dict(), ms.value


def heat_batch_autotune(batch, reps: int):
    """heat_autotune over every member of a batch; returns (table, best ms per CG iteration)."""
    t = heat_tuning()
    ms = C.c_double()
    _check(_lib.heat_batch_autotune(batch, int(reps), C.byref(t), C.byref(ms)))
    return t.as_dict(), ms.value


def make_corrosion(z0, half_width, rho_c_sound, k_sound, rho_c_corr, k_corr) -> heat_corrosion:
    return heat_corrosion(float(z0), float(half_width), float(rho_c_sound), float(k_sound), float(rho_c_corr),
                          float(k_corr))


def heat_set_face_flux(sim, face: int, q, n_face_elems: int = 0):
    """Per-element flux densities on one face (host array or CUDA tensor); q=None restores uniform."""
    if q is None:
        _check(_lib.heat_set_face_flux(sim, int(face), None, 0))
        return
    if hasattr(q, "data_ptr"):
        _check(_lib.heat_set_face_flux(sim, int(face), C.c_void_p(_dev_ptr(q)), 1))
    else:
        a = np.ascontiguousarray(q, dtype=np.float64)
        _check(_lib.heat_set_face_flux(sim, int(face), C.c_void_p(a.ctypes.data), 0))


def heat_get_coeffs(sim, n_elems: int):
    """(rho_c, k) per element as host arrays."""
    rc = np.empty(n_elems)
    kk = np.empty(n_elems)
    _check(_lib.heat_get_coeffs(sim, C.c_void_p(rc.ctypes.data), C.c_void_p(kk.ctypes.data), 0))
    return rc, kk


def heat_cheb_interval(sim):
    """(lam_lo, lam_hi) of the Chebyshev preconditioner (cheb_degree >= 2)."""
    lo, hi = C.c_double(), C.c_double()
    _check(_lib.heat_cheb_interval(sim, C.byref(lo), C.byref(hi)))
    return lo.value, hi.value


def heat_set_coeffs_corrosion(sim, geom: heat_corrosion, depth: float):
    _check(_lib.heat_set_coeffs_corrosion(sim, C.byref(geom), float(depth)))


def heat_face_loglik(sim, face: int, data, sigma: float, out):
    """-1/2 sum((U - data)/sigma)^2 over a face's nodes into out[0] (CUDA tensors)."""
    _check(_lib.heat_face_loglik(sim, int(face), C.c_void_p(_dev_ptr(data)), float(sigma),
                                 C.c_void_p(_dev_ptr(out))))


class MHDriver:
    """heat_mh_* (batched Metropolis-Hastings over the corrosion depth)."""

    def __init__(self, nx, ny, nz, extent, geom, data, sigma, nchains, nsteps, depth_max, *, origin=(0, 0, 0),
                 flux_face=-1, flux_q=None, obs_face=2, u0=0.0, dirichlet=None, flux=None, flux_steps=-1,
                 stream=None, **params):
        load_library()
        cfg = heat_mh_config()
        cfg.nx, cfg.ny, cfg.nz = int(nx), int(ny), int(nz)
        cfg.origin = (C.c_double * 3)(*origin)
        cfg.extent = (C.c_double * 3)(*extent)
        cfg.bc = make_bc(dirichlet or {}, flux or {}, flux_steps)
        cfg.params = heat_params_default(**params)
        cfg.nsteps = int(nsteps)
        cfg.u0 = float(u0)
        self._q = np.ascontiguousarray(flux_q, dtype=np.float64) if flux_q is not None else None
        cfg.flux_face = int(flux_face) if self._q is not None else -1
        cfg.flux_q = self._q.ctypes.data if self._q is not None else None
        cfg.geom = geom
        cfg.obs_face = int(obs_face)
        self._data = np.ascontiguousarray(data, dtype=np.float64)
        cfg.data = self._data.ctypes.data
        cfg.sigma = float(sigma)
        cfg.depth_max = float(depth_max)
        cfg.nchains = int(nchains)
        self.nchains = int(nchains)
        self.h = C.c_void_p()
        st = C.c_void_p(int(stream) if stream else 0)
        _check(_lib.heat_mh_create(C.byref(cfg), st, C.byref(self.h)))

    def loglik(self, depths):
        d = np.ascontiguousarray(depths, dtype=np.float64)
        out = np.empty(self.nchains)
        _check(_lib.heat_mh_loglik(self.h, C.c_void_p(d.ctypes.data), C.c_void_p(out.ctypes.data)))
        return out

    def run(self, niter, step, normals, uniforms, state, state_ll=None):
        """Returns (state, state_ll, depth_trace, ll_trace, accepted); traces are (niter, nchains)."""
        n = self.nchains
        nz = np.ascontiguousarray(normals, dtype=np.float64).reshape(niter * n)
        un = np.ascontiguousarray(uniforms, dtype=np.float64).reshape(niter * n)
        st = np.array(state, dtype=np.float64).copy()
        ll = np.array(state_ll, dtype=np.float64).copy() if state_ll is not None else self.loglik(st)
        dt = np.empty(niter * n)
        lt = np.empty(niter * n)
        acc = np.empty(niter * n, dtype=np.int32)
        _check(_lib.heat_mh_run(self.h, int(niter), float(step), C.c_void_p(nz.ctypes.data),
                                C.c_void_p(un.ctypes.data), C.c_void_p(st.ctypes.data),
                                C.c_void_p(ll.ctypes.data), C.c_void_p(dt.ctypes.data),
                                C.c_void_p(lt.ctypes.data), C.c_void_p(acc.ctypes.data)))
        return st, ll, dt.reshape(niter, n), lt.reshape(niter, n), acc.reshape(niter, n).astype(bool)

    def stats(self):
        """(forward solves, CG iterations) so far."""
        a, b = C.c_longlong(), C.c_longlong()
        _check(_lib.heat_mh_stats(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def close(self):
        if self.h:
            _lib.heat_mh_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def heat_checks_compiled() -> bool:
    load_library()
    return bool(_lib.heat_checks_compiled())


def heat_check_violations(sim) -> int:
    n = C.c_uint()
    _check(_lib.heat_check_violations(sim, C.byref(n)))
    return n.value


def heat_last_error() -> str:
    load_library()
    return _lib.heat_last_error().decode()


# ------------------------------------------------------------ convenience

@dataclass
class Simulation:
    """Owns a mesh + sim pair built from a workloads.Problem-like object."""

    mesh: C.c_void_p
    sim: C.c_void_p
    n_nodes: int
    n_elems: int

    @classmethod
    def from_problem(cls, p, precision="fp64", stream=None, coeffs_on_device=False, **param_overrides):
        mesh = heat_create_mesh(p.nx, p.ny, p.nz, p.origin, p.extent)
        try:
            nn, ne = heat_mesh_sizes(mesh)
            kw = dict(theta=p.theta, dt=p.dt, rtol=p.rtol, precision=precision,
                      element=getattr(p, "element", "q1"))
            kw.update(param_overrides)
            prm = heat_params_default(**kw)
            bc = make_bc(p.dirichlet, p.flux, p.flux_steps)
            sim = heat_sim_create(mesh, bc, prm, stream)
        except Exception:
            heat_destroy_mesh(mesh)
            raise
        self = cls(mesh, sim, nn, ne)
        try:
            if coeffs_on_device:
                import torch
                rc = torch.as_tensor(p.rho_c, dtype=torch.float64, device="cuda")
                kk = torch.as_tensor(p.k, dtype=torch.float64, device="cuda")
                heat_set_coeffs(sim, rc, kk, ne)
            else:
                heat_set_coeffs(sim, p.rho_c, p.k, ne)
            heat_set_state(sim, p.u0, nn)
        except Exception:
            self.close()
            raise
        return self

    def step(self, nsteps):
        return heat_step(self.sim, nsteps)

    def state(self):
        return heat_get_state(self.sim, self.n_nodes)

    def set_params(self, **kw):
        heat_set_params(self.sim, heat_params_default(**kw))

    def close(self):
        if self.sim:
            heat_destroy_sim(self.sim)
            self.sim = None
        if self.mesh:
            heat_destroy_mesh(self.mesh)
            self.mesh = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


load_library()


# ---- one simulation split into z-slabs (include/heat.h, §4.4) -------------

def heat_slab_plan(nz: int, nslabs: int) -> list:
    """First owned node layer of each slab, plus nz + 1 (host only, no GPU)."""
    load_library()
    out = (C.c_int * (int(nslabs) + 1))()
    _check(_lib.heat_slab_plan(int(nz), int(nslabs), out))
    return list(out)


def heat_slab_create(mesh, bc, prm, nslabs: int, merged: bool = True, stream=None):
    load_library()
    out = _VP()
    s = C.c_void_p(int(stream) if stream else 0)
    _check(_lib.heat_slab_create(mesh, C.byref(bc), C.byref(prm), int(nslabs), 1 if merged else 0, s,
                                 C.byref(out)))
    return out


def heat_slab_set_coeffs(slab, rho_c, k, ne: int):
    a, b = _host_f64(rho_c, ne), _host_f64(k, ne)
    _check(_lib.heat_slab_set_coeffs(slab, a.ctypes.data, b.ctypes.data))


def heat_slab_set_state(slab, u, nn: int):
    a = _host_f64(u, nn)
    _check(_lib.heat_slab_set_state(slab, a.ctypes.data))


def heat_slab_get_state(slab, nn: int) -> np.ndarray:
    out = np.empty(nn)
    _check(_lib.heat_slab_get_state(slab, out.ctypes.data))
    return out


def heat_slab_step(slab, nsteps: int) -> dict:
    """Advance nsteps; returns heat_step_stats as a dict (raises HeatError on failure)."""
    st = heat_step_stats()
    rc = _lib.heat_slab_step(slab, int(nsteps), C.byref(st))
    d = st.as_dict()
    if rc != HEAT_OK:
        raise HeatError(rc, _lib.heat_last_error().decode())
    return d


def heat_slab_step_iterations(slab, cap: int = 1 << 16) -> list:
    out = (C.c_int * cap)()
    n = C.c_int()
    _check(_lib.heat_slab_step_iterations(slab, out, cap, C.byref(n)))
    return list(out[: min(cap, n.value)])


def heat_slab_info(slab) -> dict:
    ns = C.c_int()
    _check(_lib.heat_slab_info(slab, C.byref(ns), None, None))
    first = (C.c_int * (ns.value + 1))()
    nb = C.c_longlong()
    _check(_lib.heat_slab_info(slab, C.byref(ns), first, C.byref(nb)))
    return {"nslabs": ns.value, "first_layer": list(first), "device_bytes": nb.value}


def heat_destroy_slab(slab):
    if slab:
        _lib.heat_destroy_slab(slab)


class SlabSimulation:
    """One Problem split into z-slabs on the current GPU (heat_slab_*)."""

    def __init__(self, mesh, slab, nn, ne):
        self.mesh, self.slab, self.nn, self.ne = mesh, slab, nn, ne

    @classmethod
    def from_problem(cls, p, nslabs: int, merged: bool = True, stream=None, **param_overrides):
        mesh = heat_create_mesh(p.nx, p.ny, p.nz, p.origin, p.extent)
        try:
            nn, ne = heat_mesh_sizes(mesh)
            kw = dict(theta=p.theta, dt=p.dt, rtol=p.rtol, precision="fp64")
            kw.update(param_overrides)
            prm = heat_params_default(**kw)
            bc = make_bc(p.dirichlet, p.flux, p.flux_steps)
            slab = heat_slab_create(mesh, bc, prm, nslabs, merged, stream)
        except Exception:
            heat_destroy_mesh(mesh)
            raise
        self = cls(mesh, slab, nn, ne)
        try:
            heat_slab_set_coeffs(slab, p.rho_c, p.k, ne)
            heat_slab_set_state(slab, p.u0, nn)
        except Exception:
            self.close()
            raise
        return self

    def step(self, nsteps):
        return heat_slab_step(self.slab, nsteps)

    def state(self) -> np.ndarray:
        return heat_slab_get_state(self.slab, self.nn)

    def set_state(self, u):
        heat_slab_set_state(self.slab, u, self.nn)

    def iterations(self) -> list:
        return heat_slab_step_iterations(self.slab)

    def close(self):
        if self.slab:
            heat_destroy_slab(self.slab)
            self.slab = None
        if self.mesh:
            heat_destroy_mesh(self.mesh)
            self.mesh = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
