"""Thin ctypes binding of libswkb.so (include/swkb.h).

Argument marshalling only: every step of the propagation runs in the CUDA
library.  There is no CPU fallback -- loading fails loudly when the in-tree
library has not been built (``python -c "import __graft_entry__ as g;
g.build()"``).  Torch is optional and used only to hand device buffers and
streams to the library (``on_device=True`` with CUDA tensors).
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_char_p, c_double, c_int32, c_size_t, c_uint64, c_void_p

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libswkb.so")

SWKB_OK = 0
SWKB_ERR_INVALID_ARG = 1
SWKB_ERR_OOM = 2
SWKB_ERR_CAUSTIC = 3
SWKB_ERR_TURNING = 4
SWKB_ERR_RANGE = 5
SWKB_ERR_CUDA = 6
SWKB_ERR_TIMEOUT = 7
SWKB_ERR_AGAIN = 8
SWKB_NOT_READY = 9
SWKB_ERR_CANCELLED = 10

SWKB_BC_PERIODIC, SWKB_BC_NEUMANN, SWKB_BC_DIRICHLET, SWKB_BC_OPEN = 0, 1, 2, 3
SWKB_FP64, SWKB_MIXED = 0, 1

KERNEL_KINDS = ("init", "reduce", "fft", "march", "bracket", "resum", "output")

EXPORTED = ("swkb_options_default", "swkb_plan_create", "swkb_plan_get_info", "swkb_propagate",
            "swkb_propagate_planes", "swkb_debug_screen", "swkb_plan_destroy", "swkb_plan_set_timing",
            "swkb_plan_get_stats", "swkb_server_create", "swkb_submit",
            "swkb_poll", "swkb_cancel", "swkb_server_get_stats", "swkb_server_destroy",
            "swkb_last_error", "swkb_status_string", "swkb_modes_noalloc", "swkb_sym_eig",
            "swkb_hill_propagate", "swkb_batch_options_default", "swkb_batch_create",
            "swkb_batch_run", "swkb_batch_get_info", "swkb_batch_destroy")


class SwkbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"swkb status {status}: {msg}")
        self.status = status


class swkb_profile(ctypes.Structure):
    _fields_ = [("n_cols", c_int32), ("x_cols", POINTER(c_double)), ("n_p", c_int32),
                ("z0_p", c_double), ("dz_p", c_double), ("eps", POINTER(c_double)),
                ("eps_z", POINTER(c_double)), ("eps_zz", POINTER(c_double))]


class swkb_domain(ctypes.Structure):
    _fields_ = [("z_a", c_double), ("z_b", c_double), ("x0", c_double), ("bc", c_int32)]


class swkb_options(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("theta_max", c_double), ("n_max", c_int32),
                ("ray_stride", c_int32), ("rk4_steps", c_int32), ("absorber_frac", c_double),
                ("autotune", c_int32), ("cuda_stream", c_void_p), ("device", c_int32),
                ("reuse_rays", c_int32), ("planes", c_int32), ("tile_points", c_int32),
                ("ctas_per_sm", c_int32), ("fft_n1", c_int32), ("fc_patch", c_int32),
                ("fc_overlap", c_int32)]


class swkb_plan_info(ctypes.Structure):
    _fields_ = [("n_fft", c_int32), ("n_max", c_int32), ("n_modes", c_int32),
                ("n_rays", c_int32), ("n_ghost", c_int32), ("n_rays_total", c_int32),
                ("tile_points", c_int32), ("mode_groups", c_int32), ("march_modes", c_int32),
                ("resum_points", c_int32), ("fft_n1", c_int32), ("dz", c_double),
                ("period", c_double), ("eps_ref", c_double), ("device_bytes", c_size_t),
                ("medium_pieces", c_int32), ("ctas_per_sm", c_int32), ("fc_patches", c_int32),
                ("fc_period_points", c_int32)]


class swkb_hill_desc(ctypes.Structure):
    _fields_ = [("bc", c_int32), ("z_a", c_double), ("z_b", c_double), ("z_sym", c_double),
                ("n_z", c_int32), ("K", c_int32), ("n_q", c_int32)]


class swkb_plan_stats(ctypes.Structure):
    _fields_ = [("launches", c_uint64), ("screens", c_uint64),
                ("kernel_launches", c_uint64 * len(KERNEL_KINDS)),
                ("kernel_timed", c_uint64 * len(KERNEL_KINDS)),
                ("kernel_ms", c_double * len(KERNEL_KINDS))]


class swkb_request(ctypes.Structure):
    _fields_ = [("profile", POINTER(swkb_profile)), ("k", c_double),
                ("domain", POINTER(swkb_domain)), ("n_z", c_int32), ("screen_dx", c_double),
                ("options", POINTER(swkb_options)), ("u0", POINTER(c_double)), ("q0", c_int32),
                ("n_screens", c_int32)]


class swkb_batch_options(ctypes.Structure):
    _fields_ = [("ctas_per_sm", c_int32), ("wait_limit_ms", c_int32), ("device", c_int32),
                ("cuda_stream", c_void_p)]


class swkb_batch_info(ctypes.Structure):
    _fields_ = [("instances", c_int32), ("precision", c_int32), ("grid", c_int32),
                ("ctas_per_sm", c_int32), ("threads", c_int32), ("jobs", c_int32),
                ("items", ctypes.c_int64), ("steps", c_int32), ("shared_bytes", c_size_t),
                ("device_bytes", c_size_t)]


class swkb_server_stats(ctypes.Structure):
    _fields_ = [("submitted", c_uint64), ("completed", c_uint64), ("failed", c_uint64),
                ("rejected", c_uint64), ("resident", c_int32), ("queued", c_int32),
                ("hbm_in_use", c_size_t)]


_lib = None


def lib():
    """Load the in-tree libswkb.so (raises if it has not been built).
    SWKB_CHECKED=1 loads the bounds-checked build libswkb_checked.so instead."""
    global _lib
    if _lib is None:
        path = LIB_PATH
        if os.environ.get("SWKB_CHECKED") == "1":
            path = LIB_PATH.replace("libswkb.so", "libswkb_checked.so")
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_2301_03814_gb300.build")
        L = ctypes.CDLL(path)
        L.swkb_options_default.argtypes = [POINTER(swkb_options)]
        L.swkb_options_default.restype = None
        L.swkb_plan_create.argtypes = [POINTER(swkb_profile), c_double, POINTER(swkb_domain),
                                       c_int32, c_double, POINTER(swkb_options), POINTER(c_void_p)]
        L.swkb_plan_get_info.argtypes = [c_void_p, POINTER(swkb_plan_info)]
        L.swkb_propagate.argtypes = [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_int32,
                                     c_int32]
        L.swkb_propagate_planes.argtypes = [c_void_p, c_void_p, c_int32, c_int32, c_int32,
                                            c_void_p, c_int32]
        L.swkb_debug_screen.argtypes = [c_void_p, c_int32] + [c_void_p] * 6
        L.swkb_plan_set_timing.argtypes = [c_void_p, c_int32, c_int32]
        L.swkb_plan_get_stats.argtypes = [c_void_p, POINTER(swkb_plan_stats)]
        L.swkb_plan_destroy.argtypes = [c_void_p]
        L.swkb_plan_destroy.restype = None
        L.swkb_server_create.argtypes = [c_size_t, c_int32, c_int32, c_int32, POINTER(c_void_p)]
        L.swkb_submit.argtypes = [c_void_p, POINTER(swkb_request), POINTER(c_uint64)]
        L.swkb_poll.argtypes = [c_void_p, c_uint64, c_void_p, c_int32]
        L.swkb_cancel.argtypes = [c_void_p, c_uint64]
        L.swkb_server_get_stats.argtypes = [c_void_p, POINTER(swkb_server_stats)]
        L.swkb_server_destroy.argtypes = [c_void_p]
        L.swkb_server_destroy.restype = None
        L.swkb_modes_noalloc.argtypes = [c_void_p, c_int32, c_int32, c_void_p, c_void_p]
        L.swkb_modes_noalloc.restype = c_int32
        L.swkb_sym_eig.argtypes = [c_int32, c_int32, c_void_p, c_void_p, c_void_p,
                                   POINTER(c_int32), c_int32, c_void_p]
        L.swkb_sym_eig.restype = c_int32
        L.swkb_hill_propagate.argtypes = [POINTER(swkb_hill_desc), c_int32, c_void_p, c_void_p,
                                          c_void_p, c_int32, c_void_p, c_void_p, c_void_p,
                                          c_int32, c_void_p]
        L.swkb_hill_propagate.restype = c_int32
        L.swkb_batch_options_default.argtypes = [POINTER(swkb_batch_options)]
        L.swkb_batch_options_default.restype = None
        L.swkb_batch_create.argtypes = [c_int32, POINTER(swkb_request), POINTER(swkb_batch_options),
                                        POINTER(c_void_p)]
        L.swkb_batch_create.restype = c_int32
        L.swkb_batch_run.argtypes = [c_void_p, c_void_p, c_void_p, c_int32]
        L.swkb_batch_run.restype = c_int32
        L.swkb_batch_get_info.argtypes = [c_void_p, POINTER(swkb_batch_info)]
        L.swkb_batch_get_info.restype = c_int32
        L.swkb_batch_destroy.argtypes = [c_void_p]
        L.swkb_batch_destroy.restype = None
        L.swkb_last_error.restype = c_char_p
        L.swkb_status_string.restype = c_char_p
        L.swkb_status_string.argtypes = [c_int32]
        for name in ("swkb_plan_create", "swkb_plan_get_info", "swkb_propagate",
                     "swkb_plan_set_timing", "swkb_plan_get_stats",
                     "swkb_debug_screen", "swkb_server_create", "swkb_submit", "swkb_poll",
                     "swkb_cancel", "swkb_server_get_stats"):
            getattr(L, name).restype = c_int32
        _lib = L
    return _lib


def check(status: int, allow=(SWKB_OK,)) -> int:
    if status not in allow:
        raise SwkbError(status, lib().swkb_last_error().decode(errors="replace"))
    return status


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(POINTER(c_double))


# --------------------------------------------------------------------------
# argument marshalling
# --------------------------------------------------------------------------
class _Keep:
    """Holds the numpy buffers a C struct points into."""

    def __init__(self):
        self.refs = []

    def f64(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        self.refs.append(a)
        return a


def make_profile(profile, keep: _Keep) -> swkb_profile:
    p = swkb_profile()
    p.n_cols = int(profile.eps.shape[0])
    p.n_p = int(profile.eps.shape[1])
    p.x_cols = _dptr(keep.f64(profile.x_cols))
    p.z0_p = float(profile.z0)
    p.dz_p = float(profile.dz)
    p.eps = _dptr(keep.f64(profile.eps))
    p.eps_z = _dptr(keep.f64(profile.eps_z))
    p.eps_zz = _dptr(keep.f64(profile.eps_zz))
    return p


def swkb_options_default() -> swkb_options:
    o = swkb_options()
    lib().swkb_options_default(byref(o))
    return o


def options_for(problem, precision=SWKB_FP64, stream=None, device=0, autotune=False,
                reuse_rays=False, planes=0, tiling=None) -> swkb_options:
    """tiling: None, or fixed launch shapes (tile_points, ctas_per_sm, fft_n1)
    as swkb_plan_info reports them."""
    o = swkb_options_default()
    o.precision = precision
    o.theta_max = float(problem.theta_max)
    o.n_max = int(problem.n_max)
    o.ray_stride = int(problem.ray_stride)
    o.rk4_steps = int(problem.rk4_steps)
    o.absorber_frac = float(problem.absorber_frac)
    o.cuda_stream = stream
    o.device = device
    o.autotune = 1 if autotune else 0
    o.reuse_rays = 1 if reuse_rays else 0
    o.planes = int(planes)
    o.fc_patch = int(getattr(problem, "fc_patch", 0))
    o.fc_overlap = int(getattr(problem, "fc_overlap", 0))
    if tiling is not None:
        o.tile_points, o.ctas_per_sm, o.fft_n1 = (int(v) for v in tiling)
    return o


def swkb_plan_create(profile, k, domain: swkb_domain, n_z, screen_dx, options: swkb_options):
    keep = _Keep()
    prof = make_profile(profile, keep)
    handle = c_void_p()
    check(lib().swkb_plan_create(byref(prof), float(k), byref(domain), int(n_z),
                                 float(screen_dx), byref(options), byref(handle)))
    return handle


def swkb_plan_get_info(plan) -> swkb_plan_info:
    info = swkb_plan_info()
    check(lib().swkb_plan_get_info(plan, byref(info)))
    return info


def swkb_propagate(plan, u0, q0, n_screens, u_out, snapshot_every=0, on_device=0):
    """u0 / u_out: numpy complex128 arrays (host) or integer device pointers
    (on_device=1)."""
    if on_device:
        return check(lib().swkb_propagate(plan, c_void_p(int(u0)), q0, n_screens,
                                          c_void_p(int(u_out)), snapshot_every, 1))
    return check(lib().swkb_propagate(plan, u0.ctypes.data_as(c_void_p), q0, n_screens,
                                      u_out.ctypes.data_as(c_void_p), snapshot_every, 0))


def swkb_propagate_planes(plan, u0, q0, n_screens, planes, u_out, on_device=0):
    """Fields on `planes` planes per screen (rows ordered (screen, plane));
    u0 / u_out as in swkb_propagate."""
    if on_device:
        return check(lib().swkb_propagate_planes(plan, c_void_p(int(u0)), q0, n_screens, planes,
                                                 c_void_p(int(u_out)), 1))
    return check(lib().swkb_propagate_planes(plan, u0.ctypes.data_as(c_void_p), q0, n_screens,
                                             planes, u_out.ctypes.data_as(c_void_p), 0))


def swkb_plan_destroy(plan):
    lib().swkb_plan_destroy(plan)


TIME_ALL = (1 << len(KERNEL_KINDS)) - 1
TIME_SERIAL = 1 << 30


def swkb_plan_set_timing(plan, kinds, every=1, serial=False):
    """kinds: True (all kernel kinds), False (off), or an int bit mask /
    an iterable of kind names ("march", "resum", ...); every: time one launch
    in `every` of each selected kind; serial: march on the plan's stream too,
    so that each timed launch has the GPU to itself."""
    if kinds is True:
        mask = TIME_ALL
    elif kinds is False or kinds is None:
        mask = 0
    elif isinstance(kinds, int):
        mask = kinds
    else:
        mask = 0
        for k in kinds:
            mask |= 1 << KERNEL_KINDS.index(k)
    if serial:
        mask |= TIME_SERIAL
    check(lib().swkb_plan_set_timing(plan, int(mask), int(every)))


def swkb_plan_get_stats(plan) -> dict:
    st = swkb_plan_stats()
    check(lib().swkb_plan_get_stats(plan, byref(st)))
    return {"launches": int(st.launches), "screens": int(st.screens),
            "kernel_launches": {k: int(st.kernel_launches[i]) for i, k in enumerate(KERNEL_KINDS)},
            "kernel_timed": {k: int(st.kernel_timed[i]) for i, k in enumerate(KERNEL_KINDS)},
            "kernel_ms": {k: float(st.kernel_ms[i]) for i, k in enumerate(KERNEL_KINDS)}}


def swkb_modes_noalloc(u_ptr: int, n_fft: int, n_max: int, c_ptr: int, stream=None) -> int:
    """Pruned DFT of a device field (device pointers) with no device allocation."""
    return lib().swkb_modes_noalloc(c_void_p(int(u_ptr)), int(n_fft), int(n_max),
                                    c_void_p(int(c_ptr)), stream)


def swkb_sym_eig(A, vectors=True):
    """Eigenpairs of real symmetric matrices (host arrays): A of shape
    (n, n) or (batch, n, n).  Returns (lam, V, sweeps): lam[..., j] in no
    particular order, row j of V[...] its unit eigenvector (None when
    vectors is False)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    single = A.ndim == 2
    if single:
        A = A[None]
    if A.ndim != 3 or A.shape[1] != A.shape[2]:
        raise ValueError("A must be (n, n) or (batch, n, n)")
    batch, n = A.shape[0], A.shape[1]
    lam = np.empty((batch, n))
    V = np.empty((batch, n, n)) if vectors else None
    sweeps = c_int32(0)
    check(lib().swkb_sym_eig(batch, n, A.ctypes.data_as(c_void_p), lam.ctypes.data_as(c_void_p),
                             V.ctypes.data_as(c_void_p) if vectors else None, byref(sweeps), 0,
                             None))
    if single:
        return lam[0], (V[0] if vectors else None), sweeps.value
    return lam, V, sweeps.value


def swkb_sym_eig_device(batch, n, a_ptr, lam_ptr, vec_ptr=None, stream=None) -> int:
    """Device-pointer form; returns the sweeps used."""
    sweeps = c_int32(0)
    check(lib().swkb_sym_eig(int(batch), int(n), c_void_p(int(a_ptr)), c_void_p(int(lam_ptr)),
                             c_void_p(int(vec_ptr)) if vec_ptr else None, byref(sweeps), 1,
                             stream))
    return sweeps.value


def hill_desc(bc, z_a, z_b, n_z, K, n_q, z_sym=0.0) -> swkb_hill_desc:
    return swkb_hill_desc(int(bc), float(z_a), float(z_b), float(z_sym), int(n_z), int(K),
                          int(n_q))


def hill_eigen_count(bc, K):
    return {SWKB_BC_NEUMANN: K + 1, SWKB_BC_DIRICHLET: K}.get(bc, 2 * K + 1)


def swkb_hill_propagate(desc: swkb_hill_desc, k, eps, u0, xs, eigenvalues=False):
    """Separation-of-variables fields (host arrays): k (batch,), eps
    (batch, n_q + 1), u0 (batch, n_z) complex, xs (n_x,) -> u (batch, n_x,
    n_z) complex [, eigenvalues (batch, n_eig)]."""
    k = np.ascontiguousarray(np.atleast_1d(k), dtype=np.float64)
    batch = len(k)
    eps = np.ascontiguousarray(eps, dtype=np.float64).reshape(batch, desc.n_q + 1)
    u0 = np.ascontiguousarray(u0, dtype=np.complex128).reshape(batch, desc.n_z)
    xs = np.ascontiguousarray(np.atleast_1d(xs), dtype=np.float64)
    out = np.empty((batch, len(xs), desc.n_z), np.complex128)
    lam = np.empty((batch, hill_eigen_count(desc.bc, desc.K))) if eigenvalues else None
    check(lib().swkb_hill_propagate(byref(desc), batch, k.ctypes.data_as(c_void_p),
                                    eps.ctypes.data_as(c_void_p), u0.ctypes.data_as(c_void_p),
                                    len(xs), xs.ctypes.data_as(c_void_p),
                                    out.ctypes.data_as(c_void_p),
                                    lam.ctypes.data_as(c_void_p) if eigenvalues else None, 0,
                                    None))
    return (out, lam) if eigenvalues else out


def swkb_hill_propagate_device(desc: swkb_hill_desc, k, eps_ptr, u0_ptr, xs, out_ptr,
                               lam_ptr=None, stream=None) -> int:
    """Device-pointer form (k and xs are host arrays)."""
    k = np.ascontiguousarray(np.atleast_1d(k), dtype=np.float64)
    xs = np.ascontiguousarray(np.atleast_1d(xs), dtype=np.float64)
    return check(lib().swkb_hill_propagate(byref(desc), len(k), k.ctypes.data_as(c_void_p),
                                           c_void_p(int(eps_ptr)), c_void_p(int(u0_ptr)),
                                           len(xs), xs.ctypes.data_as(c_void_p),
                                           c_void_p(int(out_ptr)),
                                           c_void_p(int(lam_ptr)) if lam_ptr else None, 1,
                                           stream))


def swkb_last_error() -> str:
    return lib().swkb_last_error().decode(errors="replace")


def swkb_server_create(hbm_budget_bytes, max_slots, queue_cap=0, device=0):
    handle = c_void_p()
    check(lib().swkb_server_create(int(hbm_budget_bytes), int(max_slots), int(queue_cap),
                                   int(device), byref(handle)))
    return handle


def swkb_submit(server, req: swkb_request) -> tuple[int, int]:
    """Returns (status, ticket); status SWKB_ERR_AGAIN when the queue is full."""
    t = c_uint64()
    st = lib().swkb_submit(server, byref(req), byref(t))
    return st, int(t.value)


def swkb_poll(server, ticket, u_out=None, timeout_ms=-1) -> int:
    ptr = u_out.ctypes.data_as(c_void_p) if u_out is not None else None
    return lib().swkb_poll(server, c_uint64(ticket), ptr, int(timeout_ms))


def swkb_cancel(server, ticket) -> int:
    return lib().swkb_cancel(server, c_uint64(ticket))


def swkb_server_get_stats(server) -> dict:
    st = swkb_server_stats()
    check(lib().swkb_server_get_stats(server, byref(st)))
    return {f: getattr(st, f) for f, _ in swkb_server_stats._fields_}


def swkb_server_destroy(server):
    lib().swkb_server_destroy(server)


# --------------------------------------------------------------------------
# convenience wrappers
# --------------------------------------------------------------------------
class Server:
    """Continuous-batching request server (one GPU)."""

    def __init__(self, hbm_budget_bytes, max_slots, queue_cap=0, device=0):
        self.handle = swkb_server_create(hbm_budget_bytes, max_slots, queue_cap, device)
        self.n_z = {}

    def submit(self, problem, precision=SWKB_FP64, u0=None, q0=0, n_screens=None):
        """Returns (status, ticket)."""
        keep = _Keep()
        prof = make_profile(problem.profile, keep)
        dom = swkb_domain(problem.z_a, problem.z_b, problem.x0, problem.bc)
        opt = options_for(problem, precision)
        u = np.ascontiguousarray(problem.u0 if u0 is None else u0, dtype=np.complex128)
        req = swkb_request(ctypes.pointer(prof), float(problem.k), ctypes.pointer(dom),
                           int(problem.n_z), float(problem.dx), ctypes.pointer(opt),
                           u.ctypes.data_as(POINTER(c_double)), int(q0),
                           int(problem.n_screens if n_screens is None else n_screens))
        st, t = swkb_submit(self.handle, req)
        if st == SWKB_OK:
            self.n_z[t] = problem.n_z
        return st, t

    def poll(self, ticket, timeout_ms=-1):
        """Returns (status, field or None)."""
        out = np.empty(self.n_z[ticket], np.complex128)
        st = swkb_poll(self.handle, ticket, out, timeout_ms)
        if st != SWKB_NOT_READY:
            self.n_z.pop(ticket, None)
        return st, (out if st == SWKB_OK else None)

    def cancel(self, ticket):
        return swkb_cancel(self.handle, ticket)

    def stats(self):
        return swkb_server_get_stats(self.handle)

    def close(self):
        if self.handle:
            swkb_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
def _request(problem, opt: swkb_options, keep: _Keep, u0=None, q0=0, n_screens=None):
    """swkb_request for a workloads.Problem (the buffers stay alive in keep)."""
    prof = make_profile(problem.profile, keep)
    dom = swkb_domain(problem.z_a, problem.z_b, problem.x0, problem.bc)
    u = np.ascontiguousarray(problem.u0 if u0 is None else u0, dtype=np.complex128)
    keep.refs.extend([prof, dom, opt, u])
    return swkb_request(ctypes.pointer(prof), float(problem.k), ctypes.pointer(dom),
                        int(problem.n_z), float(problem.dx), ctypes.pointer(opt),
                        u.ctypes.data_as(POINTER(c_double)), int(q0),
                        int(problem.n_screens if n_screens is None else n_screens))


class Batch:
    """Many problems advanced in one persistent launch (swkb_batch_*).
    problems: workloads.Problem list (each runs its own n_screens from its
    u0); precision shared by all; autotune / tiling as for Plan."""

    def __init__(self, problems, precision=SWKB_MIXED, ctas_per_sm=0, wait_limit_ms=0,
                 device=0, stream=None, autotune=False, tiling=None):
        keep = _Keep()
        n = len(problems)
        reqs = (swkb_request * n)()
        for i, pb in enumerate(problems):
            opt = options_for(pb, precision, None, device, autotune, False, 0, tiling)
            reqs[i] = _request(pb, opt, keep)
        bo = swkb_batch_options(int(ctas_per_sm), int(wait_limit_ms), int(device), stream)
        self.handle = c_void_p()
        check(lib().swkb_batch_create(n, reqs, byref(bo), byref(self.handle)))
        self.n_z = [int(pb.n_z) for pb in problems]
        self.offsets = np.concatenate([[0], np.cumsum(self.n_z)]).astype(np.int64)
        self.total = int(self.offsets[-1])
        self.info = swkb_batch_info()
        check(lib().swkb_batch_get_info(self.handle, byref(self.info)))

    def run(self, u_in=None):
        """Host arrays: returns the list of output fields (complex128)."""
        out = np.empty(self.total, np.complex128)
        src = None
        if u_in is not None:
            src = np.ascontiguousarray(np.concatenate(u_in), dtype=np.complex128)
        check(lib().swkb_batch_run(self.handle, None if src is None else src.ctypes.data,
                                   out.ctypes.data, 0))
        return [out[self.offsets[i]:self.offsets[i + 1]] for i in range(len(self.n_z))]

    def run_status(self):
        """Runs without reading the outputs; returns the status (no raise)."""
        return lib().swkb_batch_run(self.handle, None, None, 0)

    def run_device(self, in_ptr, out_ptr):
        """Device pointers (concatenated complex128 fields; in_ptr may be None)."""
        return check(lib().swkb_batch_run(self.handle, in_ptr, out_ptr, 1))

    def close(self):
        if self.handle:
            lib().swkb_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """A plan for one workloads.Problem (or equivalent fields)."""

    def __init__(self, problem, precision=SWKB_FP64, stream=None, device=0, autotune=False,
                 reuse_rays=False, planes=0, tiling=None):
        self.problem = problem
        dom = swkb_domain(problem.z_a, problem.z_b, problem.x0, problem.bc)
        self.options = options_for(problem, precision, stream, device, autotune, reuse_rays,
                                   planes, tiling)
        self.handle = swkb_plan_create(problem.profile, problem.k, dom, problem.n_z,
                                       problem.dx, self.options)
        self.info = swkb_plan_get_info(self.handle)
        self.n_z = problem.n_z

    def close(self):
        if self.handle:
            swkb_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def propagate(self, u0=None, q0=0, n_screens=None, snapshot_every=0):
        """Host arrays in and out (complex128)."""
        if u0 is None:
            u0 = self.problem.u0
        if n_screens is None:
            n_screens = self.problem.n_screens
        u0 = np.ascontiguousarray(u0, dtype=np.complex128)
        n_out = n_screens // snapshot_every if snapshot_every else 1
        out = np.empty(n_out * self.n_z, dtype=np.complex128)
        swkb_propagate(self.handle, u0, q0, n_screens, out, snapshot_every, 0)
        return out.reshape(n_out, self.n_z) if snapshot_every else out

    def propagate_device(self, u0_ptr: int, out_ptr: int, q0=0, n_screens=None, snapshot_every=0):
        if n_screens is None:
            n_screens = self.problem.n_screens
        return swkb_propagate(self.handle, u0_ptr, q0, n_screens, out_ptr, snapshot_every, 1)

    def propagate_planes(self, planes, u0=None, q0=0, n_screens=None):
        """Host arrays: (n_screens * planes, n_z) complex128 fields, rows
        ordered (screen, plane), the last of each screen being its field."""
        if u0 is None:
            u0 = self.problem.u0
        if n_screens is None:
            n_screens = self.problem.n_screens
        u0 = np.ascontiguousarray(u0, dtype=np.complex128)
        out = np.empty(n_screens * planes * self.n_z, dtype=np.complex128)
        swkb_propagate_planes(self.handle, u0, q0, n_screens, planes, out, 0)
        return out.reshape(n_screens * planes, self.n_z)

    def propagate_planes_device(self, planes, u0_ptr: int, out_ptr: int, q0=0, n_screens=None):
        if n_screens is None:
            n_screens = self.problem.n_screens
        return swkb_propagate_planes(self.handle, u0_ptr, q0, n_screens, planes, out_ptr, 1)

    def set_timing(self, kinds=True, every=1, serial=False):
        swkb_plan_set_timing(self.handle, kinds, every, serial)

    def stats(self) -> dict:
        return swkb_plan_get_stats(self.handle)

    def debug_screen(self, q, u_full):
        i = self.info
        u_full = np.ascontiguousarray(u_full, dtype=np.complex128)
        c = np.empty(i.n_modes, np.complex128)
        shape = (i.n_modes, i.n_rays_total)
        delta = np.empty(shape)
        r = np.empty(shape)
        a = np.empty(shape)
        un = np.empty(i.n_fft, np.complex128)
        check(lib().swkb_debug_screen(self.handle, int(q), u_full.ctypes.data_as(c_void_p),
                                      c.ctypes.data_as(c_void_p), delta.ctypes.data_as(c_void_p),
                                      r.ctypes.data_as(c_void_p), a.ctypes.data_as(c_void_p),
                                      un.ctypes.data_as(c_void_p)))
        return dict(c=c, delta=delta, r=r, a=a, u_next=un)
