"""Thin ctypes binding of liblbm.so (include/lbm.h).

Argument marshalling only: every step of the solver runs in the CUDA library.  The
module-level functions carry the C names (``lbm_create``, ``lbm_step``, ...); ``Solver``
bundles them for convenience.  Arrays may be numpy arrays (host) or torch tensors (host
or CUDA); they are passed to the library by pointer.  The library is required: importing
works without it, but the first call raises if ``liblbm.so`` has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "liblbm.so")
_lib = None

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ESTATE = 0, -1, -2, -3, -4, -5, -6
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}
FACE = {"periodic": 0, "noslip": 1, "inlet": 2, "outlet": 3, "freeslip": 4}
COLLISION = {"acm": 0, "bgk": 1, "raw": 2}
KERNEL_KINDS = ("step", "band", "interp", "spread", "boundary", "other", "tracer", "motion")


class LBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lbm error {code}: {msg}")
        self.code = code


class lbm_config(C.Structure):
    _fields_ = [("storage", C.c_int), ("face_type", C.c_int * 6), ("rho0", C.c_double), ("u_in", C.c_double),
                ("inlet_noise", C.c_double), ("seed", C.c_ulonglong), ("inflow_coef", C.c_double * 16),
                ("omega_bulk", C.c_double), ("omega_hi", C.c_double * 4), ("cuda_stream", C.c_void_p),
                ("collision", C.c_int)]


class lbm_motion(C.Structure):
    _fields_ = [("center", C.c_double * 3), ("velocity", C.c_double * 3), ("axis", C.c_double * 3),
                ("omega", C.c_double)]


class lbm_emitter(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3), ("seed", C.c_ulonglong)]


class lbm_loss(C.Structure):
    _fields_ = [("w_drag", C.c_double), ("w_ke", C.c_double), ("ke_x0", C.c_int), ("ke_x1", C.c_int)]


_SIGS = {
    "lbm_config_default": (None, [C.POINTER(lbm_config)]),
    "lbm_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.c_double,
                             C.POINTER(C.c_double), C.POINTER(lbm_config)]),
    "lbm_destroy": (C.c_int, [C.c_void_p]),
    "lbm_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_set_solids": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p, C.c_void_p]),
    "lbm_step": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_macroscopic": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_set_state_async": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_macroscopic_async": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_reductions": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "lbm_ib_forces": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_populations": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_velocity": (C.c_int, [C.c_int, C.POINTER(C.c_int)]),
    "lbm_time": (C.c_longlong, [C.c_void_p]),
    "lbm_check": (C.c_int, [C.c_void_p]),
    "lbm_synchronize": (C.c_int, [C.c_void_p, C.c_double]),
    "lbm_save": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t)]),
    "lbm_load": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "lbm_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_kernel_times": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "lbm_band_size": (C.c_longlong, [C.c_void_p]),
    "lbm_set_pair_kernel": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_solid_count": (C.c_longlong, [C.c_void_p]),
    "lbm_dims": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "lbm_set_inflow": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "lbm_set_motion": (C.c_int, [C.c_void_p, C.POINTER(lbm_motion)]),
    "lbm_solid_samples": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_solid_torque": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "lbm_set_tracers": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, C.POINTER(lbm_emitter)]),
    "lbm_tracer_count": (C.c_longlong, [C.c_void_p]),
    "lbm_tracers": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_tracer_dims": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "lbm_tracer_density": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "lbm_adjoint": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(lbm_loss), C.POINTER(C.c_double),
                              C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "lbm_sum_forces_static": (C.c_int, [C.c_void_p, C.c_longlong, C.c_void_p, C.c_void_p]),
    "lbm_last_error": (C.c_char_p, [C.c_void_p]),
}


def library(path: str | None = None):
    """Load liblbm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        p = path or _LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        lib = C.CDLL(p)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc, ctx=None):
    if rc != LBM_OK:
        msg = library().lbm_last_error(ctx)
        raise LBMError(rc, msg.decode() if msg else "")


def _ptr(a):
    """(pointer, keepalive) of a float32 array: numpy (host) or torch tensor (host or CUDA)."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):           # torch tensor
        import torch
        t = a.detach()
        if t.dtype != torch.float32 or not t.is_contiguous():
            t = t.to(torch.float32).contiguous()
        return C.c_void_p(t.data_ptr()), t
    arr = np.ascontiguousarray(a, dtype=np.float32)
    return C.c_void_p(arr.ctypes.data), arr


def _ptr_out(a, n, what):
    """Pointer of an output buffer the library fills with n float32 values: a C-contiguous
    float32 numpy array or torch tensor of at least n elements, passed as is.  Anything else
    is refused: the library would fill a converted temporary and the caller's array would keep
    stale data, or write past a short buffer."""
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float32 or not a.is_contiguous():
            raise ValueError(f"{what}: the output must be a contiguous float32 tensor")
        if a.numel() < n:
            raise ValueError(f"{what}: the output holds {a.numel()} values, {n} are written")
        return C.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"] or not a.flags["WRITEABLE"]:
        raise ValueError(f"{what}: the output must be a writeable C-contiguous float32 numpy array")
    if a.size < n:
        raise ValueError(f"{what}: the output holds {a.size} values, {n} are written")
    return C.c_void_p(a.ctypes.data)


def _ptr_nocopy(a):
    """Pointer of a float32 array that the library may read or write after the call returns
    (asynchronous transfers): a C-contiguous float32 numpy array or torch tensor, passed as is;
    anything that would need a converted temporary is refused."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float32 or not a.is_contiguous():
            raise ValueError("asynchronous transfers need a contiguous float32 tensor")
        return C.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("asynchronous transfers need a C-contiguous float32 numpy array")
    return C.c_void_p(a.ctypes.data)


# ---- the C functions under their own names -------------------------------------------

def lbm_config_default() -> lbm_config:
    cfg = lbm_config()
    library().lbm_config_default(C.byref(cfg))
    return cfg


def lbm_create(nx, ny, nz, nu, forcing=(0.0, 0.0, 0.0), cfg: lbm_config | None = None):
    h = C.c_void_p()
    f = (C.c_double * 3)(*forcing)
    _check(library().lbm_create(C.byref(h), nx, ny, nz, nu, f, C.byref(cfg) if cfg is not None else None))
    return h


def lbm_destroy(h):
    return library().lbm_destroy(h)


def lbm_set_state(h, rho, u):
    pr, kr = _ptr(rho)
    pu, ku = _ptr(u)
    _check(library().lbm_set_state(h, pr, pu), h)


def lbm_set_solids(h, samples, area=None, u_b=None):
    count = 0 if samples is None else int(np.prod(samples.shape) // 3)
    ps, ks = _ptr(samples)
    pa, ka = _ptr(area)
    pb, kb = _ptr(u_b)
    _check(library().lbm_set_solids(h, ps, count, pa, pb), h)


def lbm_step(h, n=1):
    _check(library().lbm_step(h, int(n)), h)


def lbm_macroscopic(h, rho, u):
    """Fill rho (N) and u (3 N) (either may be None) with the fields of the last collision."""
    N = _cells(h)
    pr = _ptr_out(rho, N, "lbm_macroscopic rho") if rho is not None else None
    pu = _ptr_out(u, 3 * N, "lbm_macroscopic u") if u is not None else None
    _check(library().lbm_macroscopic(h, pr, pu), h)


def lbm_set_state_async(h, rho, u):
    """The caller keeps rho and u alive and unchanged until lbm_synchronize returns."""
    _check(library().lbm_set_state_async(h, _ptr_nocopy(rho), _ptr_nocopy(u)), h)


def lbm_macroscopic_async(h, rho, u):
    """rho and u (either may be None) are filled when lbm_synchronize returns."""
    _check(library().lbm_macroscopic_async(h, _ptr_nocopy(rho), _ptr_nocopy(u)), h)


def lbm_reductions(h):
    m = C.c_double()
    mom = (C.c_double * 3)()
    drag = (C.c_double * 3)()
    _check(library().lbm_reductions(h, C.byref(m), mom, drag), h)
    return m.value, np.array(mom[:]), np.array(drag[:])


def lbm_ib_forces(h, out):
    """Fill out (S, 3) with the penalty forces of the last step, S = lbm_solid_count(h)."""
    _check(library().lbm_ib_forces(h, _ptr_out(out, 3 * lbm_solid_count(h), "lbm_ib_forces")), h)


def lbm_populations(h, out):
    """Fill out (27, N) with the post-collision populations of the current time."""
    _check(library().lbm_populations(h, _ptr_out(out, 27 * _cells(h), "lbm_populations")), h)


def lbm_velocity(i):
    c = (C.c_int * 3)()
    _check(library().lbm_velocity(i, c))
    return tuple(c[:])


def lbm_time(h):
    return library().lbm_time(h)


def lbm_check(h):
    return library().lbm_check(h)


def lbm_synchronize(h, timeout_s=0.0):
    _check(library().lbm_synchronize(h, timeout_s), h)


def lbm_save(h) -> bytes:
    n = C.c_size_t(0)
    _check(library().lbm_save(h, None, C.byref(n)), h)
    buf = C.create_string_buffer(n.value)
    _check(library().lbm_save(h, buf, C.byref(n)), h)
    return buf.raw[: n.value]


def lbm_load(h, data: bytes):
    _check(library().lbm_load(h, data, len(data)), h)


def lbm_profile(h, enable=True):
    _check(library().lbm_profile(h, 1 if enable else 0), h)


def lbm_kernel_times(h):
    ms = (C.c_double * len(KERNEL_KINDS))()
    n = (C.c_longlong * len(KERNEL_KINDS))()
    _check(library().lbm_kernel_times(h, ms, n), h)
    return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_KINDS)}


def lbm_band_size(h):
    return library().lbm_band_size(h)


def lbm_set_pair_kernel(h, bulk):
    """bulk: False / 0 (pair kernel), True / 1 (tensor-copy fed kernel), 2 (its wait-limit self-test)."""
    _check(library().lbm_set_pair_kernel(h, int(bulk)), h)


def lbm_solid_count(h):
    return library().lbm_solid_count(h)


def lbm_dims(h):
    d = (C.c_int * 3)()
    _check(library().lbm_dims(h, d), h)
    return tuple(d[:])


def _cells(h):
    nx, ny, nz = lbm_dims(h)
    return nx * ny * nz


def lbm_set_inflow(h, coef):
    c = (C.c_double * 16)(*[float(v) for v in np.asarray(coef, dtype=np.float64).ravel()])
    _check(library().lbm_set_inflow(h, c), h)


def lbm_set_motion(h, motion=None):
    """motion = (center, velocity, axis, omega) or None (stop)."""
    m = None
    if motion is not None:
        c, v, a, w = motion
        m = lbm_motion((C.c_double * 3)(*c), (C.c_double * 3)(*v), (C.c_double * 3)(*a), float(w))
    _check(library().lbm_set_motion(h, C.byref(m) if m is not None else None), h)


def lbm_solid_samples(h, out):
    _check(library().lbm_solid_samples(h, _ptr_out(out, 3 * lbm_solid_count(h), "lbm_solid_samples")), h)


def lbm_solid_torque(h, center=None):
    t = (C.c_double * 3)()
    c = (C.c_double * 3)(*center) if center is not None else None
    _check(library().lbm_solid_torque(h, c, t), h)
    return np.array(t[:])


def lbm_set_tracers(h, X, emitter=None):
    """X: (count, 3) positions (numpy or torch); emitter = (lo, hi, seed) or None."""
    count = 0 if X is None else int(np.prod(X.shape) // 3)
    px, kx = _ptr(X) if count else (None, None)
    em = None
    if emitter is not None:
        lo, hi, seed = emitter
        em = lbm_emitter((C.c_double * 3)(*lo), (C.c_double * 3)(*hi), int(seed))
    _check(library().lbm_set_tracers(h, px, count, C.byref(em) if em is not None else None), h)


def lbm_tracer_count(h):
    return library().lbm_tracer_count(h)


def lbm_tracers(h, out):
    _check(library().lbm_tracers(h, _ptr_out(out, 3 * lbm_tracer_count(h), "lbm_tracers")), h)


def lbm_tracer_dims(h, s):
    d = (C.c_int * 3)()
    _check(library().lbm_tracer_dims(h, int(s), d), h)
    return tuple(d[:])


def lbm_tracer_density(h, s, out):
    gx, gy, gz = lbm_tracer_dims(h, s)
    _check(library().lbm_tracer_density(h, int(s), _ptr_out(out, gx * gy * gz, "lbm_tracer_density")), h)


def lbm_adjoint(h, n, K, w_drag=1.0, w_ke=0.0, ke_x0=0, ke_x1=0, count=None):
    """Run n steps with the adjoint; returns (L, dL/d inflow coefficients (16,), dL/dX (S, 3)),
    S = lbm_solid_count(h).  ``count``, when given, must equal S (a check of the caller's
    sample count; the library writes 3 S position gradients)."""
    S = lbm_solid_count(h)
    if count is not None and int(count) != S:
        raise ValueError(f"lbm_adjoint: count {count} differs from the context's {S} samples")
    loss = lbm_loss(w_drag, w_ke, ke_x0, ke_x1)
    dinf = (C.c_double * 16)()
    dpos = (C.c_double * (3 * S))() if S > 0 else None
    L = C.c_double()
    _check(library().lbm_adjoint(h, int(n), int(K), C.byref(loss), dinf, dpos, C.byref(L)), h)
    grad_X = np.array(dpos[:]).reshape(S, 3) if S > 0 else np.zeros((0, 3))
    return L.value, np.array(dinf[:]), grad_X


def lbm_sum_forces_static(g, out, stream=None):
    """Allocation-free FP64 sum of per-sample forces: g (S, 3) contiguous float32 CUDA tensor,
    out contiguous float64 CUDA tensor of at least 3 values, both on the current device;
    launched on ``stream`` (default: torch's current stream)."""
    import torch
    if not (isinstance(g, torch.Tensor) and isinstance(out, torch.Tensor)):
        raise ValueError("lbm_sum_forces_static: g and out must be torch tensors")
    if g.dtype != torch.float32 or not g.is_contiguous() or g.dim() != 2 or g.shape[1] != 3:
        raise ValueError(f"lbm_sum_forces_static: g must be a contiguous float32 (S, 3) tensor, got "
                         f"{tuple(g.shape)} {g.dtype}")
    if out.dtype != torch.float64 or not out.is_contiguous() or out.numel() < 3:
        raise ValueError("lbm_sum_forces_static: out must be a contiguous float64 tensor of at least 3 values")
    if not (g.is_cuda and out.is_cuda):
        raise ValueError("lbm_sum_forces_static: g and out must be CUDA tensors")
    dev = torch.cuda.current_device()
    if g.device.index != dev or out.device.index != dev:
        raise ValueError("lbm_sum_forces_static: g and out must be on the current CUDA device")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    count = g.shape[0]
    rc = library().lbm_sum_forces_static(C.c_void_p(g.data_ptr()) if count else None, count,
                                         C.c_void_p(out.data_ptr()), C.c_void_p(stream))
    if rc != LBM_OK:
        raise LBMError(rc, f"lbm_sum_forces_static failed for {count} samples")


# ---- convenience wrapper -----------------------------------------------------------

class Solver:
    """One simulation on the current CUDA device (see include/lbm.h)."""

    def __init__(self, nx, ny, nz, nu, forcing=(0.0, 0.0, 0.0), storage="f32", faces=("periodic",) * 6,
                 rho0=1.0, u_in=0.0, noise=0.0, seed=2101, inflow_coef=None, omega_bulk=1.0,
                 omega_hi=(1.0, 1.0, 1.0, 1.0), stream=None, collision="acm"):
        cfg = lbm_config_default()
        cfg.storage = STORAGE[storage]
        cfg.collision = COLLISION[collision]
        for k, t in enumerate(faces):
            cfg.face_type[k] = FACE[t]
        cfg.rho0, cfg.u_in, cfg.inlet_noise, cfg.seed = rho0, u_in, noise, seed
        if inflow_coef is not None:
            for k, v in enumerate(np.asarray(inflow_coef, dtype=np.float64).ravel()):
                cfg.inflow_coef[k] = float(v)
        cfg.omega_bulk = omega_bulk
        for k in range(4):
            cfg.omega_hi[k] = omega_hi[k]
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                stream = None
        cfg.cuda_stream = stream
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.h = lbm_create(nx, ny, nz, nu, forcing, cfg)

    def close(self):
        if self.h:
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, rho, u):
        lbm_set_state(self.h, rho, u)

    def set_solids(self, X, area=None, u_b=None):
        lbm_set_solids(self.h, X, area, u_b)

    def step(self, n=1):
        lbm_step(self.h, n)

    def set_pair_kernel(self, bulk):
        """16-bit storage: main range in the tensor-copy fed kernel (True) or one pair per thread (False, default)."""
        lbm_set_pair_kernel(self.h, bulk)

    def macroscopic(self):
        """(rho (nz, ny, nx), u (3, nz, ny, nx)) as float32 numpy arrays."""
        rho = np.empty(self.shape, np.float32)
        u = np.empty((3,) + self.shape, np.float32)
        lbm_macroscopic(self.h, rho, u)
        return rho, u

    def set_state_async(self, rho, u):
        """Queue the upload and initialisation (keep rho, u unchanged until synchronize)."""
        lbm_set_state_async(self.h, rho, u)

    def macroscopic_async(self, rho, u):
        """Queue the moments and their copy into rho, u (filled at synchronize)."""
        lbm_macroscopic_async(self.h, rho, u)

    def synchronize(self, timeout_s=0.0):
        lbm_synchronize(self.h, timeout_s)

    def reductions(self):
        return lbm_reductions(self.h)

    def set_motion(self, motion=None):
        lbm_set_motion(self.h, motion)

    def solid_samples(self, count=None):
        """Current sample positions (S, 3), in the order given to set_solids."""
        S = lbm_solid_count(self.h)
        if count is not None and int(count) != S:
            raise ValueError(f"solid_samples: count {count} differs from the context's {S} samples")
        out = np.empty((S, 3), np.float32)
        lbm_solid_samples(self.h, out)
        return out

    def torque(self, center=None):
        return lbm_solid_torque(self.h, center)

    def set_tracers(self, X, emitter=None):
        lbm_set_tracers(self.h, X, emitter)

    def tracers(self):
        """Tracer positions (count, 3) as a float32 numpy array."""
        out = np.empty((lbm_tracer_count(self.h), 3), np.float32)
        if out.shape[0]:
            lbm_tracers(self.h, out)
        return out

    def tracer_density(self, s=1):
        """Cloud-in-cell tracer density on the grid of spacing s, (gz, gy, gx) float32."""
        gx, gy, gz = lbm_tracer_dims(self.h, s)
        out = np.empty((gz, gy, gx), np.float32)
        lbm_tracer_density(self.h, s, out)
        return out

    def ib_forces(self, count=None):
        """Penalty forces (S, 3) of the last step, in the order given to set_solids."""
        S = lbm_solid_count(self.h)
        if count is not None and int(count) != S:
            raise ValueError(f"ib_forces: count {count} differs from the context's {S} samples")
        g = np.empty((S, 3), np.float32)
        lbm_ib_forces(self.h, g)
        return g

    def populations(self):
        f = np.empty((27,) + self.shape, np.float32)
        lbm_populations(self.h, f)
        return f

    def adjoint(self, n, K=20, w_drag=1.0, w_ke=0.0, ke_x0=0, ke_x1=0, count=None):
        return lbm_adjoint(self.h, n, K, w_drag, w_ke, ke_x0, ke_x1, count)

    def set_inflow(self, coef):
        lbm_set_inflow(self.h, coef)

    @property
    def time(self):
        return lbm_time(self.h)


# ---- autograd ------------------------------------------------------------------------

def _autograd_function():
    import torch

    class LBMSolve(torch.autograd.Function):
        """L(a, X) of n solver steps as a differentiable function of the 16 inflow coefficients a
        and the sample positions X (count, 3).  forward sets a, the samples and the initial
        state (rho0, u0), then runs lbm_adjoint (n steps with checkpoints every K, loss and
        both gradients in one pass); backward returns grad_L times the stored gradients.
        The solver must have an inlet on -x and is left at the state after the n steps."""

        @staticmethod
        def forward(ctx, coef, X, solver, rho0, u0, n, K, w_drag, w_ke, ke_x0, ke_x1, area):
            solver.set_inflow(coef.detach().double().cpu().numpy())
            Xf = X.detach().to(torch.float32).contiguous()
            solver.set_solids(Xf, area)
            solver.set_state(rho0, u0)
            L, dcoef, dpos = solver.adjoint(n, K, w_drag, w_ke, ke_x0, ke_x1, Xf.shape[0])
            ctx.save_for_backward(torch.as_tensor(dcoef, dtype=coef.dtype, device=coef.device),
                                  torch.as_tensor(dpos, dtype=X.dtype, device=X.device))
            return torch.tensor(L, dtype=torch.float64, device=coef.device)

        @staticmethod
        def backward(ctx, grad_L):
            dcoef, dpos = ctx.saved_tensors
            g = grad_L.to(torch.float64)
            return ((g * dcoef.double()).to(dcoef.dtype), (g * dpos.double()).to(dpos.dtype),
                    None, None, None, None, None, None, None, None, None, None)

    return LBMSolve


_LBMSolve = None


def LBMSolve():
    """The torch.autograd.Function class (created on first use, so importing this module does
    not import torch)."""
    global _LBMSolve
    if _LBMSolve is None:
        _LBMSolve = _autograd_function()
    return _LBMSolve


def lbm_solve(coef, X, solver, rho0, u0, n, K=20, w_drag=1.0, w_ke=0.0, ke_x0=0, ke_x1=0, area=None):
    """Differentiable loss of n steps (see LBMSolve): coef (16,) and X (count, 3) torch tensors."""
    return LBMSolve().apply(coef, X, solver, rho0, u0, n, K, w_drag, w_ke, ke_x0, ke_x1, area)
