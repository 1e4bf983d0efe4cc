"""ctypes binding of ``liblbm_gb300.so``: argument marshalling only.

Every function carries the name of the C entry point it calls (see
``include/lbm.h`` for argument meaning, layout, ownership and errors) and
raises :class:`LbmError` on a non-zero status.  All arithmetic of the method
runs inside the CUDA library; nothing here computes on the fields.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

c_int, c_double, c_void_p, c_size_t = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
c_float_p = ctypes.POINTER(ctypes.c_float)

LBM_D2Q9, LBM_D3Q19, LBM_D3Q15 = 0, 1, 2
LBM_PERIODIC_X, LBM_PERIODIC_Y, LBM_PERIODIC_Z = 1, 2, 4
LBM_STORE_G_F16 = 1
STATUS = {0: "LBM_OK", -1: "LBM_EINVAL", -2: "LBM_ENOMEM", -3: "LBM_ECUDA", -4: "LBM_EDIVERGED",
          -5: "LBM_ETIMEOUT", -6: "LBM_ESTATE", -7: "LBM_EUNSUPPORTED"}

# every symbol include/lbm.h declares
EXPORTS = [
    "lbm_default_params", "lbm_create", "lbm_create_batch", "lbm_create_ex", "lbm_create_multi",
    "lbm_get_instance_shape", "lbm_tune", "lbm_destroy", "lbm_set_stream",
    "lbm_set_launch", "lbm_set_solid", "lbm_set_solid_device", "lbm_set_phase", "lbm_set_phase_device",
    "lbm_step", "lbm_sync", "lbm_get_fields", "lbm_get_populations", "lbm_get_state", "lbm_set_state",
    "lbm_observables", "lbm_contact_angle", "lbm_get_shape", "lbm_strerror", "lbm_last_error", "lbm_set_profiling", "lbm_kernel_time", "lbm_kernel_time_split", "lbm_observables_noalloc", "lbm_set_inout",
    "lbm_phase_flux", "lbm_create_alloc", "lbm_set_wait_limit", "lbm_derive",
]

# device-memory callbacks of lbm_create_alloc
lbm_alloc_fn = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
lbm_free_fn = ctypes.CFUNCTYPE(None, c_void_p, c_size_t, c_void_p, c_void_p)


class lbm_params(ctypes.Structure):
    _fields_ = [("W", c_double), ("M_deg", c_double), ("M_cst", c_double), ("theta_deg", c_double),
                ("kappa", c_double), ("sigma", c_double), ("rho", c_double * 3), ("mu", c_double * 3),
                ("d0", c_double), ("eta_hat", c_double), ("s_free_ch", c_double), ("s_free_ns", c_double),
                ("body_force", c_double * 3)]


class lbm_derived(ctypes.Structure):
    _fields_ = [("k", c_double), ("gamma", c_double * 3), ("gamma_T", c_double), ("eta", c_double),
                ("s1_ch", c_double), ("cs2", c_double), ("w", c_double * 3), ("visc", c_double * 2),
                ("p_f", c_double), ("p_w", c_double), ("p_K", c_double), ("p_h", c_double * 3)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


class lbm_obs(ctypes.Structure):
    _fields_ = [("mass1", c_double), ("mass0", c_double), ("umax", c_double), ("p_in", c_double),
                ("p_out", c_double), ("dp", c_double), ("n_in", ctypes.c_int64), ("n_out", ctypes.c_int64),
                ("step", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lbm_flux(ctypes.Structure):
    _fields_ = [("q1", c_double), ("q2", c_double), ("q", c_double), ("s1", c_double), ("s2", c_double),
                ("n_pore", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LbmError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({detail})")


_LIB = None


def library():
    """Load the shared library; raise if it has not been built (no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB):
        raise RuntimeError(f"{LIB} is missing: build it with __graft_entry__.build() "
                           "(the CUDA library is the only implementation)")
    lib = ctypes.CDLL(LIB)
    P = c_void_p
    sig = {
        "lbm_default_params": (c_int, [ctypes.POINTER(lbm_params)]),
        "lbm_create": (c_int, [c_int, c_int, c_int, c_int, c_int, ctypes.POINTER(lbm_params), ctypes.POINTER(P)]),
        "lbm_create_batch": (c_int, [c_int, c_int, c_int, c_int, c_int, c_int, ctypes.POINTER(lbm_params),
                                     ctypes.POINTER(P)]),
        "lbm_create_ex": (c_int, [c_int, c_int, c_int, c_int, c_int, c_int, ctypes.POINTER(lbm_params), c_int,
                                  ctypes.POINTER(P)]),
        "lbm_create_multi": (c_int, [c_int, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int), c_int,
                                     ctypes.POINTER(lbm_params), c_int, ctypes.POINTER(P)]),
        "lbm_get_instance_shape": (c_int, [P, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                           ctypes.POINTER(ctypes.c_int64)]),
        "lbm_tune": (c_int, [P, c_int, ctypes.POINTER(c_int)]),
        "lbm_destroy": (None, [P]),
        "lbm_set_stream": (c_int, [P, P]),
        "lbm_set_launch": (c_int, [P, c_int, c_int]),
        "lbm_set_wait_limit": (c_int, [P, c_int]),
        "lbm_derive": (c_int, [c_int, ctypes.POINTER(lbm_params), ctypes.POINTER(lbm_derived)]),
        "lbm_set_solid": (c_int, [P, c_float_p]),
        "lbm_set_solid_device": (c_int, [P, P]),
        "lbm_set_phase": (c_int, [P, c_float_p]),
        "lbm_set_phase_device": (c_int, [P, P]),
        "lbm_step": (c_int, [P, c_int]),
        "lbm_set_inout": (c_int, [P, c_int, c_float_p, c_double, c_double]),
        "lbm_phase_flux": (c_int, [P, c_int, c_int, ctypes.POINTER(lbm_flux)]),
        "lbm_create_alloc": (c_int, [c_int, c_int, c_int, c_int, c_int, c_int, ctypes.POINTER(lbm_params), c_int, P,
                                     lbm_alloc_fn, lbm_free_fn, P, ctypes.POINTER(P)]),
        "lbm_sync": (c_int, [P]),
        "lbm_get_fields": (c_int, [P, c_float_p, c_float_p, c_float_p]),
        "lbm_get_populations": (c_int, [P, c_float_p, c_float_p]),
        "lbm_get_state": (c_int, [P, P, ctypes.POINTER(c_size_t)]),
        "lbm_set_state": (c_int, [P, P, c_size_t]),
        "lbm_observables": (c_int, [P, c_int, ctypes.POINTER(lbm_obs)]),
        "lbm_contact_angle": (c_int, [P, c_int, c_int, c_int, c_double, c_double, ctypes.POINTER(c_double),
                                      ctypes.POINTER(c_double)]),
        "lbm_get_shape": (c_int, [P] + [ctypes.POINTER(c_int)] * 5),
        "lbm_strerror": (ctypes.c_char_p, [c_int]),
        "lbm_set_profiling": (c_int, [P, c_int]),
        "lbm_observables_noalloc": (c_int, [P, P, P, c_int, P, ctypes.c_longlong, P, P]),
        "lbm_kernel_time": (c_int, [P, ctypes.POINTER(c_double), ctypes.POINTER(ctypes.c_int64)]),
        "lbm_kernel_time_split": (c_int, [P, ctypes.POINTER(c_double), ctypes.POINTER(ctypes.c_int64)]),
        "lbm_last_error": (ctypes.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(status, where, ctx=None):
    if status != 0:
        detail = library().lbm_last_error(ctx)
        raise LbmError(status, where, detail.decode() if detail else "")


def _fptr(a):
    return a.ctypes.data_as(c_float_p)


def _f32(a, n):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def lbm_default_params(**overrides) -> lbm_params:
    p = lbm_params()
    _check(library().lbm_default_params(ctypes.byref(p)), "lbm_default_params")
    for k, v in overrides.items():
        if k in ("rho", "mu", "body_force"):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(p, k, v)
    return p


def lbm_create(lattice, nx, ny, nz, periodic_mask, params: lbm_params):
    out = c_void_p()
    _check(library().lbm_create(lattice, nx, ny, nz, periodic_mask, ctypes.byref(params), ctypes.byref(out)),
           "lbm_create")
    return out


def lbm_create_batch(lattice, nx, ny, nz, periodic_mask, params_list):
    arr = (lbm_params * len(params_list))(*params_list)
    out = c_void_p()
    _check(library().lbm_create_batch(lattice, nx, ny, nz, periodic_mask, len(params_list), arr,
                                      ctypes.byref(out)), "lbm_create_batch")
    return out


def lbm_create_ex(lattice, nx, ny, nz, periodic_mask, params_list, flags):
    arr = (lbm_params * len(params_list))(*params_list)
    out = c_void_p()
    _check(library().lbm_create_ex(lattice, nx, ny, nz, periodic_mask, len(params_list), arr, flags,
                                   ctypes.byref(out)), "lbm_create_ex")
    return out


def lbm_create_alloc(lattice, nx, ny, nz, periodic_mask, params_list, flags, stream, allocator):
    arr = (lbm_params * len(params_list))(*params_list)
    out = c_void_p()
    _check(library().lbm_create_alloc(lattice, nx, ny, nz, periodic_mask, len(params_list), arr, flags, stream,
                                      allocator.alloc, allocator.free, None, ctypes.byref(out)), "lbm_create_alloc")
    return out


class TorchAllocator:
    """Device memory of a context from PyTorch's caching allocator (lbm_create_alloc callbacks).

    Keep the object alive as long as the context: the context holds the C callbacks it wraps."""

    def __init__(self):
        import torch
        self._torch = torch

        def _alloc(nbytes, stream, user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0)))
            except Exception:        # reported by the library as LBM_ENOMEM
                return None

        def _free(ptr, nbytes, stream, user):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = lbm_alloc_fn(_alloc)
        self.free = lbm_free_fn(_free)


def lbm_create_multi(lattice, sizes, periodic_mask, params_list, flags=0):
    n = len(sizes)
    nx = (c_int * n)(*[int(a) for a, _ in sizes])
    ny = (c_int * n)(*[int(b) for _, b in sizes])
    arr = (lbm_params * n)(*params_list)
    out = c_void_p()
    _check(library().lbm_create_multi(lattice, n, nx, ny, periodic_mask, arr, flags, ctypes.byref(out)),
           "lbm_create_multi")
    return out


def lbm_get_instance_shape(ctx, instance):
    nx, ny, off = c_int(), c_int(), ctypes.c_int64()
    _check(library().lbm_get_instance_shape(ctx, instance, ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(off)),
           "lbm_get_instance_shape", ctx)
    return nx.value, ny.value, off.value


def lbm_tune(ctx, trial, nbatch):
    out = (c_int * nbatch)()
    _check(library().lbm_tune(ctx, trial, out), "lbm_tune", ctx)
    return list(out)


def lbm_destroy(ctx):
    library().lbm_destroy(ctx)


def lbm_set_stream(ctx, stream_handle):
    _check(library().lbm_set_stream(ctx, c_void_p(stream_handle)), "lbm_set_stream", ctx)


def lbm_set_launch(ctx, strip, depth=0):
    _check(library().lbm_set_launch(ctx, strip, depth), "lbm_set_launch", ctx)


def lbm_derive(lattice, params: lbm_params) -> dict:
    """The float64 constants a context with these parameters would use (host only)."""
    out = lbm_derived()
    _check(library().lbm_derive(lattice, ctypes.byref(params), ctypes.byref(out)), "lbm_derive")
    return out.as_dict()


def lbm_set_wait_limit(ctx, polls):
    _check(library().lbm_set_wait_limit(ctx, int(polls)), "lbm_set_wait_limit", ctx)


def lbm_get_shape(ctx):
    v = [c_int() for _ in range(5)]
    _check(library().lbm_get_shape(ctx, *[ctypes.byref(x) for x in v]), "lbm_get_shape", ctx)
    return tuple(x.value for x in v)   # nx, ny, nz, nbatch, q


def _nodes(ctx):
    nx, ny, nz, nb, q = lbm_get_shape(ctx)
    return nx * ny * nz, nb, q


def lbm_set_solid(ctx, phi0):
    n, nb, _ = _nodes(ctx)
    a = _f32(phi0, n * nb)
    _check(library().lbm_set_solid(ctx, _fptr(a)), "lbm_set_solid", ctx)


def lbm_set_solid_device(ctx, dev_ptr):
    _check(library().lbm_set_solid_device(ctx, c_void_p(dev_ptr)), "lbm_set_solid_device", ctx)


def lbm_set_phase(ctx, phi1):
    n, nb, _ = _nodes(ctx)
    a = _f32(phi1, n * nb)
    _check(library().lbm_set_phase(ctx, _fptr(a)), "lbm_set_phase", ctx)


def lbm_set_phase_device(ctx, dev_ptr):
    _check(library().lbm_set_phase_device(ctx, c_void_p(dev_ptr)), "lbm_set_phase_device", ctx)


def lbm_set_inout(ctx, mode, u_in=None, phi_in=-1.0, p_out=0.0):
    """mode bit 0: velocity inlet at x = 0 (u_in: [d][nz][ny] or [d][ny]); bit 1: pressure outlet at x = nx - 1."""
    nx, ny, nz, nb, q = lbm_get_shape(ctx)
    d = 2 if q == 9 else 3
    ptr = None
    if mode & 1:
        a = _f32(u_in, d * ny * nz)
        ptr = _fptr(a)
    _check(library().lbm_set_inout(ctx, mode, ptr, float(phi_in), float(p_out)), "lbm_set_inout", ctx)


def lbm_step(ctx, n):
    _check(library().lbm_step(ctx, n), "lbm_step", ctx)


def lbm_phase_flux(ctx, instance=0, axis=0) -> dict:
    out = lbm_flux()
    _check(library().lbm_phase_flux(ctx, instance, axis, ctypes.byref(out)), "lbm_phase_flux", ctx)
    return out.as_dict()


def relative_permeability(two_phase, single_1, single_2):
    """K_1, K_2 (Eq. eq-Kp) from lbm_phase_flux records: a two-phase run and single-phase runs of each fluid."""
    return two_phase["q1"] / single_1["q"], two_phase["q2"] / single_2["q"]


def lbm_sync(ctx):
    _check(library().lbm_sync(ctx), "lbm_sync", ctx)


def lbm_get_fields(ctx, phi1=None, u=None, p=None):
    """Fill (or allocate) float32 arrays phi1 [b, nodes], u [b, d, nodes], p [b, nodes]."""
    n, nb, q = _nodes(ctx)
    d = 2 if q == 9 else 3
    phi1 = np.empty((nb, n), np.float32) if phi1 is None else phi1
    u = np.empty((nb, d, n), np.float32) if u is None else u
    p = np.empty((nb, n), np.float32) if p is None else p
    for a, size in ((phi1, nb * n), (u, nb * d * n), (p, nb * n)):
        if a.dtype != np.float32 or not a.flags.c_contiguous or a.size != size:
            raise ValueError("output arrays must be C-contiguous float32 of the right size")
    _check(library().lbm_get_fields(ctx, _fptr(phi1), _fptr(u), _fptr(p)), "lbm_get_fields", ctx)
    return phi1, u, p


def lbm_get_populations(ctx):
    n, nb, q = _nodes(ctx)
    f = np.empty((nb, q, n), np.float32)
    g = np.empty((nb, q, n), np.float32)
    _check(library().lbm_get_populations(ctx, _fptr(f), _fptr(g)), "lbm_get_populations", ctx)
    return f, g


def lbm_get_state(ctx) -> bytes:
    size = c_size_t(0)
    _check(library().lbm_get_state(ctx, None, ctypes.byref(size)), "lbm_get_state", ctx)
    buf = ctypes.create_string_buffer(size.value)
    _check(library().lbm_get_state(ctx, buf, ctypes.byref(size)), "lbm_get_state", ctx)
    return buf.raw


def lbm_set_state(ctx, image: bytes):
    buf = ctypes.create_string_buffer(image, len(image))
    _check(library().lbm_set_state(ctx, buf, len(image)), "lbm_set_state", ctx)


def lbm_observables(ctx, instance=0) -> dict:
    o = lbm_obs()
    _check(library().lbm_observables(ctx, instance, ctypes.byref(o)), "lbm_observables", ctx)
    return o.as_dict()


def lbm_observables_noalloc(phi0_ptr, phi1_ptr, u_ptr, d, p_ptr, n, out_ptr, stream=0):
    """Allocation-free diagnostics on caller-owned device buffers (see include/lbm.h);
    returns the status code instead of raising so that callers can test the refusals."""
    return library().lbm_observables_noalloc(c_void_p(phi0_ptr), c_void_p(phi1_ptr), c_void_p(u_ptr), d,
                                             c_void_p(p_ptr), n, c_void_p(out_ptr), c_void_p(stream))


def lbm_contact_angle(ctx, instance, mode, column, y_c=0.0, disk_radius=0.0):
    th, h = c_double(), c_double()
    _check(library().lbm_contact_angle(ctx, instance, mode, column, y_c, disk_radius, ctypes.byref(th),
                                       ctypes.byref(h)), "lbm_contact_angle", ctx)
    return th.value, h.value


def lbm_set_profiling(ctx, enable):
    _check(library().lbm_set_profiling(ctx, 1 if enable else 0), "lbm_set_profiling", ctx)


def lbm_kernel_time(ctx):
    """(summed device milliseconds, steps) of the step kernels timed since the last read."""
    ms, n = c_double(), ctypes.c_int64()
    _check(library().lbm_kernel_time(ctx, ctypes.byref(ms), ctypes.byref(n)), "lbm_kernel_time", ctx)
    return ms.value, n.value


def lbm_kernel_time_split(ctx):
    """((moment-pass ms, fused-kernel ms), steps) timed since the last read."""
    ms, n = (c_double * 2)(), ctypes.c_int64()
    _check(library().lbm_kernel_time_split(ctx, ms, ctypes.byref(n)), "lbm_kernel_time_split", ctx)
    return (ms[0], ms[1]), n.value


def lbm_strerror(status) -> str:
    return library().lbm_strerror(status).decode()


class Context:
    """Owns one lbm_ctx; each method forwards to the C call of the same name."""

    def __init__(self, lattice, nx, ny, nz=1, periodic=(True, True, True), params=None, batch=None, flags=0,
                 allocator=None, stream=None):
        mask = sum(bit for bit, on in zip((1, 2, 4), periodic) if on)
        self.shape = (nx, ny, nz)
        self._allocator = allocator          # the callbacks must outlive the context
        if allocator is not None:
            plist = batch if batch is not None else [params if params is not None else lbm_default_params()]
            self.ctx = lbm_create_alloc(lattice, nx, ny, nz, mask, plist, flags, stream, allocator)
        elif flags:
            plist = batch if batch is not None else [params if params is not None else lbm_default_params()]
            self.ctx = lbm_create_ex(lattice, nx, ny, nz, mask, plist, flags)
        elif batch is not None:
            self.ctx = lbm_create_batch(lattice, nx, ny, nz, mask, batch)
        else:
            self.ctx = lbm_create(lattice, nx, ny, nz, mask, params if params is not None else lbm_default_params())
        self.q = {LBM_D2Q9: 9, LBM_D3Q19: 19, LBM_D3Q15: 15}[lattice]
        self.d = 2 if lattice == LBM_D2Q9 else 3

    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, handle): lbm_set_stream(self.ctx, handle)
    def set_launch(self, strip, depth=0): lbm_set_launch(self.ctx, strip, depth)
    def set_wait_limit(self, polls): lbm_set_wait_limit(self.ctx, polls)
    def tune(self, trial=10): return lbm_tune(self.ctx, trial, lbm_get_shape(self.ctx)[3])
    def set_solid(self, phi0): lbm_set_solid(self.ctx, phi0)
    def set_phase(self, phi1): lbm_set_phase(self.ctx, phi1)
    def set_solid_device(self, ptr): lbm_set_solid_device(self.ctx, ptr)
    def set_phase_device(self, ptr): lbm_set_phase_device(self.ctx, ptr)
    def step(self, n=1): lbm_step(self.ctx, n)
    def set_inout(self, mode, u_in=None, phi_in=-1.0, p_out=0.0): lbm_set_inout(self.ctx, mode, u_in, phi_in, p_out)
    def sync(self): lbm_sync(self.ctx)
    def get_fields(self, *a): return lbm_get_fields(self.ctx, *a)
    def get_populations(self): return lbm_get_populations(self.ctx)
    def get_state(self): return lbm_get_state(self.ctx)
    def set_state(self, image): lbm_set_state(self.ctx, image)
    def observables(self, instance=0): return lbm_observables(self.ctx, instance)
    def phase_flux(self, instance=0, axis=0): return lbm_phase_flux(self.ctx, instance, axis)
    def set_profiling(self, enable): lbm_set_profiling(self.ctx, enable)
    def kernel_time(self): return lbm_kernel_time(self.ctx)
    def kernel_time_split(self): return lbm_kernel_time_split(self.ctx)
    def contact_angle(self, instance, mode, column, y_c=0.0, disk_radius=0.0):
        return lbm_contact_angle(self.ctx, instance, mode, column, y_c, disk_radius)


class MultiContext:
    """Owns one lbm_ctx of D2Q9 instances of different sizes (lbm_create_multi).

    Fields go in and out per instance: lists of [ny, nx] arrays; the C calls
    see the instances' blocks back to back.
    """

    def __init__(self, sizes, periodic=(True, True), batch=None, flags=0):
        mask = sum(bit for bit, on in zip((1, 2), periodic) if on)
        self.sizes = [(int(a), int(b)) for a, b in sizes]
        params = batch if batch is not None else [lbm_default_params() for _ in sizes]
        self.ctx = lbm_create_multi(LBM_D2Q9, self.sizes, mask, params, flags)
        self.offsets = [lbm_get_instance_shape(self.ctx, k)[2] for k in range(len(self.sizes))]
        self.total = self.offsets[-1] + self.sizes[-1][0] * self.sizes[-1][1]

    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _flat(self, fields):
        out = np.empty(self.total, np.float32)
        for k, ((nx, ny), off) in enumerate(zip(self.sizes, self.offsets)):
            a = np.ascontiguousarray(fields[k], dtype=np.float32).ravel()
            if a.size != nx * ny:
                raise ValueError(f"instance {k}: expected {nx * ny} values, got {a.size}")
            out[off:off + nx * ny] = a
        return out

    def set_solid(self, fields):
        a = self._flat(fields)
        _check(library().lbm_set_solid(self.ctx, _fptr(a)), "lbm_set_solid", self.ctx)

    def set_phase(self, fields):
        a = self._flat(fields)
        _check(library().lbm_set_phase(self.ctx, _fptr(a)), "lbm_set_phase", self.ctx)

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def sync(self):
        lbm_sync(self.ctx)

    def set_launch(self, strip, depth=0):
        lbm_set_launch(self.ctx, strip, depth)

    def set_stream(self, handle):
        lbm_set_stream(self.ctx, handle)

    def tune(self, trial=10):
        return lbm_tune(self.ctx, trial, len(self.sizes))

    def get_fields(self):
        """Per instance: (phi1 [ny, nx], u [2, ny, nx], p [ny, nx])."""
        phi1 = np.empty(self.total, np.float32)
        u = np.empty(2 * self.total, np.float32)
        p = np.empty(self.total, np.float32)
        _check(library().lbm_get_fields(self.ctx, _fptr(phi1), _fptr(u), _fptr(p)), "lbm_get_fields", self.ctx)
        out = []
        for (nx, ny), off in zip(self.sizes, self.offsets):
            n = nx * ny
            out.append((phi1[off:off + n].reshape(ny, nx), u[2 * off:2 * off + 2 * n].reshape(2, ny, nx),
                        p[off:off + n].reshape(ny, nx)))
        return out

    def get_populations(self):
        """Per instance: (f [9, ny, nx], g [9, ny, nx])."""
        f = np.empty(9 * self.total, np.float32)
        g = np.empty(9 * self.total, np.float32)
        _check(library().lbm_get_populations(self.ctx, _fptr(f), _fptr(g)), "lbm_get_populations", self.ctx)
        return [(f[9 * off:9 * (off + nx * ny)].reshape(9, ny, nx), g[9 * off:9 * (off + nx * ny)].reshape(9, ny, nx))
                for (nx, ny), off in zip(self.sizes, self.offsets)]

    def get_state(self):
        return lbm_get_state(self.ctx)

    def set_state(self, image):
        lbm_set_state(self.ctx, image)

    def observables(self, instance=0):
        return lbm_observables(self.ctx, instance)

    def contact_angle(self, instance, mode, column, y_c=0.0, disk_radius=0.0):
        return lbm_contact_angle(self.ctx, instance, mode, column, y_c, disk_radius)

    def set_profiling(self, enable):
        lbm_set_profiling(self.ctx, enable)

    def kernel_time(self):
        return lbm_kernel_time(self.ctx)
