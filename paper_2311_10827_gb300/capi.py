"""ctypes binding of the C ABI in include/lbm.h (argument marshalling only).

Every function keeps its C name.  There is no fallback: if the CUDA library
has not been built, :func:`lib` raises.  Device buffers may be passed as
integers (raw device pointers, e.g. ``tensor.data_ptr()``) together with
``on_device=1``; host buffers as C-contiguous float64 numpy arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LBM_OK = 0
LBM_ERR_INVALID_ARG = -1
LBM_ERR_OOM = -2
LBM_ERR_CUDA = -3
LBM_ERR_NONFINITE = -4
LBM_ERR_TIMEOUT = -5
LBM_ERR_STATE = -6

LBM_D2Q9, LBM_D3Q19 = 0, 1
LBM_FP64, LBM_FP32, LBM_FP32_F16OFF, LBM_FP32_BF16OFF = 0, 1, 2, 3

# every symbol declared in include/lbm.h
EXPORTS = ("lbm_params_default", "lbm_create", "lbm_init_phi", "lbm_step", "lbm_moments",
           "lbm_diagnostics", "lbm_last_diagnostics", "lbm_get_state", "lbm_set_state",
           "lbm_save", "lbm_load", "lbm_sync", "lbm_time", "lbm_derived", "lbm_debug_poke",
           "lbm_destroy", "lbm_strerror", "lbm_diagnostics_noalloc", "lbm_batch_create",
           "lbm_batch_case", "lbm_batch_step", "lbm_batch_tune", "lbm_batch_shape",
           "lbm_batch_destroy", "lbm_batch_set_shape", "lbm_adjoint_create", "lbm_adjoint_forward",
           "lbm_adjoint_backward", "lbm_adjoint_destroy", "lbm_state_bytes",
           "lbm_create_with_buffers", "lbm_batch_set_persistent", "lbm_batch_persistent",
           "lbm_batch_debug_stall", "lbm_batch_set_diag_every", "lbm_batch_last_diagnostics",
           "lbm_batch_sync")


class lbm_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int)]


class lbm_params(ctypes.Structure):
    _fields_ = [("W", ctypes.c_double), ("M", ctypes.c_double), ("alpha", ctypes.c_double),
                ("sigma", ctypes.c_double), ("phi_l", ctypes.c_double),
                ("phi_v", ctypes.c_double), ("rho_l", ctypes.c_double),
                ("rho_v", ctypes.c_double), ("nu_l", ctypes.c_double), ("nu_v", ctypes.c_double),
                ("body_force", ctypes.c_double * 3), ("tau_f", ctypes.c_double),
                ("precision", ctypes.c_int), ("diag_every", ctypes.c_int)]


class lbm_diag(ctypes.Structure):
    _fields_ = [("sum_phi", ctypes.c_double), ("kinetic_energy", ctypes.c_double),
                ("u_max", ctypes.c_double), ("mu_min", ctypes.c_double),
                ("mu_max", ctypes.c_double), ("budget", ctypes.c_double),
                ("step", ctypes.c_longlong), ("nonfinite", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LbmError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


_lib = None
vp = ctypes.c_void_p
dp = ctypes.c_void_p  # double* passed as raw address (host or device)


def lib(path: str | None = None):
    """Load liblbm.so (built in-tree by ``build.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build() "
                           "(no CPU fallback exists)")
    L = ctypes.CDLL(path)
    L.lbm_params_default.argtypes = [ctypes.POINTER(lbm_params)]
    L.lbm_create.argtypes = [ctypes.POINTER(lbm_grid), ctypes.c_int, ctypes.POINTER(lbm_params),
                             vp, ctypes.POINTER(vp)]
    L.lbm_state_bytes.argtypes = [ctypes.POINTER(lbm_grid), ctypes.c_int,
                                  ctypes.POINTER(lbm_params), ctypes.POINTER(ctypes.c_size_t)]
    L.lbm_create_with_buffers.argtypes = [ctypes.POINTER(lbm_grid), ctypes.c_int,
                                          ctypes.POINTER(lbm_params), vp,
                                          ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(vp)]
    L.lbm_init_phi.argtypes = [vp, dp, ctypes.c_int]
    L.lbm_step.argtypes = [vp, ctypes.c_int]
    L.lbm_moments.argtypes = [vp, dp, dp, dp, dp, ctypes.c_int]
    L.lbm_diagnostics.argtypes = [vp, ctypes.POINTER(lbm_diag)]
    L.lbm_last_diagnostics.argtypes = [vp, ctypes.POINTER(lbm_diag)]
    L.lbm_get_state.argtypes = [vp, dp, dp, dp, ctypes.c_int]
    L.lbm_set_state.argtypes = [vp, dp, dp, dp, ctypes.c_longlong, ctypes.c_int]
    L.lbm_save.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t)]
    L.lbm_load.argtypes = [vp, vp, ctypes.c_size_t]
    L.lbm_sync.argtypes = [vp]
    L.lbm_time.argtypes = [vp]
    L.lbm_time.restype = ctypes.c_longlong
    L.lbm_derived.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.lbm_debug_poke.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
                                 ctypes.c_double]
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_diagnostics_noalloc.argtypes = [ctypes.POINTER(lbm_grid), ctypes.c_int,
                                          ctypes.POINTER(lbm_params), vp, vp, vp, vp, vp]
    L.lbm_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(lbm_grid),
                                   ctypes.POINTER(lbm_params), vp, ctypes.POINTER(vp)]
    L.lbm_batch_case.argtypes = [vp, ctypes.c_int, ctypes.POINTER(vp)]
    L.lbm_batch_step.argtypes = [vp, ctypes.c_int]
    L.lbm_batch_tune.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.lbm_batch_shape.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_int)]
    L.lbm_batch_set_shape.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.lbm_batch_set_persistent.argtypes = [vp, ctypes.c_int]
    L.lbm_batch_debug_stall.argtypes = [vp, ctypes.c_int]
    L.lbm_batch_persistent.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.lbm_batch_set_diag_every.argtypes = [vp, ctypes.c_int]
    L.lbm_batch_last_diagnostics.argtypes = [vp, ctypes.POINTER(lbm_diag)]
    L.lbm_batch_sync.argtypes = [vp]
    L.lbm_batch_destroy.argtypes = [vp]
    L.lbm_batch_destroy.restype = None
    L.lbm_adjoint_create.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)]
    L.lbm_adjoint_forward.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int]
    L.lbm_adjoint_backward.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_double)]
    L.lbm_adjoint_destroy.argtypes = [vp]
    L.lbm_adjoint_destroy.restype = None
    L.lbm_strerror.argtypes = [ctypes.c_int]
    L.lbm_strerror.restype = ctypes.c_char_p
    _lib = L
    return L


def strerror(code: int) -> str:
    return lib().lbm_strerror(int(code)).decode()


def check(code: int, what: str = "lbm") -> int:
    if code != LBM_OK:
        raise LbmError(code, what)
    return code


def addr(buf) -> int | None:
    """Raw address of a host numpy array or a device tensor; None stays NULL."""
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    if isinstance(buf, np.ndarray):
        assert buf.flags["C_CONTIGUOUS"]
        return buf.ctypes.data
    if hasattr(buf, "data_ptr"):
        assert buf.is_contiguous()
        return buf.data_ptr()
    raise TypeError(f"unsupported buffer type {type(buf)}")


# ------------------------------------------------------------- same names

def lbm_params_default() -> lbm_params:
    p = lbm_params()
    check(lib().lbm_params_default(ctypes.byref(p)), "lbm_params_default")
    return p


def lbm_create(grid, lattice, params, cuda_stream=0):
    """Returns (rc, handle).  ``grid`` is (nx, ny[, nz]) or an lbm_grid."""
    if not isinstance(grid, lbm_grid):
        g = tuple(grid) + (1,) * (3 - len(grid))
        grid = lbm_grid(*g)
    h = vp()
    rc = lib().lbm_create(ctypes.byref(grid), int(lattice), ctypes.byref(params),
                          vp(cuda_stream or None), ctypes.byref(h))
    return rc, h


def _grid(grid):
    if isinstance(grid, lbm_grid):
        return grid
    return lbm_grid(*(tuple(grid) + (1,) * (3 - len(grid))))


def lbm_state_bytes(grid, lattice, params):
    """Returns (rc, (f_bytes, g_bytes, S_bytes))."""
    out = (ctypes.c_size_t * 3)()
    rc = lib().lbm_state_bytes(ctypes.byref(_grid(grid)), int(lattice), ctypes.byref(params), out)
    return rc, tuple(int(v) for v in out)


def lbm_create_with_buffers(grid, lattice, params, buffers, cuda_stream=0):
    """Returns (rc, handle); ``buffers`` = five device tensors (or raw device
    addresses): f buffer 0, f buffer 1, g buffer 0, g buffer 1, S_prev."""
    arr = (ctypes.c_void_p * 5)(*[addr(b) if not isinstance(b, int) else b for b in buffers])
    h = vp()
    rc = lib().lbm_create_with_buffers(ctypes.byref(_grid(grid)), int(lattice),
                                       ctypes.byref(params), vp(cuda_stream or None), arr,
                                       ctypes.byref(h))
    return rc, h


def lbm_init_phi(h, phi, on_device):
    return lib().lbm_init_phi(h, addr(phi), int(on_device))


def lbm_step(h, n):
    return lib().lbm_step(h, int(n))


def lbm_moments(h, phi, p, u, mu, on_device):
    return lib().lbm_moments(h, addr(phi), addr(p), addr(u), addr(mu), int(on_device))


def lbm_diagnostics(h):
    d = lbm_diag()
    rc = lib().lbm_diagnostics(h, ctypes.byref(d))
    return rc, d


def lbm_last_diagnostics(h):
    d = lbm_diag()
    rc = lib().lbm_last_diagnostics(h, ctypes.byref(d))
    return rc, d


def lbm_get_state(h, f, g, S_prev, on_device):
    return lib().lbm_get_state(h, addr(f), addr(g), addr(S_prev), int(on_device))


def lbm_set_state(h, f, g, S_prev, step, on_device):
    return lib().lbm_set_state(h, addr(f), addr(g), addr(S_prev), int(step), int(on_device))


def lbm_save(h):
    n = ctypes.c_size_t(0)
    check(lib().lbm_save(h, None, ctypes.byref(n)), "lbm_save(size)")
    buf = np.empty(n.value, dtype=np.uint8)
    rc = lib().lbm_save(h, buf.ctypes.data, ctypes.byref(n))
    return rc, buf


def lbm_load(h, buf):
    return lib().lbm_load(h, addr(buf), buf.nbytes)


def lbm_sync(h):
    return lib().lbm_sync(h)


def lbm_time(h):
    return lib().lbm_time(h)


def lbm_derived(h):
    out = (ctypes.c_double * 4)()
    check(lib().lbm_derived(h, out), "lbm_derived")
    return tuple(out)


def lbm_debug_poke(h, field, i, n, value):
    return lib().lbm_debug_poke(h, int(field), int(i), int(n), float(value))


def lbm_destroy(h):
    lib().lbm_destroy(h)


def lbm_strerror(code):
    return strerror(code)


def lbm_diagnostics_noalloc(grid, lattice, params, f, g, S_prev, out, cuda_stream=0):
    """All buffers are device addresses (ints or CUDA tensors); see lbm.h."""
    if not isinstance(grid, lbm_grid):
        gg = tuple(grid) + (1,) * (3 - len(grid))
        grid = lbm_grid(*gg)
    return lib().lbm_diagnostics_noalloc(ctypes.byref(grid), int(lattice), ctypes.byref(params),
                                         addr(f), addr(g), addr(S_prev), addr(out),
                                         vp(cuda_stream or None))


def lbm_batch_create(grids, params, cuda_stream=0):
    """grids: list of (nx, ny); params: list of lbm_params.  Returns (rc, handle)."""
    n = len(grids)
    ga = (lbm_grid * n)(*[lbm_grid(g[0], g[1], 1) for g in grids])
    pa = (lbm_params * n)(*params)
    h = vp()
    rc = lib().lbm_batch_create(n, ga, pa, vp(cuda_stream or None), ctypes.byref(h))
    return rc, h


def lbm_batch_case(b, c):
    h = vp()
    rc = lib().lbm_batch_case(b, int(c), ctypes.byref(h))
    return rc, h


def lbm_batch_step(b, n):
    return lib().lbm_batch_step(b, int(n))


def lbm_batch_tune(b):
    w, r = ctypes.c_int(), ctypes.c_int()
    rc = lib().lbm_batch_tune(b, ctypes.byref(w), ctypes.byref(r))
    return rc, w.value, r.value


def lbm_batch_shape(b):
    w, r, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(lib().lbm_batch_shape(b, ctypes.byref(w), ctypes.byref(r), ctypes.byref(t)))
    return w.value, r.value, t.value


def lbm_batch_set_shape(b, width, rows):
    return lib().lbm_batch_set_shape(b, int(width), int(rows))


def lbm_batch_set_persistent(b, on):
    return lib().lbm_batch_set_persistent(b, int(on))


def lbm_batch_persistent(b, read_timeout=False):
    """Returns (on, timed_out); timed_out is None unless read_timeout (which
    synchronises the device)."""
    on, to = ctypes.c_int(), ctypes.c_int()
    check(lib().lbm_batch_persistent(b, ctypes.byref(on), ctypes.byref(to) if read_timeout else None))
    return bool(on.value), (bool(to.value) if read_timeout else None)


def lbm_batch_debug_stall(b, tile):
    return lib().lbm_batch_debug_stall(b, int(tile))


def lbm_batch_set_diag_every(b, k):
    return lib().lbm_batch_set_diag_every(b, int(k))


def lbm_batch_last_diagnostics(b, ncases):
    """(rc, [lbm_diag] * ncases)."""
    out = (lbm_diag * int(ncases))()
    rc = lib().lbm_batch_last_diagnostics(b, out)
    return rc, list(out)


def lbm_batch_sync(b):
    return lib().lbm_batch_sync(b)


def lbm_batch_destroy(b):
    lib().lbm_batch_destroy(b)


def lbm_adjoint_create(ctx, checkpoint_every, max_steps):
    h = vp()
    rc = lib().lbm_adjoint_create(ctx, int(checkpoint_every), int(max_steps), ctypes.byref(h))
    return rc, h


def lbm_adjoint_forward(a, phi0, on_device, nsteps):
    return lib().lbm_adjoint_forward(a, addr(phi0), int(on_device), int(nsteps))


def lbm_adjoint_backward(a, dL_dphi, on_device, dL_dphi0):
    """Returns (rc, (dL/dsigma, dL/dM, dL/dkappa, dL/dbeta))."""
    g = (ctypes.c_double * 4)()
    rc = lib().lbm_adjoint_backward(a, addr(dL_dphi), int(on_device), addr(dL_dphi0), g)
    return rc, tuple(g)


def lbm_adjoint_destroy(a):
    lib().lbm_adjoint_destroy(a)
