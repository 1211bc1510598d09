"""Convenience wrapper around one C-ABI context (marshalling only).

All arithmetic happens in the CUDA library; this class converts arguments,
allocates output arrays and turns error codes into exceptions.
"""
from __future__ import annotations

import numpy as np

from . import capi

PARAM_KEYS = ("W", "M", "alpha", "sigma", "phi_l", "phi_v", "rho_l", "rho_v", "nu_l", "nu_v",
              "Gx", "Gy", "Gz", "tau_f")
PRECISIONS = {"fp64": capi.LBM_FP64, "fp32": capi.LBM_FP32, "f16off": capi.LBM_FP32_F16OFF,
              "bf16off": capi.LBM_FP32_BF16OFF}
LATTICES = {"D2Q9": capi.LBM_D2Q9, "D3Q19": capi.LBM_D3Q19}


def make_params(precision="fp32", diag_every=0, **kw) -> capi.lbm_params:
    unknown = set(kw) - set(PARAM_KEYS)
    if unknown:
        raise KeyError(f"unknown parameters {sorted(unknown)}")
    p = capi.lbm_params_default()
    for k, v in kw.items():
        if k in ("Gx", "Gy", "Gz"):
            p.body_force["xyz".index(k[1])] = float(v)
        else:
            setattr(p, k, float(v))
    p.precision = PRECISIONS[precision]
    p.diag_every = int(diag_every)
    return p


class Simulation:
    """One periodic grid on the current CUDA device (or, with ``_borrow``, a
    view of a grid owned by a :class:`Batch`).

    ``shape`` is (nx, ny) or (nx, ny, nz).  ``stream`` is a raw cudaStream_t
    (e.g. ``torch.cuda.current_stream().cuda_stream``) or 0.
    """

    def __init__(self, shape, lattice="D2Q9", precision="fp32", stream=0, diag_every=0,
                 _borrow=None, **params):
        self.shape = tuple(shape)
        nx, ny = shape[0], shape[1]
        nz = shape[2] if len(shape) > 2 else 1
        self.nx, self.ny, self.nz = nx, ny, nz
        self.D = 2 if lattice == "D2Q9" else 3
        self.Q = 9 if lattice == "D2Q9" else 19
        self.precision = precision
        self.params = make_params(precision, diag_every, **params)
        self._owned = _borrow is None
        if _borrow is None:
            rc, h = capi.lbm_create((nx, ny, nz), LATTICES[lattice], self.params, stream)
            capi.check(rc, "lbm_create")
        else:
            h = _borrow
        self._h = h
        self.kappa, self.beta, self.tau_f, self.alpha = capi.lbm_derived(h)

    @property
    def handle(self):
        return self._h

    @property
    def N(self):
        return self.nx * self.ny * self.nz

    @property
    def fshape(self):
        return (self.nz, self.ny, self.nx) if self.nz > 1 else (self.ny, self.nx)

    @property
    def t(self):
        return capi.lbm_time(self._h)

    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                capi.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------
    def init_phi(self, phi):
        """phi: host float64 array of N values, or a CUDA float64 tensor."""
        if isinstance(phi, np.ndarray):
            a = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
            assert a.size == self.N
            capi.check(capi.lbm_init_phi(self._h, a, 0), "lbm_init_phi")
        else:
            assert phi.numel() == self.N and phi.is_cuda
            capi.check(capi.lbm_init_phi(self._h, phi.contiguous(), 1), "lbm_init_phi")

    def step(self, n=1):
        capi.check(capi.lbm_step(self._h, n), "lbm_step")

    def sync(self):
        capi.check(capi.lbm_sync(self._h), "lbm_sync")

    def moments(self):
        """Host dict(phi, p, mu, u[D, ...]) at the current time."""
        N = self.N
        phi, p, mu = np.empty(N), np.empty(N), np.empty(N)
        u = np.empty(self.D * N)
        capi.check(capi.lbm_moments(self._h, phi, p, u, mu, 0), "lbm_moments")
        fs = self.fshape
        return dict(phi=phi.reshape(fs), p=p.reshape(fs), mu=mu.reshape(fs),
                    u=u.reshape((self.D,) + fs))

    def moments_device(self, phi=None, p=None, u=None, mu=None):
        """Write the requested fields into CUDA float64 tensors (asynchronous)."""
        capi.check(capi.lbm_moments(self._h, phi, p, u, mu, 1), "lbm_moments")

    def diagnostics(self):
        rc, d = capi.lbm_diagnostics(self._h)
        capi.check(rc, "lbm_diagnostics")
        return d.as_dict()

    def last_diagnostics(self):
        rc, d = capi.lbm_last_diagnostics(self._h)
        capi.check(rc, "lbm_last_diagnostics")
        return d.as_dict()

    def get_state(self):
        N, Q = self.N, self.Q
        f, g, S = np.empty(Q * N), np.empty(Q * N), np.empty(N)
        capi.check(capi.lbm_get_state(self._h, f, g, S, 0), "lbm_get_state")
        fs = self.fshape
        return f.reshape((Q,) + fs), g.reshape((Q,) + fs), S.reshape(fs)

    def set_state(self, f, g, S_prev, step=0):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        g = np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
        S = np.ascontiguousarray(S_prev, dtype=np.float64).reshape(-1)
        assert f.size == self.Q * self.N and g.size == f.size and S.size == self.N
        capi.check(capi.lbm_set_state(self._h, f, g, S, step, 0), "lbm_set_state")

    def save(self) -> np.ndarray:
        rc, buf = capi.lbm_save(self._h)
        capi.check(rc, "lbm_save")
        return buf

    def load(self, buf: np.ndarray):
        capi.check(capi.lbm_load(self._h, np.ascontiguousarray(buf)), "lbm_load")


class Batch:
    """Many independent D2Q9 grids advanced by one launch per step.

    ``cases`` is a list of ``(shape, params_dict)``; all at ``precision``.
    ``batch.case(i)`` is a :class:`Simulation` view of grid i (initialise,
    read moments, diagnostics, state) owned by the batch.
    """

    def __init__(self, cases, precision="fp32", stream=0):
        self.shapes = [tuple(sh) for sh, _ in cases]
        plist = [make_params(precision, 0, **prm) for _, prm in cases]
        rc, h = capi.lbm_batch_create(self.shapes, plist, stream)
        capi.check(rc, "lbm_batch_create")
        self._h = h
        self._cases = []
        for i, (sh, prm) in enumerate(cases):
            rc, ch = capi.lbm_batch_case(h, i)
            capi.check(rc, "lbm_batch_case")
            self._cases.append(Simulation(sh, precision=precision, _borrow=ch, **prm))

    def __len__(self):
        return len(self._cases)

    def case(self, i) -> Simulation:
        return self._cases[i]

    def step(self, n=1):
        capi.check(capi.lbm_batch_step(self._h, n), "lbm_batch_step")

    def tune(self):
        rc, w, r = capi.lbm_batch_tune(self._h)
        capi.check(rc, "lbm_batch_tune")
        return w, r

    def shape(self):
        return capi.lbm_batch_shape(self._h)

    def set_shape(self, width, rows):
        capi.check(capi.lbm_batch_set_shape(self._h, width, rows), "lbm_batch_set_shape")

    def set_persistent(self, on=True):
        """Multi-step launches (lbm_batch_set_persistent): one cooperative
        launch per step(n) call, tiles synchronised with their neighbours."""
        capi.check(capi.lbm_batch_set_persistent(self._h, int(on)), "lbm_batch_set_persistent")

    def persistent(self, read_timeout=False):
        """(on, timed_out) of lbm_batch_persistent."""
        return capi.lbm_batch_persistent(self._h, read_timeout)

    def set_diag_every(self, k):
        """Fused diagnostics of every grid every k steps (lbm_batch_set_diag_every)."""
        capi.check(capi.lbm_batch_set_diag_every(self._h, k), "lbm_batch_set_diag_every")

    def last_diagnostics(self):
        """Records of the last fused diagnostics step, one dict per grid."""
        rc, recs = capi.lbm_batch_last_diagnostics(self._h, len(self))
        capi.check(rc, "lbm_batch_last_diagnostics")
        return [r.as_dict() for r in recs]

    def sync(self):
        capi.check(capi.lbm_batch_sync(self._h), "lbm_batch_sync")

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            for c in self._cases:
                c._h = None
            capi.lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
