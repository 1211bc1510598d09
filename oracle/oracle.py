"""Python handle on the FP64 CPU oracle (``wb_oracle.c``).

TEST INFRASTRUCTURE.  Only the tests, the package smoke check and the
CPU-baseline leg of the benchmark may import this module.  It imports nothing
from the CUDA package and the CUDA package never imports it.

The oracle follows the paper (arXiv:2311.10827, Section 2.3) stage by stage;
the readings it takes where the paper is silent are listed at the top of
``wb_oracle.c``.  Paper names: ``f`` is the Cahn-Hilliard population, ``g`` the
hydrodynamic one.  All arrays are float64, SoA, node index
``n = (z*ny + y)*nx + x``; populations are ``[Q, nz, ny, nx]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libwb_oracle.so")
_lock = threading.Lock()
_lib = None

# parameter vector layout (must match the enum in wb_oracle.c)
PARAM_KEYS = ("W", "M", "alpha", "sigma", "phi_l", "phi_v", "rho_l", "rho_v",
              "nu_l", "nu_v", "Gx", "Gy", "Gz", "tau_f")
DEFAULTS = dict(W=4.0, M=0.1, alpha=1.0, sigma=1e-3, phi_l=1.0, phi_v=0.0,
                rho_l=10.0, rho_v=1.0, nu_l=0.1, nu_v=0.1, Gx=0.0, Gy=0.0,
                Gz=0.0, tau_f=0.0)
LATTICES = {"D2Q9": 0, "D3Q19": 1}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build`` (plain C, -O2)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.wbo_create.restype = ctypes.c_void_p
        L.wbo_create.argtypes = [ctypes.c_int] * 4 + [dp]
        L.wbo_destroy.argtypes = [ctypes.c_void_p]
        L.wbo_init_phi.argtypes = [ctypes.c_void_p, dp]
        L.wbo_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.wbo_macros.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
        L.wbo_diag.argtypes = [ctypes.c_void_p, dp]
        L.wbo_get_state.argtypes = [ctypes.c_void_p, dp, dp, dp]
        L.wbo_set_state.argtypes = [ctypes.c_void_p, dp, dp, dp, ctypes.c_long]
        L.wbo_time.restype = ctypes.c_long
        L.wbo_time.argtypes = [ctypes.c_void_p]
        L.wbo_derived.argtypes = [ctypes.c_void_p, dp]
        L.wbo_lattice.argtypes = [ctypes.c_int, ip, ip, ip, dp]
        L.wbo_node_feq.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, dp]
        L.wbo_node_F.argtypes = [ctypes.c_int, ctypes.c_double, dp]
        L.wbo_node_geq.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp]
        L.wbo_node_G.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp, dp, dp]
        L.wbo_field_grad.argtypes = [ctypes.c_void_p, dp, dp]
        L.wbo_field_lap.argtypes = [ctypes.c_void_p, dp, dp]
        L.wbo_field_mu.argtypes = [ctypes.c_void_p, dp, dp]
        L.wbo_kappa_beta.argtypes = [ctypes.c_double] * 4 + [dp, dp]
        L.wbo_adjoint.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, dp, dp, dp]
        L.wbo_adjoint_init.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
        L.wbo_psi.restype = ctypes.c_double
        L.wbo_psi.argtypes = [ctypes.c_double] * 4
        L.wbo_dpsi.restype = ctypes.c_double
        L.wbo_dpsi.argtypes = [ctypes.c_double] * 4
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def lattice(name: str = "D2Q9"):
    """(D, Q, c[Q,3] int, w[Q]) of the oracle's lattice."""
    D = ctypes.c_int()
    Q = ctypes.c_int()
    c = np.zeros(19 * 3, dtype=np.int32)
    w = np.zeros(19)
    rc = lib().wbo_lattice(LATTICES[name], ctypes.byref(D), ctypes.byref(Q),
                           c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(w))
    assert rc == 0
    q = Q.value
    return D.value, q, c.reshape(19, 3)[:q].copy(), w[:q].copy()


def kappa_beta(W, sigma, phi_l=1.0, phi_v=0.0):
    k = ctypes.c_double()
    b = ctypes.c_double()
    lib().wbo_kappa_beta(W, sigma, phi_l, phi_v, ctypes.byref(k), ctypes.byref(b))
    return k.value, b.value


def psi(beta, phi, phi_l=1.0, phi_v=0.0):
    return lib().wbo_psi(beta, phi_l, phi_v, phi)


def dpsi(beta, phi, phi_l=1.0, phi_v=0.0):
    return lib().wbo_dpsi(beta, phi_l, phi_v, phi)


def node_feq(phi, mu, alpha, lat="D2Q9"):
    q = lattice(lat)[1]
    out = np.zeros(q)
    lib().wbo_node_feq(LATTICES[lat], phi, mu, alpha, _p(out))
    return out


def node_F(S, lat="D2Q9"):
    q = lattice(lat)[1]
    out = np.zeros(q)
    lib().wbo_node_F(LATTICES[lat], S, _p(out))
    return out


def _vec3(v):
    a = np.zeros(3)
    a[:len(v)] = v
    return a


def node_geq(p, rho, u, lat="D2Q9"):
    q = lattice(lat)[1]
    out = np.zeros(q)
    lib().wbo_node_geq(LATTICES[lat], p, rho, _p(_vec3(u)), _p(out))
    return out


def node_G(tau_g, u, grad_rho, F, lat="D2Q9"):
    q = lattice(lat)[1]
    out = np.zeros(q)
    lib().wbo_node_G(LATTICES[lat], tau_g, _p(_vec3(u)), _p(_vec3(grad_rho)),
                     _p(_vec3(F)), _p(out))
    return out


class Oracle:
    """One periodic grid advanced by the oracle.

    ``shape`` is ``(nx, ny)`` or ``(nx, ny, nz)``; params are the paper's
    (W, M, alpha, sigma, phi_l, phi_v, rho_l, rho_v, nu_l, nu_v, body force G,
    optional tau_f).
    """

    def __init__(self, shape, lattice_name="D2Q9", **params):
        nx, ny = shape[0], shape[1]
        nz = shape[2] if len(shape) > 2 else 1
        self.nx, self.ny, self.nz = nx, ny, nz
        self.lattice_name = lattice_name
        self.D, self.Q, self.c, self.w = lattice(lattice_name)
        prm = dict(DEFAULTS)
        unknown = set(params) - set(prm)
        if unknown:
            raise KeyError(f"unknown oracle parameters {sorted(unknown)}")
        prm.update(params)
        self.params = prm
        vec = np.array([float(prm[k]) for k in PARAM_KEYS])
        self._h = lib().wbo_create(nx, ny, nz, LATTICES[lattice_name], _p(vec))
        if not self._h:
            raise ValueError("oracle rejected the grid/lattice")
        d = np.zeros(4)
        lib().wbo_derived(self._h, _p(d))
        self.kappa, self.beta, self.tau_f, self.alpha = (float(v) for v in d)

    # grid shape of a scalar field, slowest axis first
    @property
    def fshape(self):
        return (self.nz, self.ny, self.nx) if self.nz > 1 else (self.ny, self.nx)

    @property
    def N(self):
        return self.nx * self.ny * self.nz

    def close(self):
        if getattr(self, "_h", None):
            lib().wbo_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_phi(self, phi0):
        a = np.ascontiguousarray(phi0, dtype=np.float64).reshape(-1)
        assert a.size == self.N
        lib().wbo_init_phi(self._h, _p(a))

    def step(self, n=1):
        lib().wbo_step(self._h, int(n))

    @property
    def t(self):
        return lib().wbo_time(self._h)

    def macros(self):
        """dict(phi, mu, p, u) at the current time; u is [D, *fshape]."""
        N = self.N
        phi, mu, p = np.zeros(N), np.zeros(N), np.zeros(N)
        u = np.zeros(self.D * N)
        lib().wbo_macros(self._h, _p(phi), _p(mu), _p(p), _p(u))
        fs = self.fshape
        return dict(phi=phi.reshape(fs), mu=mu.reshape(fs), p=p.reshape(fs),
                    u=u.reshape((self.D,) + fs))

    def diag(self):
        out = np.zeros(6)
        lib().wbo_diag(self._h, _p(out))
        keys = ("sum_phi", "E", "umax", "mu_min", "mu_max", "budget")
        return dict(zip(keys, (float(v) for v in out)))

    def get_state(self):
        N, Q = self.N, self.Q
        f, g, S = np.zeros(Q * N), np.zeros(Q * N), np.zeros(N)
        lib().wbo_get_state(self._h, _p(f), _p(g), _p(S))
        fs = self.fshape
        return f.reshape((Q,) + fs), g.reshape((Q,) + fs), S.reshape(fs)

    def set_state(self, f, g, S_prev, t=0):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        g = np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
        S = np.ascontiguousarray(S_prev, dtype=np.float64).reshape(-1)
        assert f.size == self.Q * self.N and g.size == f.size and S.size == self.N
        lib().wbo_set_state(self._h, _p(f), _p(g), _p(S), int(t))

    def grad(self, psi_field):
        a = np.ascontiguousarray(psi_field, dtype=np.float64).reshape(-1)
        out = np.zeros(self.D * self.N)
        lib().wbo_field_grad(self._h, _p(a), _p(out))
        return out.reshape((self.D,) + self.fshape)

    def lap(self, psi_field):
        a = np.ascontiguousarray(psi_field, dtype=np.float64).reshape(-1)
        out = np.zeros(self.N)
        lib().wbo_field_lap(self._h, _p(a), _p(out))
        return out.reshape(self.fshape)

    def mu_of(self, phi):
        a = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
        out = np.zeros(self.N)
        lib().wbo_field_mu(self._h, _p(a), _p(out))
        return out.reshape(self.fshape)


# ------------------------------------------------------------------ adjoint

def adjoint_run(sim: Oracle, n: int, lf, lg, lS):
    """From sim's current state run n steps, then propagate the final-state
    adjoint (lf, lg, lS) back; returns (lf0, lg0, lS0, dpar) with
    dpar = [dL/dkappa, dL/dbeta, dL/d(1/tau_f)] (sim ends at t + n)."""
    lf = np.ascontiguousarray(lf, dtype=np.float64).reshape(-1).copy()
    lg = np.ascontiguousarray(lg, dtype=np.float64).reshape(-1).copy()
    lS = np.ascontiguousarray(lS, dtype=np.float64).reshape(-1).copy()
    dpar = np.zeros(3)
    lib().wbo_adjoint(sim._h, int(n), _p(lf), _p(lg), _p(lS), _p(dpar))
    fs = sim.fshape
    return (lf.reshape((sim.Q,) + fs), lg.reshape((sim.Q,) + fs), lS.reshape(fs), dpar)


def adjoint_init(sim: Oracle, phi0, lf0, dpar):
    """dL/dphi0 from the adjoint of the initial populations; adds the
    kappa/beta terms of mu(phi0) to dpar (in place)."""
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64).reshape(-1)
    lf0 = np.ascontiguousarray(lf0, dtype=np.float64).reshape(-1)
    out = np.zeros(sim.N)
    lib().wbo_adjoint_init(sim._h, _p(phi0), _p(lf0), _p(out), _p(dpar))
    return out.reshape(sim.fshape)


def phi_loss_gradients(shape, params, phi0, target, n, lattice_name="D2Q9"):
    """L = sum (phi^n - target)^2 from the initial condition phi0; returns
    (L, dL/dphi0, dL/dsigma, dL/dM) by the discrete adjoint."""
    fwd = Oracle(shape, lattice_name, **params)
    fwd.init_phi(phi0)
    fwd.step(n)
    phiN = fwd.macros()["phi"]
    loss = float(((phiN - target) ** 2).sum())
    sim = Oracle(shape, lattice_name, **params)
    sim.init_phi(phi0)
    lf = np.broadcast_to(2.0 * (phiN - target), (sim.Q,) + sim.fshape)
    lg = np.zeros((sim.Q,) + sim.fshape)
    lS = np.zeros(sim.fshape)
    lf0, _, _, dpar = adjoint_run(sim, n, lf, lg, lS)
    dphi0 = adjoint_init(sim, phi0, lf0, dpar)
    prm = dict(DEFAULTS)
    prm.update(params)
    d2 = (prm["phi_l"] - prm["phi_v"]) ** 2
    dsigma = dpar[0] * 3.0 * prm["W"] / (2.0 * d2) + dpar[1] * 12.0 / (prm["W"] * d2 * d2)
    # 1/tau_f = 1/(1/2 + M/(cs2 alpha)): d(1/tau_f)/dM = -1/(tau_f^2 cs2 alpha)
    dM = dpar[2] * (-1.0 / (sim.tau_f ** 2 * (1.0 / 3.0) * sim.alpha))
    return loss, dphi0, dsigma, dM
