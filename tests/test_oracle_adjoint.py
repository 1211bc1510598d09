"""The FP64 discrete adjoint of the oracle against central finite
differences of the oracle's own forward map (the gradient of the discrete
map is fixed by the mathematics, not by the paper).  Loss: L = sum (phi^n -
phi_target)^2 from the initial field phi0; gradients w.r.t. phi0 (sampled
nodes), sigma and M, on a tiny grid with every term of the step active
(density and viscosity ratios, moving interface, body force)."""
import numpy as np
import pytest

from paper_2311_10827_gb300 import workloads as wl

PRM = dict(W=4.0, M=0.08, alpha=1.0, sigma=4e-3, rho_l=5.0, rho_v=1.0, nu_l=0.3, nu_v=0.1,
           Gx=2e-5, Gy=-1e-5)


def _loss(O, shape, prm, phi0, target, n):
    o = O.Oracle(shape, **prm)
    o.init_phi(phi0)
    o.step(n)
    return float(((o.macros()["phi"] - target) ** 2).sum())


@pytest.mark.parametrize("shape,n", [((12, 10), 12), ((9, 14), 25)])
def test_adjoint_matches_finite_differences(oracle_mod, shape, n):
    O = oracle_mod
    nx, ny = shape
    phi0 = wl.two_droplets(nx, ny, 2.5, 4.0, gap=1.0)
    target = np.roll(phi0, 1, axis=1) * 0.97 + 0.01
    L, g_phi0, g_sigma, g_M = O.phi_loss_gradients(shape, PRM, phi0, target, n)
    assert L > 1e-3
    rng = np.random.default_rng(4)
    for _ in range(5):
        j, i = rng.integers(ny), rng.integers(nx)
        h = 1e-6
        pp, pm = phi0.copy(), phi0.copy()
        pp[j, i] += h
        pm[j, i] -= h
        fd = (_loss(O, shape, PRM, pp, target, n) - _loss(O, shape, PRM, pm, target, n)) / (2 * h)
        assert abs(fd - g_phi0[j, i]) <= 1e-6 * max(abs(fd), 1e-4), (fd, g_phi0[j, i])
    for key, g in (("sigma", g_sigma), ("M", g_M)):
        h = 1e-6 * PRM[key]
        lp = _loss(O, shape, dict(PRM, **{key: PRM[key] + h}), phi0, target, n)
        lm = _loss(O, shape, dict(PRM, **{key: PRM[key] - h}), phi0, target, n)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g) <= 1e-5 * abs(fd) + 1e-12, (key, fd, g)


def test_adjoint_of_zero_loss_is_zero(oracle_mod):
    O = oracle_mod
    phi0 = wl.droplet(10, 10, 3.0, 4.0)
    o = O.Oracle((10, 10), **PRM)
    o.init_phi(phi0)
    o.step(5)
    target = o.macros()["phi"]
    L, g_phi0, g_sigma, g_M = O.phi_loss_gradients((10, 10), PRM, phi0, target, 5)
    assert L == 0.0 and np.abs(g_phi0).max() == 0.0 and g_sigma == 0.0 and g_M == 0.0
