"""The oracle reproduces the magnitudes the paper quotes for its own model
(tests/golden/paper_magnitudes.json, each entry with its citation), plus two
equilibrium facts: the tanh profile of a plane interface (Eq. flatinitial) and
the Laplace pressure jump of a droplet (sigma / R in 2D; with the potential
force -phi grad(mu) the hydrodynamic p is uniform and the jump sits in the
total pressure p + phi mu - psi).

The flat interface is one-dimensional, so it runs on a 1 x 32 periodic column
(x-independent fields make every x-neighbour equal to the node itself), with
the paper's W = 4, M = 0.1, alpha = 1, sigma = 5e-3, nu_v = 0.1.  E is
compared per node (the paper's grid has 32 x 128 nodes).
"""
import json
import os

import numpy as np
import pytest

from paper_2311_10827_gb300 import workloads as wl

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_magnitudes.json")))
PAPER_NODES = 32 * 128


def _flat(O, ratio, nu_l, steps):
    o = O.Oracle((1, 32), W=4.0, M=0.1, alpha=1.0, sigma=5e-3, rho_l=float(ratio), rho_v=1.0,
                 nu_l=nu_l, nu_v=0.1)
    o.init_phi(wl.flat_interface(1, 32, 4.0))
    o.step(steps)
    return o


@pytest.mark.parametrize("nu_ratio", [0.01, 0.1, 1.0])
def test_flat_rho1000_viscosity_ratios(oracle_mod, nu_ratio):
    """Dynamic viscosity ratio 10/100/1000 at rho 1000 = kinematic 0.01/0.1/1."""
    ref = GOLD["flat_rho1000_viscosity_ratios"]
    o = _flat(oracle_mod, 1000, 0.1 * nu_ratio, 200_000)
    d = o.diag()
    assert d["umax"] < 10 * ref["sv_final"]
    assert d["E"] / o.N < 10 * ref["E_final"] / PAPER_NODES
    assert d["mu_max"] - d["mu_min"] < 1e-12


@pytest.mark.slow
def test_flat_rho10_reaches_machine_accuracy(oracle_mod):
    """Density ratio 10: E first rises (the paper notes a rise near 1e-5) and
    then falls to round-off."""
    ref = GOLD["flat_rho10_nu1"]
    o = oracle_mod.Oracle((1, 32), W=4.0, M=0.1, alpha=1.0, sigma=5e-3, rho_l=10.0, rho_v=1.0,
                          nu_l=0.1, nu_v=0.1)
    o.init_phi(wl.flat_interface(1, 32, 4.0))
    peak = 0.0
    for _ in range(10):
        o.step(100_000)
        peak = max(peak, o.diag()["E"])
    d = o.diag()
    assert peak > 1e-12                  # the transient rise happened
    assert d["umax"] < 1e-14             # "machine accuracy"
    assert d["E"] / o.N < 10 * ref["E_final"] / PAPER_NODES
    assert d["mu_max"] - d["mu_min"] < 1e-13


def test_flat_equilibrium_profile_is_tanh(oracle_mod):
    o = _flat(oracle_mod, 1000, 0.1, 200_000)
    phi = o.macros()["phi"][:, 0]
    tanh = wl.flat_interface(1, 32, 4.0)[:, 0]
    assert np.abs(phi - tanh).max() < 1e-2
    # the discrete equilibrium is a close but not exact tanh
    assert np.abs(phi - tanh).max() > 1e-6


def test_droplet_laplace_law(oracle_mod):
    """R = 8, W = 4 (R/W = 2): finite-thickness corrections of a few per cent."""
    L, R, sigma = 32, 8.0, 5e-3
    o = oracle_mod.Oracle((L, L), M=0.5, sigma=sigma, W=4.0, rho_l=10.0, rho_v=1.0,
                          nu_l=0.1, nu_v=0.1)
    o.init_phi(wl.droplet(L, L, R, 4.0))
    o.step(10_000)
    m = o.macros()
    phi, mu, p = m["phi"], m["mu"], m["p"]
    r_eq = np.sqrt(phi.sum() / np.pi)              # equimolar radius (phi_v = 0)
    psi = o.beta * phi ** 2 * (phi - 1) ** 2
    ptot = p + phi * mu - psi
    dp = ptot[L // 2, L // 2] - ptot[0, 0]
    assert abs(dp * r_eq / sigma - 1) < 0.1
    assert (p.max() - p.min()) < 0.05 * dp          # hydrodynamic p uniform
