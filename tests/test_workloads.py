"""The seeded synthetic inputs (paper_2311_10827_gb300/workloads.py) against
the formulas they are stated from: the tanh profiles of the paper's numerical
tests (Section 3: Eq. flatinitial, Eq. case1 written for phi, the two droplets
of the coalescence test) and the ensemble recipe (default_rng(seed), then N,
R/N and the density ratio, in that order).  Values are checked at nodes where
the profile is known in closed form."""
import math

import numpy as np
import pytest

from paper_2311_10827_gb300 import workloads as wl


def test_flat_interface_profile():
    phi = wl.flat_interface(3, 64, 4.0)  # y1 = 16, y2 = 48
    assert phi.shape == (64, 3)
    assert np.array_equal(phi, np.repeat(phi[:, :1], 3, axis=1))  # x-independent
    assert abs(phi[16, 0] - 0.5) < 1e-12 and abs(phi[48, 0] - 0.5) < 1e-12
    assert abs(phi[32, 0] - math.tanh(8.0)) < 1e-15  # the slab's middle
    assert phi[0, 0] < 1e-6 and phi.min() >= 0.0 and phi.max() <= 1.0
    k = np.arange(32)
    assert np.allclose(phi[32 + k, 0], phi[32 - k, 0], rtol=0, atol=1e-15)  # symmetric slab
    # near y1 the profile is 1/2 + 1/2 tanh(2 (y - y1) / W)
    assert abs(phi[17, 0] - (0.5 + 0.5 * math.tanh(0.5))) < 1e-12


def test_flat_interface_phases_and_positions():
    phi = wl.flat_interface(1, 40, 2.0, phi_l=0.8, phi_v=-0.2, y1=10.0, y2=30.0)
    assert abs(phi[20, 0] - 0.8) < 1e-8 and abs(phi[0, 0] + 0.2) < 1e-8
    assert abs(phi[10, 0] - 0.3) < 1e-12 and abs(phi[30, 0] - 0.3) < 1e-12


def test_droplet_profile():
    phi = wl.droplet(64, 48, 10.0, 4.0)  # centre (32, 24)
    assert phi.shape == (48, 64)
    assert phi[24, 32] == 0.5 + 0.5 * math.tanh(5.0)
    assert phi[24, 42] == 0.5 and phi[34, 32] == 0.5  # r = R
    k = np.arange(1, 20)
    assert np.array_equal(phi[24, 32 + k], phi[24, 32 - k])
    assert np.array_equal(phi[24 + k[:15], 32], phi[24, 32 + k[:15]])  # radial
    assert phi.min() > 0.0 and phi.max() < 1.0


def test_droplet_3d_and_phases():
    phi = wl.droplet(16, 12, 4.0, 2.0, nz=8)  # centre (8, 6, 4)
    assert phi.shape == (8, 12, 16)
    assert phi[4, 6, 8] == 0.5 + 0.5 * math.tanh(4.0)
    assert phi[4, 6, 12] == 0.5 and phi[0, 6, 8] == 0.5 and phi[4, 10, 8] == 0.5
    p2 = wl.droplet(64, 64, 20.0, 4.0, phi_l=0.8, phi_v=-0.2)
    assert abs(p2[32, 32] - 0.8) < 1e-8 and abs(p2[0, 0] + 0.2) < 1e-8


def test_two_droplets_layout():
    R, W = 20.0, 4.0
    phi = wl.two_droplets(128, 64, R, W)  # centres x = 64 -/+ (R + W/2) = 42, 86; y = 32
    assert phi.shape == (64, 128)
    # the midpoint lies W/2 outside both droplets
    assert abs(phi[32, 64] - (0.5 + 0.5 * (1.0 - 2.0 * math.tanh(1.0)))) < 1e-15
    # the first droplet's centre: d1 = -R, d2 = 2 (R + W/2) - R = 24
    assert abs(phi[32, 42] - (0.5 + 0.5 * (1.0 - math.tanh(-10.0) - math.tanh(12.0)))) < 1e-15
    k = np.arange(64)
    # mirror about x = L/2 (the two tanh terms swap: equal to rounding)
    assert np.allclose(phi[:, 64 + k], phi[:, 64 - k], rtol=0, atol=1e-15)
    g = wl.two_droplets(128, 64, R, W, gap=10.0)  # centres 64 -/+ 25
    assert abs(g[32, 39] - (0.5 + 0.5 * (1.0 - math.tanh(-10.0) - math.tanh(2 * (50 - R) / W)))) < 1e-14


def test_two_droplets_3d_matches_2d_midplane():
    p3 = wl.two_droplets(64, 32, 8.0, 4.0, nz=32)
    p2 = wl.two_droplets(64, 32, 8.0, 4.0)
    assert p3.shape == (32, 32, 64)
    assert np.array_equal(p3[16], p2)  # z = L/2 plane


@pytest.mark.parametrize("seed", [0, 1, 17, 255])
def test_ensemble_recipe(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(64, 513))
    R = float(rng.uniform(0.15, 0.35)) * n
    ratio = float(rng.uniform(1.0, 100.0))
    assert wl.ensemble_case(seed) == dict(n=n, R=R, rho_ratio=ratio)


def test_ensemble_ranges_and_size():
    cases = [wl.ensemble_case(s) for s in range(256)]
    assert all(64 <= c["n"] <= 512 for c in cases)
    assert all(0.15 * c["n"] <= c["R"] <= 0.35 * c["n"] for c in cases)
    assert all(1.0 <= c["rho_ratio"] <= 100.0 for c in cases)
    # the batch the bench times: 27,534,303 nodes per step (expected value of
    # 256 E[N^2] for N ~ U{64..512}: 25.5M)
    assert sum(c["n"] ** 2 for c in cases) == 27_534_303
    assert wl.ensemble_case(3) != wl.ensemble_case(4)
