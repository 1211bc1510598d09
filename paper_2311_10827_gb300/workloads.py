"""Seeded synthetic inputs: initial order-parameter fields and run parameters.

This module holds only the initial conditions of the paper's numerical tests
(arXiv:2311.10827, Section 3) and the parameter sets of the workloads built on
them.  It contains none of the lattice Boltzmann arithmetic, so both the CUDA
path and the CPU oracle can be fed from it.

Node-centre convention (one reading, used everywhere): node (i, j[, k]) sits
at x = i, y = j[, z = k]; a droplet centred in an L x L box sits at (L/2, L/2).
"""
from __future__ import annotations

import numpy as np


def flat_interface(nx: int, ny: int, W: float, phi_l: float = 1.0, phi_v: float = 0.0,
                   y1: float | None = None, y2: float | None = None) -> np.ndarray:
    """Liquid slab between y1 and y2 (defaults 0.25 Ly, 0.75 Ly), Eq. flatinitial.

    phi(y) = phi_v + (phi_l - phi_v)/2 [tanh(2 (y - y1)/W) - tanh(2 (y - y2)/W)].
    Returns a (ny, nx) float64 array.
    """
    y1 = 0.25 * ny if y1 is None else y1
    y2 = 0.75 * ny if y2 is None else y2
    y = np.arange(ny, dtype=np.float64)[:, None]
    prof = phi_v + 0.5 * (phi_l - phi_v) * (np.tanh(2 * (y - y1) / W) - np.tanh(2 * (y - y2) / W))
    return np.ascontiguousarray(np.broadcast_to(prof, (ny, nx)))


def droplet(nx: int, ny: int, R: float, W: float, phi_l: float = 1.0, phi_v: float = 0.0,
            center: tuple[float, float] | None = None, nz: int = 1,
            zc: float | None = None) -> np.ndarray:
    """One droplet of radius R, Eq. case1 written for phi (rho is linear in phi).

    phi = (phi_l + phi_v)/2 + (phi_l - phi_v)/2 tanh(2 (R - r)/W).
    Returns (ny, nx) for nz == 1, else (nz, ny, nx).
    """
    xc, yc = (0.5 * nx, 0.5 * ny) if center is None else center
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    if nz == 1:
        r = np.sqrt((x[None, :] - xc) ** 2 + (y[:, None] - yc) ** 2)
    else:
        zc = 0.5 * nz if zc is None else zc
        z = np.arange(nz, dtype=np.float64)
        r = np.sqrt((x[None, None, :] - xc) ** 2 + (y[None, :, None] - yc) ** 2
                    + (z[:, None, None] - zc) ** 2)
    return 0.5 * (phi_l + phi_v) + 0.5 * (phi_l - phi_v) * np.tanh(2 * (R - r) / W)


def two_droplets(nx: int, ny: int, R0: float, W: float, phi_l: float = 1.0,
                 phi_v: float = 0.0, gap: float | None = None, nz: int = 1) -> np.ndarray:
    """Two droplets side by side on the x axis (the coalescence test, Section 3.3).

    phi = (phi_l+phi_v)/2 + (phi_l-phi_v)/2 [1 - tanh(2 d1/W) - tanh(2 d2/W)],
    d_k = |x - x_k| - R0, centres (L/2 -/+ (R0 + gap/2), L/2[, L/2]); the paper
    uses gap = W.  Returns (ny, nx) for nz == 1, else (nz, ny, nx).
    """
    gap = W if gap is None else gap
    off = R0 + 0.5 * gap
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    xs = (0.5 * nx - off, 0.5 * nx + off)
    if nz == 1:
        d = [np.sqrt((x[None, :] - xk) ** 2 + (y[:, None] - 0.5 * ny) ** 2) - R0 for xk in xs]
    else:
        z = np.arange(nz, dtype=np.float64)
        d = [np.sqrt((x[None, None, :] - xk) ** 2 + (y[None, :, None] - 0.5 * ny) ** 2
                     + (z[:, None, None] - 0.5 * nz) ** 2) - R0 for xk in xs]
    return (0.5 * (phi_l + phi_v) + 0.5 * (phi_l - phi_v)
            * (1.0 - np.tanh(2 * d[0] / W) - np.tanh(2 * d[1] / W)))


def ensemble_case(seed: int) -> dict:
    """One case of the batched droplet ensemble, drawn from default_rng(seed) in
    the order N ~ U{64..512}, R = U(0.15, 0.35) N, rho_l/rho_v = U(1, 100)."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(64, 513))
    r = float(rng.uniform(0.15, 0.35)) * n
    ratio = float(rng.uniform(1.0, 100.0))
    return dict(n=n, R=r, rho_ratio=ratio)


def perturbed_state(shape_q_grid, scale: float, seed: int) -> np.ndarray:
    """Seeded N(0, 1) noise times ``scale`` (used to drive parity cases off
    equilibrium so that every term of the update is exercised)."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(shape_q_grid)


# Parameter sets of the workloads (the paper's notation; phi_l = 1, phi_v = 0).
# Flat interface, 16 x 128 periodic, density ratio 10, equal viscosities
# (tau_g = 1, i.e. nu = 1/6), M = 0.1, alpha = 1, sigma = 1e-3, W = 4.
FLAT_16x128 = dict(shape=(16, 128), W=4.0, M=0.1, alpha=1.0, sigma=1e-3,
                   rho_l=10.0, rho_v=1.0, nu_l=1.0 / 6.0, nu_v=1.0 / 6.0)
# The paper's own flat-interface set: 32 x 128, sigma = 5e-3, nu_v = 0.1.
FLAT_PAPER = dict(shape=(32, 128), W=4.0, M=0.1, alpha=1.0, sigma=5e-3,
                  rho_l=10.0, rho_v=1.0, nu_l=0.1, nu_v=0.1)
# Stationary droplet 1024 x 1024, R = 128, W = 4, sigma = 1e-3, M = 0.05,
# density ratio 10 (or 100), viscosity ratio 10 (nu_l = 1.0, nu_v = 0.1).
DROPLET_1024 = dict(shape=(1024, 1024), R=128.0, W=4.0, M=0.05, alpha=1.0, sigma=1e-3,
                    rho_l=10.0, rho_v=1.0, nu_l=1.0, nu_v=0.1)
# The paper's droplet: 128 x 128, R = 32, parameters of the flat case.
DROPLET_PAPER = dict(shape=(128, 128), R=32.0, W=4.0, M=0.1, alpha=1.0, sigma=5e-3,
                     rho_l=10.0, rho_v=1.0, nu_l=0.1, nu_v=0.1)


# 3D coalescence: 512^3 periodic, D3Q19, two droplets R = 64 whose centres are
# 2R + 3 apart (gap 3), W = 5, density ratio 10, other parameters of the
# 1024^2 droplet.
COALESCENCE_3D = dict(shape=(512, 512, 512), R=64.0, gap=3.0, W=5.0, M=0.05, alpha=1.0,
                      sigma=1e-3, rho_l=10.0, rho_v=1.0, nu_l=1.0, nu_v=0.1)
# Its reduced copy for comparisons with the FP64 oracle: 64^3, R = 8, same W.
COALESCENCE_3D_SMALL = dict(COALESCENCE_3D, shape=(64, 64, 64), R=8.0)
# Two-droplet coalescence of Section 3.3 (512^2, M = 0.1, alpha = 1, sigma = 5e-3,
# W = 8, nu_v = 0.1, centres 2R + W apart) with R = 48, density ratio 10 and
# equal viscosities: the differentiated run.
COALESCENCE_ADJ = dict(shape=(512, 512), R=48.0, W=8.0, M=0.1, alpha=1.0, sigma=5e-3,
                       rho_l=10.0, rho_v=1.0, nu_l=0.1, nu_v=0.1)


def physical(params: dict) -> dict:
    """Strip workload-only keys (shape, R, gap) from a parameter set."""
    return {k: v for k, v in params.items() if k not in ("shape", "R", "gap")}
