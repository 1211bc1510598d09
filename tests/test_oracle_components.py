"""Pins of the oracle's building blocks against what the paper and the
mathematics fix (no GPU).

Each check is chosen so that a plausible slip (a dropped term, a wrong sign,
a wrong weight or index) fails it:
* lattice: the isotropy moments that make Eqs. gradient/Laplace and the CE
  analysis hold (sum w = 1, sum w c = 0, sum w c c = cs2 I, 4th-order tensor);
* stencils: exact discrete Fourier symbols of Eqs. gradient and Laplace;
* parameters: Eqs. beta, suiface_tension and mobility, plus the surface
  tension as the excess free energy of the tanh profile (Eq. energy_function);
* chemical potential: d psi/d phi of Eq. bulk_energy by finite differences;
* single-node moments: Eq. sumfeqandF for f^eq and F_i; the moments of g^eq
  and G_i that the pressure/velocity recovery below Eq. GGi relies on.
"""
import itertools

import numpy as np
import pytest

CS2 = 1.0 / 3.0


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_lattice_isotropy(oracle_mod, lat):
    D, Q, c, w = oracle_mod.lattice(lat)
    c = c[:, :D].astype(float)
    assert Q == (9 if lat == "D2Q9" else 19)
    # distinct velocities, each with its opposite
    assert len({tuple(v) for v in c}) == Q
    for v in c:
        assert any(np.array_equal(-v, u) for u in c)
    assert np.isclose(w.sum(), 1.0, atol=1e-15)
    assert np.allclose(w @ c, 0.0, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), CS2 * np.eye(D), atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0.0, atol=1e-15)
    d = np.eye(D)
    iso4 = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                       + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso4, atol=1e-15)


def test_d2q9_matches_paper_velocity_formula(oracle_mod):
    """Eq. eq:ci: c_1..4 = (cos((i-2)pi/2), sin((i-2)pi/2)); c_5..8 along
    (i-5) pi/2 + pi/4 (length sqrt 2, reading R6); weights 4/9, 1/9, 1/36."""
    D, Q, c, w = oracle_mod.lattice("D2Q9")
    expect = [(0, 0), (0, -1), (1, 0), (0, 1), (-1, 0), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    assert [tuple(v[:2]) for v in c] == expect
    assert np.allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, atol=0)


def _grid(oracle_mod, shape, lat="D2Q9"):
    return oracle_mod.Oracle(shape, lattice_name=lat)


@pytest.mark.parametrize("kx,ky", [(1, 0), (0, 2), (3, 1), (2, 5)])
def test_gradient_symbol_2d(oracle_mod, kx, ky):
    """Eq. gradient on exp(i k.x): the D2Q9 stencil's exact symbol is
    i[sin(a)(2 + cos b)/3, sin(b)(2 + cos a)/3] with a = k_x, b = k_y."""
    nx, ny = 16, 12
    o = _grid(oracle_mod, (nx, ny))
    a, b = 2 * np.pi * kx / nx, 2 * np.pi * ky / ny
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    ph = a * x + b * y
    gs = o.grad(np.sin(ph))
    sx = np.sin(a) * (2 + np.cos(b)) / 3
    sy = np.sin(b) * (2 + np.cos(a)) / 3
    assert np.allclose(gs[0], sx * np.cos(ph), atol=1e-14)
    assert np.allclose(gs[1], sy * np.cos(ph), atol=1e-14)


@pytest.mark.parametrize("kx,ky", [(1, 0), (0, 2), (3, 1), (2, 5)])
def test_laplacian_symbol_2d(oracle_mod, kx, ky):
    """Eq. Laplace on a plane wave: symbol
    (2/3)[2 cos a + 2 cos b + cos a cos b - 5] (-> -(a^2 + b^2) as k -> 0)."""
    nx, ny = 16, 12
    o = _grid(oracle_mod, (nx, ny))
    a, b = 2 * np.pi * kx / nx, 2 * np.pi * ky / ny
    ph = a * np.arange(nx)[None, :] + b * np.arange(ny)[:, None]
    lam = (2.0 / 3.0) * (2 * np.cos(a) + 2 * np.cos(b) + np.cos(a) * np.cos(b) - 5.0)
    assert np.allclose(o.lap(np.cos(ph)), lam * np.cos(ph), atol=1e-14)


def test_stencils_second_order(oracle_mod):
    """The isotropic stencils are second-order accurate: halving the
    wavenumber cuts the relative symbol error by ~4."""
    errs_g, errs_l = [], []
    for n in (16, 32, 64):
        o = _grid(oracle_mod, (n, n))
        a = b = 2 * np.pi / n
        ph = a * np.arange(n)[None, :] + b * np.arange(n)[:, None]
        g = o.grad(np.sin(ph))[0]
        errs_g.append(np.abs(g - a * np.cos(ph)).max() / a)
        lap = o.lap(np.cos(ph))
        errs_l.append(np.abs(lap + (a * a + b * b) * np.cos(ph)).max() / (a * a + b * b))
    for e in (errs_g, errs_l):
        assert 3.6 < e[0] / e[1] < 4.4 and 3.6 < e[1] / e[2] < 4.4


def test_gradient_symbol_3d(oracle_mod):
    n = 8
    o = _grid(oracle_mod, (n, n, n), "D3Q19")
    a, b, cz = 2 * np.pi * 1 / n, 2 * np.pi * 2 / n, 2 * np.pi * 3 / n
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ph = a * x + b * y + cz * z
    gs = o.grad(np.sin(ph))
    # D3Q19: face weight 1/18, edge weight 1/36
    sx = 3 * np.sin(a) * (2 / 18 + 4 / 36 * (np.cos(b) + np.cos(cz)))
    assert np.allclose(gs[0], sx * np.cos(ph), atol=1e-14)
    lam = 6 * (2 / 18 * (np.cos(a) + np.cos(b) + np.cos(cz) - 3)
               + 4 / 36 * (np.cos(a) * np.cos(b) + np.cos(a) * np.cos(cz)
                           + np.cos(b) * np.cos(cz) - 3))
    assert np.allclose(o.lap(np.cos(ph)), lam * np.cos(ph), atol=1e-14)


@pytest.mark.parametrize("W,sigma", [(4.0, 1e-3), (4.0, 5e-3), (5.0, 1e-3), (8.0, 5e-3)])
def test_kappa_beta_roundtrip(oracle_mod, W, sigma):
    """Eq. beta and Eq. suiface_tension both hold for the derived (kappa, beta)."""
    for phil, phiv in ((1.0, 0.0), (1.0, -1.0)):
        k, b = oracle_mod.kappa_beta(W, sigma, phil, phiv)
        d = abs(phil - phiv)
        assert np.isclose(b, 8 * k / (W * W * d * d), rtol=1e-14)
        assert np.isclose(d ** 3 / 6 * np.sqrt(2 * k * b), sigma, rtol=1e-14)


def test_surface_tension_is_excess_energy(oracle_mod):
    """Independent of the printed sigma formula: the excess free energy of the
    planar equilibrium (Eq. energy_function) integrated numerically,
    sigma = int kappa |phi'|^2 dz, with the profile of Eq. flatinitial, whose
    width W must solve psi'(phi) = kappa phi'' (then mu = 0)."""
    W, sigma = 4.0, 5e-3
    k, b = oracle_mod.kappa_beta(W, sigma)
    z = np.linspace(-40, 40, 400001)
    phi = 0.5 + 0.5 * np.tanh(2 * z / W)
    dphi = (1.0 / W) / np.cosh(2 * z / W) ** 2
    assert np.isclose(np.trapezoid(k * dphi ** 2, z), sigma, rtol=1e-8)
    # the tanh profile with width W is the equilibrium: dpsi - kappa phi'' = 0
    d2phi = -(4.0 / W ** 2) * np.tanh(2 * z / W) / np.cosh(2 * z / W) ** 2
    mu = np.array([oracle_mod.dpsi(b, p) for p in phi[::1000]]) - k * d2phi[::1000]
    assert np.abs(mu).max() < 1e-15


def test_dpsi_is_derivative_of_psi(oracle_mod):
    """Bulk term of Eq. chemical_potencial = d/dphi of Eq. bulk_energy."""
    beta = 3e-3
    for phil, phiv in ((1.0, 0.0), (1.0, -1.0), (0.8, 0.1)):
        for phi in np.linspace(-0.3, 1.3, 17):
            h = 1e-5
            fd = (oracle_mod.psi(beta, phi + h, phil, phiv)
                  - oracle_mod.psi(beta, phi - h, phil, phiv)) / (2 * h)
            assert np.isclose(oracle_mod.dpsi(beta, phi, phil, phiv), fd, rtol=1e-8, atol=1e-11)


def test_mu_field(oracle_mod):
    """mu = dpsi(phi) - kappa lap_h(phi) on a plane wave (Eq. chemical_potencial
    with the Laplace symbol)."""
    n = 16
    o = oracle_mod.Oracle((n, n), W=4.0, sigma=2e-3)
    a = 2 * np.pi * 2 / n
    phi = 0.5 + 0.3 * np.cos(a * np.arange(n))[None, :] * np.ones((n, 1))
    lam = (2.0 / 3.0) * (2 * np.cos(a) + 2 + np.cos(a) - 5.0)
    lap = lam * (phi - 0.5)
    bulk = np.vectorize(lambda p: oracle_mod.dpsi(o.beta, p))(phi)
    assert np.allclose(o.mu_of(phi), bulk - o.kappa * lap, atol=1e-15)


def test_mobility_and_viscosity_relations(oracle_mod):
    """Eq. mobility: M = cs2 alpha (tau_f - 1/2); and the inverse when tau_f is
    given (alpha derived)."""
    for M, alpha in ((0.1, 1.0), (0.05, 1.0), (0.02, 0.5)):
        o = oracle_mod.Oracle((4, 4), M=M, alpha=alpha)
        assert np.isclose(CS2 * o.alpha * (o.tau_f - 0.5), M, rtol=1e-14)
    o = oracle_mod.Oracle((4, 4), M=0.1, tau_f=1.0)
    assert np.isclose(o.alpha, 0.1 / (CS2 * 0.5), rtol=1e-14)


def _rng_cases(n=20, seed=7):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        yield rng


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_feq_and_F_moments(oracle_mod, lat):
    """Eq. sumfeqandF: sum f^eq = phi, sum c f^eq = 0, sum cc f^eq = cs2 alpha mu I;
    sum F = -u.grad(phi), sum c F = 0, sum cc F = 0."""
    D, Q, c, w = oracle_mod.lattice(lat)
    c = c[:, :D].astype(float)
    for rng in _rng_cases():
        phi, mu, alpha, S = rng.uniform(-0.2, 1.2), rng.normal() * 1e-3, rng.uniform(0.5, 2), rng.normal()
        fe = oracle_mod.node_feq(phi, mu, alpha, lat)
        assert np.isclose(fe.sum(), phi, atol=1e-15)
        assert np.allclose(fe @ c, 0, atol=1e-16)
        assert np.allclose(np.einsum("i,ia,ib->ab", fe, c, c), CS2 * alpha * mu * np.eye(D), atol=1e-16)
        F = oracle_mod.node_F(S, lat)
        assert np.isclose(F.sum(), -S, atol=1e-15)
        assert np.allclose(F @ c, 0, atol=1e-15)
        assert np.allclose(np.einsum("i,ia,ib->ab", F, c, c), 0, atol=1e-15)


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_geq_moments(oracle_mod, lat):
    """Eqs. G_i and Siu: sum g^eq = 0, sum c g^eq = rho u, sum cc g^eq = p I + rho u u
    (the moments behind the recovery of u and p below Eq. GGi)."""
    D, Q, c, w = oracle_mod.lattice(lat)
    c = c[:, :D].astype(float)
    for rng in _rng_cases():
        p, rho, u = rng.normal() * 1e-2, rng.uniform(1, 100), rng.normal(size=D) * 0.05
        ge = oracle_mod.node_geq(p, rho, u, lat)
        assert np.isclose(ge.sum(), 0, atol=1e-14)
        assert np.allclose(ge @ c, rho * u, rtol=1e-13, atol=1e-14)
        assert np.allclose(np.einsum("i,ia,ib->ab", ge, c, c), p * np.eye(D) + rho * np.outer(u, u),
                           rtol=1e-12, atol=1e-14)
        # pressure recovery formula inverts g^eq exactly (F = 0, grad rho = 0)
        s0 = w[0] * (-(u @ u) / (2 * CS2))
        p_rec = CS2 / (1 - w[0]) * (ge[1:].sum() + rho * s0)
        assert np.isclose(p_rec, p, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_forceG_moments(oracle_mod, lat):
    """Eq. GGi (reading R4): sum G = (1-1/2tau) u.grad rho,
    sum c G = (1-1/2tau) F, sum cc G = (1-1/2tau) cs2 [(u.grad rho) I + u grad rho + grad rho u]."""
    D, Q, c, w = oracle_mod.lattice(lat)
    c = c[:, :D].astype(float)
    for rng in _rng_cases():
        tau = rng.uniform(0.55, 3.0)
        u, gr, F = rng.normal(size=D) * 0.05, rng.normal(size=D), rng.normal(size=D) * 1e-3
        G = oracle_mod.node_G(tau, u, gr, F, lat)
        k = 1 - 1 / (2 * tau)
        assert np.isclose(G.sum(), k * (u @ gr), atol=1e-15)
        assert np.allclose(G @ c, k * F, atol=1e-15)
        want = k * CS2 * ((u @ gr) * np.eye(D) + np.outer(u, gr) + np.outer(gr, u))
        assert np.allclose(np.einsum("i,ia,ib->ab", G, c, c), want, atol=1e-15)


def test_source_coefficients_d2q9(oracle_mod):
    """F_i / (w_i S) = -2, -1/2, 1 for rest, axis, diagonal (Eq. F_i with D = 2)."""
    F = oracle_mod.node_F(1.0, "D2Q9")
    D, Q, c, w = oracle_mod.lattice("D2Q9")
    b = F / w
    assert np.allclose(b, [-2] + [-0.5] * 4 + [1] * 4, atol=1e-15)


def test_combinations_cover_all_pairs():
    # guard for the parametrisations above: every lattice is tested
    assert set(itertools.chain(["D2Q9", "D3Q19"])) == {"D2Q9", "D3Q19"}
