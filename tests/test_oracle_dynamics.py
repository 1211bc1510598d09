"""Pins of the oracle's full time step (no GPU).

* exact phi budget per step (Eq. sumfeqandF: sum f^eq = phi, sum F_i = -S);
* a uniform state is a fixed point;
* a uniform body force accelerates the fluid by exactly F per step, with the
  half-force shift of the velocity definition below Eq. GGi;
* a shear wave decays at nu k^2 with nu = cs2 (tau_g - 1/2) (Section 2.3.2),
  second-order convergent, in each bulk phase (linear nu(phi), Eq. vis);
* a small order-parameter wave relaxes at the linearised Cahn-Hilliard rate
  M k^2 (psi''(phi) + kappa k^2) (Eqs. CH_equation3, mobility), second order;
* a phase-field wave is carried by a uniform flow at the flow speed
  (convection as a source, Eq. F_i);
* a brute-force exact-rational re-evaluation of two steps on a 3 x 4 grid
  (push form, different loop structure) pins indexing, wrap and every term.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

from paper_2311_10827_gb300 import workloads as wl

CS2 = 1.0 / 3.0


def _perturbed(O, shape, lat="D2Q9", seed=3, **prm):
    """A droplet state pushed off equilibrium: random g (momentum, pressure)
    and random S_prev, so every term of the update is active."""
    o = O.Oracle(shape, lattice_name=lat, **prm)
    nx, ny = shape[0], shape[1]
    nz = shape[2] if len(shape) > 2 else 1
    phi0 = wl.droplet(nx, ny, 0.3 * min(nx, ny), 4.0, nz=nz)
    o.init_phi(phi0)
    f, g, S = o.get_state()
    g = g + wl.perturbed_state(g.shape, 1e-3, seed)
    S = S + wl.perturbed_state(S.shape, 1e-4, seed + 1)
    o.set_state(f, g, S, 0)
    return o


@pytest.mark.parametrize("lat,shape", [("D2Q9", (24, 20)), ("D3Q19", (10, 8, 6))])
def test_phi_budget_exact(oracle_mod, lat, shape):
    o = _perturbed(oracle_mod, shape, lat, rho_l=10.0, nu_l=0.3, Gx=1e-5)
    for _ in range(6):
        d0 = o.diag()
        o.step(1)
        d1 = o.diag()
        assert abs(d1["sum_phi"] - (d0["sum_phi"] - d0["budget"])) < 1e-13 * d0["sum_phi"]
    assert abs(d0["budget"]) > 1e-6  # the budget term is really exercised


@pytest.mark.parametrize("lat,shape", [("D2Q9", (6, 5)), ("D3Q19", (4, 3, 5))])
def test_uniform_state_is_fixed_point(oracle_mod, lat, shape):
    o = oracle_mod.Oracle(shape, lattice_name=lat, rho_l=10.0)
    o.init_phi(np.full(o.fshape, 0.3))
    f0, g0, _ = o.get_state()
    o.step(20)
    f1, g1, S1 = o.get_state()
    assert np.abs(f1 - f0).max() < 1e-14
    assert np.abs(g1).max() < 1e-18 and np.abs(S1).max() < 1e-18


@pytest.mark.parametrize("lat,shape,phi0", [("D2Q9", (4, 6), 1.0), ("D2Q9", (5, 3), 0.5),
                                            ("D3Q19", (3, 4, 5), 0.25)])
def test_uniform_body_force_newton(oracle_mod, lat, shape, phi0):
    """rho u^n = (n + 1/2) G: momentum grows by exactly F per step."""
    G = (2e-6, -1e-6, 5e-7)
    o = oracle_mod.Oracle(shape, lattice_name=lat, rho_l=10.0, rho_v=1.0, nu_l=0.4, nu_v=0.1,
                          Gx=G[0], Gy=G[1], Gz=G[2])
    o.init_phi(np.full(o.fshape, phi0))
    rho = 1.0 + 9.0 * phi0
    for n in (0, 1, 7, 30):
        o.step(n - o.t)
        u = o.macros()["u"]
        for a in range(o.D):
            assert np.allclose(u[a], (n + 0.5) * G[a] / rho, rtol=1e-12, atol=0)


def _shear_rate(O, L, phi0, nu_l, nu_v):
    o = O.Oracle((2, L), rho_l=10.0, rho_v=1.0, nu_l=nu_l, nu_v=nu_v, sigma=1e-3)
    o.init_phi(np.full((L, 2), phi0))
    f, g, S = o.get_state()
    D, Q, c, w = O.lattice()
    k, U = 2 * np.pi / L, 1e-4
    ux = U * np.sin(k * np.arange(L))[:, None] * np.ones((1, 2))
    rho = 1.0 + 9.0 * phi0
    for i in range(Q):  # g = g^eq(p = 0, u), Eq. G_i with Eq. Siu
        cu = c[i, 0] * ux
        g[i] = rho * w[i] * (cu / CS2 + cu * cu / (2 * CS2 * CS2) - ux * ux / (2 * CS2))
    o.set_state(f, g, S, 0)
    o.step(50)
    a1 = np.abs(o.macros()["u"][0]).max()
    n = 400
    o.step(n)
    a2 = np.abs(o.macros()["u"][0]).max()
    return -np.log(a2 / a1) / (k * k * n)


@pytest.mark.parametrize("phi0", [1.0, 0.0])
def test_shear_wave_viscosity(oracle_mod, phi0):
    nu = 0.05 if phi0 == 1.0 else 0.2
    e16 = _shear_rate(oracle_mod, 16, phi0, 0.05, 0.2) / nu - 1
    e32 = _shear_rate(oracle_mod, 32, phi0, 0.05, 0.2) / nu - 1
    assert abs(e32) < 5e-3
    assert 3.0 < abs(e16 / e32) < 5.0  # second-order convergence to nu k^2


def _ch_rate(O, L):
    o = O.Oracle((L, 2), M=0.1, sigma=5e-3, W=4.0, rho_l=1.0, rho_v=1.0)
    k = 2 * np.pi / L
    o.init_phi(1e-6 * np.cos(k * np.arange(L))[None, :] * np.ones((2, 1)))
    o.step(20)
    a1 = np.abs(o.macros()["phi"]).max()
    lam_c = 0.1 * k * k * (2 * o.beta + o.kappa * k * k)  # psi''(phi_v) = 2 beta
    n = int(2.0 / lam_c)
    o.step(n)
    a2 = np.abs(o.macros()["phi"]).max()
    return -np.log(a2 / a1) / n / lam_c - 1


def test_cahn_hilliard_relaxation_rate(oracle_mod):
    e16, e32 = _ch_rate(oracle_mod, 16), _ch_rate(oracle_mod, 32)
    assert abs(e32) < 5e-3
    assert 3.0 < abs(e16 / e32) < 5.0


def test_convection_moves_pattern_downstream(oracle_mod):
    """A small phi wave around phi_v in a uniform flow U x^ moves by U t
    (the force -phi grad mu is second order in the amplitude there)."""
    L, U, n = 32, 2e-3, 2000
    o = oracle_mod.Oracle((L, 2), M=0.02, sigma=1e-3, rho_l=1.0, rho_v=1.0, nu_l=0.1, nu_v=0.1)
    k = 2 * np.pi / L
    x = np.arange(L)
    o.init_phi(1e-6 * np.cos(k * x)[None, :] * np.ones((2, 1)))
    f, g, S = o.get_state()
    D, Q, c, w = oracle_mod.lattice()
    for i in range(Q):
        cu = c[i, 0] * U
        g[i] = w[i] * (cu / CS2 + cu * cu / (2 * CS2 * CS2) - U * U / (2 * CS2))
    o.set_state(f, g, S, 0)
    o.step(n)
    phi = o.macros()["phi"][0]
    shift = -np.angle(np.sum(phi * np.exp(-1j * k * x))) / k
    assert abs(shift - U * n) < 0.02 * U * n


# ---------------------------------------------------------------- brute force

def _exact_two_steps(nx, ny, phi0, gpert, Sp, P):
    """Exact rational arithmetic, push form, node dictionaries."""
    vel = [(0, 0), (0, -1), (1, 0), (0, 1), (-1, 0), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    wt = [Fr(4, 9)] + [Fr(1, 9)] * 4 + [Fr(1, 36)] * 4
    cs2 = Fr(1, 3)
    W, sig, M, al = Fr(P["W"]), Fr(P["sigma"]), Fr(P["M"]), Fr(P["alpha"])
    rl, rv, nl, nv = Fr(P["rho_l"]), Fr(P["rho_v"]), Fr(P["nu_l"]), Fr(P["nu_v"])
    Gb = (Fr(P["Gx"]), Fr(P["Gy"]))
    kap = 3 * W * sig / 2
    bet = 12 * sig / W
    tf = Fr(1, 2) + M / (cs2 * al)
    nodes = [(x, y) for y in range(ny) for x in range(nx)]

    def sh(p, v):
        return ((p[0] + v[0]) % nx, (p[1] + v[1]) % ny)

    def mu_of(phi):
        out = {}
        for p in nodes:
            lap = sum(2 * wt[i] * (phi[sh(p, vel[i])] - phi[p]) for i in range(1, 9)) / cs2
            out[p] = 4 * bet * (phi[p] - 1) * phi[p] * (phi[p] - Fr(1, 2)) - kap * lap
        return out

    def grad(fld, p):
        gx = sum(wt[i] * vel[i][0] * fld[sh(p, vel[i])] for i in range(1, 9)) / cs2
        gy = sum(wt[i] * vel[i][1] * fld[sh(p, vel[i])] for i in range(1, 9)) / cs2
        return gx, gy

    phi = {p: Fr(phi0[p[1], p[0]]) for p in nodes}
    mu = mu_of(phi)
    f = {}
    g = {}
    for p in nodes:
        for i in range(9):
            f[p, i] = (phi[p] - (1 - wt[0]) * al * mu[p]) if i == 0 else wt[i] * al * mu[p]
            g[p, i] = Fr(gpert[i, p[1], p[0]])
    Sprev = {p: Fr(Sp[p[1], p[0]]) for p in nodes}
    for _ in range(2):
        phi = {p: sum(f[p, i] for i in range(9)) for p in nodes}
        mu = mu_of(phi)
        fn, gn, Snew = {}, {}, {}
        for p in nodes:
            gp, gm = grad(phi, p), grad(mu, p)
            rho = rv + phi[p] * (rl - rv)
            nu = nv + phi[p] * (nl - nv)
            tg = Fr(1, 2) + nu / cs2
            F = (-phi[p] * gm[0] + Gb[0], -phi[p] * gm[1] + Gb[1])
            gr = ((rl - rv) * gp[0], (rl - rv) * gp[1])
            ux = (sum(vel[i][0] * g[p, i] for i in range(9)) + F[0] / 2) / rho
            uy = (sum(vel[i][1] * g[p, i] for i in range(9)) + F[1] / 2) / rho
            uu = ux * ux + uy * uy
            ugr = ux * gr[0] + uy * gr[1]
            s0 = wt[0] * (-uu / (2 * cs2))
            pr = cs2 / (1 - wt[0]) * (sum(g[p, i] for i in range(1, 9)) + ugr / 2 + rho * s0)
            S = ux * gp[0] + uy * gp[1]
            Snew[p] = S
            for i in range(9):
                cx, cy = vel[i]
                cc = cx * cx + cy * cy
                b = -1 + (cc - 2 * cs2) / (2 * cs2)
                Fi = wt[i] * S * b
                Fo = wt[i] * Sprev[p] * b
                feq = (phi[p] - (1 - wt[0]) * al * mu[p]) if i == 0 else wt[i] * al * mu[p]
                fstar = f[p, i] - (f[p, i] - feq) / tf + Fi + (Fi - Fo) / 2
                cu = cx * ux + cy * uy
                si = wt[i] * (cu / cs2 + cu * cu / (2 * cs2 * cs2) - uu / (2 * cs2))
                geq = pr / cs2 * (wt[i] - (1 if i == 0 else 0)) + rho * si
                cF = cx * F[0] + cy * F[1]
                cg = cx * gr[0] + cy * gr[1]
                Gi = (1 - 1 / (2 * tg)) * wt[i] * (ugr + cF / cs2 + (cu * cg - cs2 * ugr) / cs2)
                gstar = g[p, i] - (g[p, i] - geq) / tg + Gi
                fn[sh(p, vel[i]), i] = fstar
                gn[sh(p, vel[i]), i] = gstar
        f, g, Sprev = fn, gn, Snew
    F_ = np.array([[[float(f[(x, y), i]) for x in range(nx)] for y in range(ny)] for i in range(9)])
    G_ = np.array([[[float(g[(x, y), i]) for x in range(nx)] for y in range(ny)] for i in range(9)])
    S_ = np.array([[float(Sprev[(x, y)]) for x in range(nx)] for y in range(ny)])
    return F_, G_, S_


def test_brute_force_exact_rational(oracle_mod):
    nx, ny = 3, 4
    rng = np.random.default_rng(11)
    P = dict(W=4.0, sigma=1e-2, M=0.1, alpha=1.0, rho_l=10.0, rho_v=1.0, nu_l=0.3, nu_v=0.1,
             Gx=1e-4, Gy=-2e-4)
    phi0 = rng.uniform(0.0, 1.0, (ny, nx))
    gp = rng.normal(size=(9, ny, nx)) * 1e-3
    Sp = rng.normal(size=(ny, nx)) * 1e-3
    o = oracle_mod.Oracle((nx, ny), **P)
    o.init_phi(phi0)
    f, _, _ = o.get_state()
    o.set_state(f, gp, Sp, 0)
    o.step(2)
    fo, go, So = o.get_state()
    fe, ge, Se = _exact_two_steps(nx, ny, phi0, gp, Sp, P)
    assert np.abs(fo - fe).max() < 1e-14
    assert np.abs(go - ge).max() < 1e-14 * max(1.0, np.abs(ge).max())
    assert np.abs(So - Se).max() < 1e-14
    assert np.abs(ge).max() > 1e-4 and np.abs(Se).max() > 1e-4


def _translating_slab(O, U, steps, ny=64, ratio=10.0):
    """A flat slab (Eq. flatinitial, interfaces normal to y, density ratio
    `ratio`, tau_g = 1 in both phases) relaxed at rest for 3000 steps, then
    given the uniform velocity (0, U): g = g^eq(p, rho(phi), U) from the
    relaxed pressure, S_prev = U.grad(phi).  Returns (displacement of the
    slab / (U t), max |u_y - U| / U, pressure range, the largest
    cs2/(1 - w0) |u.grad(rho)| / 2 of the final state)."""
    prm = dict(W=4.0, M=0.1, alpha=1.0, sigma=1e-3, rho_l=ratio, rho_v=1.0,
               nu_l=1.0 / 6.0, nu_v=1.0 / 6.0)
    o = O.Oracle((2, ny), **prm)
    o.init_phi(wl.flat_interface(2, ny, 4.0))
    o.step(3000)
    m = o.macros()
    f, g, S = o.get_state()
    gp = o.grad(m["phi"])
    for y in range(ny):
        for x in range(2):
            rho = 1.0 + (ratio - 1.0) * m["phi"][y, x]
            g[:, y, x] = O.node_geq(m["p"][y, x], rho, (0.0, U))
            S[y, x] = U * gp[1, y, x]
    o.set_state(f, g, S, 0)

    def centroid(phi):  # periodic: phase of the first Fourier mode of the profile
        z = (phi[:, 0] * np.exp(2j * np.pi * np.arange(ny) / ny)).sum()
        return np.angle(z) / (2 * np.pi) * ny

    c0 = centroid(m["phi"])
    o.step(steps)
    m = o.macros()
    disp = (centroid(m["phi"]) - c0 + 0.5 * ny) % ny - 0.5 * ny
    uy = m["u"][1][:, 0]
    p = m["p"][:, 0]
    grho = (ratio - 1.0) * o.grad(m["phi"])[1][:, 0]
    term = (1.0 / 3.0) / (1.0 - 4.0 / 9.0) * 0.5 * np.abs(uy * grho).max()
    return disp / (U * steps), np.abs(uy - U).max() / U, p.max() - p.min(), term


def test_translating_slab_pins_pressure_recovery(oracle_mod):
    """Galilean invariance of the macroscopic equations the scheme recovers
    (Section 2: incompressible Navier-Stokes with the surface force, and the
    Cahn-Hilliard equation with convection): a flat equilibrium interface
    moving with a uniform velocity U normal to it is an exact solution with
    u = U and uniform p.  Only the u.grad(rho)/2 term of the pressure
    recovery below Eq. GGi carries the density jump into p when u crosses
    the interfaces (it is zero in every other pin: static states, rho_l =
    rho_v, or flows along the interfaces).  At U = 1e-3 and density ratio 10
    the slab must move at U within 3%, u stay within 20% of U, and p stay
    uniform to a third of that term's largest value."""
    U = 1e-3
    ratio, dev_u, p_range, term = _translating_slab(oracle_mod, U, 2000)
    assert abs(ratio - 1.0) < 0.03, ratio
    assert dev_u < 0.2, dev_u
    assert p_range < term / 3.0, (p_range, term)


@pytest.mark.parametrize("coef", ["0.0", "1.0", "-0.5"])
def test_translating_slab_fails_with_a_wrong_pressure_term(oracle_mod, coef, tmp_path,
                                                          monkeypatch):
    """The pin above is sharp: the oracle rebuilt with the u.grad(rho) term
    dropped, doubled or sign-flipped (the only change) fails it."""
    import subprocess
    so = str(tmp_path / "libwb_oracle_variant.so")
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", f"-DWBO_P_UGR={coef}",
                    "-o", so, oracle_mod._SRC, "-lm"], check=True)
    monkeypatch.setattr(oracle_mod, "_LIB", so)
    monkeypatch.setattr(oracle_mod, "_lib", None)
    monkeypatch.setattr(oracle_mod, "build", lambda force=False: so)
    with np.errstate(all="ignore"):
        ratio, dev_u, p_range, term = _translating_slab(oracle_mod, 1e-3, 2000)
    ok = abs(ratio - 1.0) < 0.03 and dev_u < 0.2 and p_range < term / 3.0
    assert not ok, (coef, ratio, dev_u, p_range, term)
