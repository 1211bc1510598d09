"""D3Q19 path (the 3D form of the method on the 19-velocity lattice) against
the FP64 oracle, through the C ABI.  Same tolerances as the 2D parity tests.
Grids are ragged against the 32 x 8 column tiles and the z marching."""
import numpy as np
import pytest

from paper_2311_10827_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

PRM = dict(W=5.0, M=0.05, alpha=1.0, sigma=1e-3, rho_l=10.0, rho_v=1.0, nu_l=1.0, nu_v=0.1)


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_10827_gb300 import build, sim
    build.build()
    return sim


def close(a, b, rtol, atol, what):
    err = np.abs(np.asarray(a) - np.asarray(b)).max()
    scale = np.abs(b).max()
    assert err <= rtol * scale + atol, f"{what}: err {err:.3e} scale {scale:.3e}"


def perturbed(O, shape, prm, seed):
    o = O.Oracle(shape, lattice_name="D3Q19", **prm)
    nx, ny, nz = shape
    o.init_phi(wl.two_droplets(nx, ny, min(shape) / 4 + 1.0, 5.0, nz=nz))
    f, g, S = o.get_state()
    g = g + wl.perturbed_state(g.shape, 1e-3, seed)
    S = S + wl.perturbed_state(S.shape, 1e-4, seed + 1)
    o.set_state(f, g, S, 0)
    return o, (f, g, S)


@pytest.mark.parametrize("shape", [(16, 12, 10), (33, 9, 7), (40, 24, 5), (8, 8, 3)])
def test_fp64_d3q19_parity(gpu, oracle_mod, shape):
    prm = dict(PRM, Gx=1e-6, Gz=-2e-6)
    o, st = perturbed(oracle_mod, shape, prm, 3)
    s = gpu.Simulation(shape, lattice="D3Q19", precision="fp64", **prm)
    s.set_state(*st, 0)
    s.step(8)
    o.step(8)
    fg, gg, Sg = s.get_state()
    fo, go, So = o.get_state()
    atol = 1e-14 * max(np.abs(fo).max(), np.abs(go).max())
    close(fg, fo, 1e-12, atol, "f")
    close(gg, go, 1e-12, atol, "g")
    close(Sg, So, 1e-12, atol, "S")
    mg, mo = s.moments(), o.macros()
    for k in ("phi", "mu", "p", "u"):
        close(mg[k], mo[k], 1e-12, atol, k)
    dg, do = s.diagnostics(), o.diag()
    assert np.isclose(dg["sum_phi"], do["sum_phi"], rtol=1e-13)
    assert np.isclose(dg["kinetic_energy"], do["E"], rtol=1e-10)


def test_fp64_d3q19_init_and_budget(gpu, oracle_mod):
    shape = (24, 20, 16)
    phi0 = wl.droplet(24, 20, 6.0, 5.0, nz=16)
    s = gpu.Simulation(shape, lattice="D3Q19", precision="fp64", **PRM)
    o = oracle_mod.Oracle(shape, lattice_name="D3Q19", **PRM)
    s.init_phi(phi0)
    o.init_phi(phi0)
    fg, _, _ = s.get_state()
    fo, _, _ = o.get_state()
    close(fg, fo, 1e-14, 0.0, "f at t=0")
    for _ in range(3):
        d0 = s.diagnostics()
        s.step(1)
        d1 = s.diagnostics()
        assert abs(d1["sum_phi"] - (d0["sum_phi"] - d0["budget"])) < 1e-12 * d0["sum_phi"]


def test_fp32_d3q19_one_step(gpu, oracle_mod):
    shape = (40, 24, 12)
    o, (f, g, S) = perturbed(oracle_mod, shape, PRM, 8)
    f, g, S = (a.astype(np.float32).astype(np.float64) for a in (f, g, S))
    o.set_state(f, g, S, 0)
    s = gpu.Simulation(shape, lattice="D3Q19", precision="fp32", **PRM)
    s.set_state(f, g, S, 0)
    s.step(1)
    o.step(1)
    fg, gg, Sg = s.get_state()
    fo, go, So = o.get_state()
    close(fg, fo, 1e-6, 0.0, "f")
    close(gg, go, 1e-5, 0.0, "g")
    close(Sg, So, 1e-4, 0.0, "S")


def test_fp32_d3q19_coalescence_64(gpu, oracle_mod):
    """Two droplets, 64^3, R = 8, W = 5 (the 3D coalescence case scaled to the
    oracle), 120 steps: FP32 within 1e-5 (phi) and 1e-6 (u) of the oracle."""
    shape = (64, 64, 64)
    phi0 = wl.two_droplets(64, 64, 8.0, 5.0, gap=3.0, nz=64)
    s = gpu.Simulation(shape, lattice="D3Q19", precision="fp32", **PRM)
    o = oracle_mod.Oracle(shape, lattice_name="D3Q19", **PRM)
    s.init_phi(phi0)
    o.init_phi(phi0)
    s.step(120)
    o.step(120)
    mg, mo = s.moments(), o.macros()
    assert np.abs(mg["phi"] - mo["phi"]).max() < 1e-5
    assert np.abs(mg["u"] - mo["u"]).max() < 1e-6


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_d3q19_graph_and_checkpoint(gpu, precision):
    shape = (36, 20, 18)
    phi0 = wl.droplet(36, 20, 6.0, 5.0, nz=18)
    a = gpu.Simulation(shape, lattice="D3Q19", precision=precision, **PRM)
    b = gpu.Simulation(shape, lattice="D3Q19", precision=precision, **PRM)
    a.init_phi(phi0)
    b.init_phi(phi0)
    a.step(70)
    for _ in range(35):
        b.step(1)
    ck = b.save()
    b.step(35)
    fa, ga, Sa = a.get_state()
    fb, gb, Sb = b.get_state()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb) and np.array_equal(Sa, Sb)
    c = gpu.Simulation(shape, lattice="D3Q19", precision=precision, **PRM)
    c.load(ck)
    c.step(35)
    fc, gc, Sc = c.get_state()
    assert np.array_equal(fa, fc) and np.array_equal(ga, gc) and np.array_equal(Sa, Sc)
