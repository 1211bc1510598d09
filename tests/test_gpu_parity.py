"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances:
* FP64 path: every field X within 1e-12 max|X| + 1e-14 max(|f|, |g|) of the
  oracle: 1e-12 relative to the field's own largest magnitude (a node-wise
  relative test is meaningless for populations and velocities that cross
  zero), plus ~100 ulp of the state's magnitude, because FP64 round-off
  enters every field from the O(1) order parameter (near equilibrium g, u and
  mu are orders of magnitude below it);
* FP32 path: phi within 1e-5 absolute and |u| within 1e-6 lattice units of the
  FP64 oracle.

Grids span several CTA strips (128 columns) with ragged edges in x and y, and
the degenerate widths the method allows (a single column, 3 x 4).
"""
import numpy as np
import pytest

from paper_2311_10827_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

RTOL64 = 1e-12


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_10827_gb300 import build, sim
    build.build()
    return sim


def close(a, b, rtol, what, atol=0.0):
    a, b = np.asarray(a), np.asarray(b)
    scale = max(np.abs(b).max(), 1e-300)
    err = np.abs(a - b).max()
    assert err <= rtol * scale + atol, (f"{what}: max err {err:.3e} vs scale {scale:.3e}, "
                                        f"atol {atol:.1e}")
    return err


def pair(gpu, oracle_mod, shape, precision="fp64", **prm):
    return gpu.Simulation(shape, precision=precision, **prm), oracle_mod.Oracle(shape, **prm)


STATE_TOL64 = 1e-14


def compare_all(s, o, rtol, tag=""):
    fg, gg, Sg = s.get_state()
    fo, go, So = o.get_state()
    atol = STATE_TOL64 * max(np.abs(fo).max(), np.abs(go).max())
    close(fg, fo, rtol, tag + "f", atol)
    close(gg, go, rtol, tag + "g", atol)
    close(Sg, So, rtol, tag + "S", atol)
    mg, mo = s.moments(), o.macros()
    for k in ("phi", "mu", "p", "u"):
        close(mg[k], mo[k], rtol, tag + k, atol)


def perturb(o, seed):
    f, g, S = o.get_state()
    g = g + wl.perturbed_state(g.shape, 1e-3, seed)
    S = S + wl.perturbed_state(S.shape, 1e-4, seed + 1)
    return f, g, S


PRM = dict(W=4.0, M=0.05, alpha=1.0, sigma=1e-3, rho_l=10.0, rho_v=1.0, nu_l=1.0, nu_v=0.1)


def test_fp64_flat_interface(gpu, oracle_mod):
    """16 x 128 flat interface (density ratio 10, tau_g = 1, M = 0.1), 300 steps."""
    p = wl.physical(wl.FLAT_16x128)
    s, o = pair(gpu, oracle_mod, (16, 128), **p)
    phi0 = wl.flat_interface(16, 128, 4.0)
    s.init_phi(phi0)
    o.init_phi(phi0)
    compare_all(s, o, RTOL64, "t0 ")
    s.step(300)
    o.step(300)
    compare_all(s, o, RTOL64)


@pytest.mark.parametrize("shape", [(300, 37), (129, 16), (64, 48), (5, 7), (1, 32), (3, 4),
                                   (256, 9)])
def test_fp64_perturbed_droplet(gpu, oracle_mod, shape):
    """Off-equilibrium state (random g and S_prev, body force): every term of
    the update is active."""
    prm = dict(PRM, Gx=1e-6, Gy=-2e-6)
    s, o = pair(gpu, oracle_mod, shape, **prm)
    nx, ny = shape
    o.init_phi(wl.droplet(nx, ny, 0.3 * min(nx, ny) + 1.0, 4.0))
    f, g, S = perturb(o, 5)
    o.set_state(f, g, S, 0)
    s.set_state(f, g, S, 0)
    compare_all(s, o, RTOL64, "t0 ")
    s.step(25)
    o.step(25)
    compare_all(s, o, RTOL64)


def test_fp64_diagnostics_match_oracle(gpu, oracle_mod):
    s, o = pair(gpu, oracle_mod, (200, 50), **PRM)
    phi0 = wl.two_droplets(200, 50, 15.0, 4.0)
    s.init_phi(phi0)
    o.init_phi(phi0)
    s.step(40)
    o.step(40)
    dg, do = s.diagnostics(), o.diag()
    assert np.isclose(dg["sum_phi"], do["sum_phi"], rtol=1e-13)
    for k, kk in (("kinetic_energy", "E"), ("u_max", "umax"), ("budget", "budget")):
        assert np.isclose(dg[k], do[kk], rtol=1e-10), k
    assert np.isclose(dg["mu_min"], do["mu_min"], rtol=1e-11)
    assert np.isclose(dg["mu_max"], do["mu_max"], rtol=1e-11)
    assert dg["step"] == 40 and not dg["nonfinite"]


def test_fp64_phi_budget_on_gpu(gpu, oracle_mod):
    """sum phi^{t+1} = sum phi^t - budget^t to round-off (Eq. sumfeqandF)."""
    s = gpu.Simulation((96, 80), precision="fp64", **PRM)
    o = oracle_mod.Oracle((96, 80), **PRM)
    o.init_phi(wl.droplet(96, 80, 20.0, 4.0))
    f, g, S = perturb(o, 9)
    s.set_state(f, g, S, 0)
    for _ in range(5):
        d0 = s.diagnostics()
        s.step(1)
        d1 = s.diagnostics()
        assert abs(d1["sum_phi"] - (d0["sum_phi"] - d0["budget"])) < 1e-12 * d0["sum_phi"]


@pytest.mark.parametrize("precision,nx", [("fp64", 160), ("fp32", 160), ("fp32", 256)])
def test_graph_and_plain_steps_identical(gpu, precision, nx):
    """lbm_step(n) (CUDA graph of 32 steps) equals n single steps bit for bit
    (nx = 256: full 128-column strips; nx = 160: a ragged last strip)."""
    a = gpu.Simulation((nx, 70), precision=precision, **PRM)
    b = gpu.Simulation((nx, 70), precision=precision, **PRM)
    phi0 = wl.droplet(nx, 70, 20.0, 4.0)
    a.init_phi(phi0)
    b.init_phi(phi0)
    a.step(1)
    b.step(1)  # start the graph from the odd buffer
    a.step(99)
    for _ in range(99):
        b.step(1)
    fa, ga, Sa = a.get_state()
    fb, gb, Sb = b.get_state()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb) and np.array_equal(Sa, Sb)


@pytest.mark.parametrize("precision,nx", [("fp64", 144), ("fp32", 144), ("fp32", 256)])
def test_checkpoint_resume_bit_exact(gpu, precision, nx):
    a = gpu.Simulation((nx, 40), precision=precision, **PRM)
    phi0 = wl.droplet(nx, 40, 12.0, 4.0)
    a.init_phi(phi0)
    a.step(37)
    ck = a.save()
    a.step(50)
    fa, ga, Sa = a.get_state()
    b = gpu.Simulation((nx, 40), precision=precision, **PRM)
    b.load(ck)
    assert b.t == 37
    b.step(50)
    fb, gb, Sb = b.get_state()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb) and np.array_equal(Sa, Sb)
    # a checkpoint of another grid is refused
    c = gpu.Simulation((nx - 4, 40), precision=precision, **PRM)
    from paper_2311_10827_gb300 import capi
    with pytest.raises(capi.LbmError):
        c.load(ck)


@pytest.mark.parametrize("lattice,shape", [("D2Q9", (96, 80)), ("D3Q19", (40, 24, 20))])
def test_fp32_equilibrium_shift_is_exact(gpu, lattice, shape):
    """The FP32 storage's uniform equilibrium shift (moved by lbm_diagnostics)
    is a symmetry of the step: a run re-centred midway agrees with one that
    is not to FP32 rounding, and a checkpoint taken with a shift resumes bit
    for bit."""
    nx, ny = shape[0], shape[1]
    nz = shape[2] if len(shape) > 2 else 1
    prm = dict(PRM, W=5.0) if lattice == "D3Q19" else PRM
    phi0 = wl.droplet(nx, ny, 8.0, prm["W"], nz=nz)
    a = gpu.Simulation(shape, lattice=lattice, precision="fp32", **prm)
    b = gpu.Simulation(shape, lattice=lattice, precision="fp32", **prm)
    a.init_phi(phi0)
    b.init_phi(phi0)
    a.step(150)
    b.step(150)
    a.diagnostics()  # re-centres a's shift (alpha times the mid mu)
    a.step(150)
    b.step(150)
    fa, ga, Sa = a.get_state()
    fb, gb, Sb = b.get_state()
    assert np.abs(fa - fb).max() <= 1e-6 * np.abs(fb).max()
    assert np.abs(a.moments()["phi"] - b.moments()["phi"]).max() <= 1e-6
    ck = a.save()
    a.step(20)
    c = gpu.Simulation(shape, lattice=lattice, precision="fp32", **prm)
    c.load(ck)
    c.step(20)
    for x, y in zip(a.get_state(), c.get_state()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("lattice,shape,precision", [("D2Q9", (144, 50), "fp32"),
                                                    ("D2Q9", (144, 50), "fp64"),
                                                    ("D3Q19", (36, 20, 12), "f16off")])
def test_create_with_caller_buffers(gpu, lattice, shape, precision):
    """A context on caller-owned device memory (torch tensors) steps exactly
    like one that allocates its own state, and leaves the memory to its owner."""
    torch = pytest.importorskip("torch")
    from paper_2311_10827_gb300 import capi, sim
    prm = dict(PRM, W=5.0) if lattice == "D3Q19" else PRM
    params = sim.make_params(precision, **prm)
    lat = capi.LBM_D3Q19 if lattice == "D3Q19" else capi.LBM_D2Q9
    rc, (fb, gb, sb) = capi.lbm_state_bytes(shape, lat, params)
    assert rc == 0
    bufs = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in (fb, fb, gb, gb, sb)]
    rc, h = capi.lbm_create_with_buffers(shape, lat, params, bufs)
    assert rc == 0
    a = sim.Simulation(shape, lattice=lattice, precision=precision, _borrow=h, **prm)
    b = sim.Simulation(shape, lattice=lattice, precision=precision, **prm)
    nx, ny = shape[0], shape[1]
    nz = shape[2] if len(shape) > 2 else 1
    phi0 = wl.droplet(nx, ny, 8.0, prm["W"], nz=nz)
    for s in (a, b):
        s.init_phi(phi0)
        s.step(45)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    capi.lbm_destroy(h)
    torch.cuda.synchronize()
    for t in bufs:            # still the caller's, still usable
        t.zero_()
    torch.cuda.synchronize()
    assert int(bufs[0].sum()) == 0


def test_fused_diagnostics_equal_on_demand(gpu):
    a = gpu.Simulation((130, 60), precision="fp64", diag_every=10, **PRM)
    b = gpu.Simulation((130, 60), precision="fp64", **PRM)
    phi0 = wl.droplet(130, 60, 15.0, 4.0)
    a.init_phi(phi0)
    b.init_phi(phi0)
    a.step(21)      # fused diagnostics at steps 0, 10, 20
    b.step(20)
    da, db = a.last_diagnostics(), b.diagnostics()
    assert da["step"] == 20
    for k in ("sum_phi", "kinetic_energy", "u_max", "mu_min", "mu_max", "budget"):
        assert da[k] == db[k], k


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nonfinite_is_reported(gpu, precision):
    """Host-side fault injection: a NaN population makes the fused diagnostics
    report LBM_ERR_NONFINITE; no device fault is involved."""
    from paper_2311_10827_gb300 import capi
    s = gpu.Simulation((64, 32), precision=precision, diag_every=1, **PRM)
    s.init_phi(wl.droplet(64, 32, 10.0, 4.0))
    s.step(3)
    s.sync()
    capi.check(capi.lbm_debug_poke(s.handle, 0, 3, 64 * 16 + 20, float("nan")))
    rc = capi.lbm_step(s.handle, 2)
    if rc == capi.LBM_OK:
        rc = capi.lbm_sync(s.handle)
    assert rc == capi.LBM_ERR_NONFINITE
    assert s.last_diagnostics()["nonfinite"]


def test_fp32_fused_diagnostics_close_to_on_demand(gpu):
    """The FP32 step's fused diagnostics agree with the on-demand pass."""
    a = gpu.Simulation((256, 64), precision="fp32", diag_every=5, **PRM)
    b = gpu.Simulation((256, 64), precision="fp32", **PRM)
    phi0 = wl.droplet(256, 64, 15.0, 4.0)
    a.init_phi(phi0)
    b.init_phi(phi0)
    a.step(11)
    b.step(10)
    da, db = a.last_diagnostics(), b.diagnostics()
    assert da["step"] == 10
    assert np.isclose(da["sum_phi"], db["sum_phi"], rtol=1e-12)
    for k in ("kinetic_energy", "u_max", "mu_min", "mu_max"):
        assert np.isclose(da[k], db[k], rtol=1e-5), k
    assert abs(da["budget"] - db["budget"]) <= 1e-5 * abs(db["budget"]) + 1e-9


def test_call_order_and_arguments(gpu):
    from paper_2311_10827_gb300 import capi
    s = gpu.Simulation((32, 32), precision="fp32", **PRM)
    assert capi.lbm_step(s.handle, 1) == capi.LBM_ERR_STATE
    assert capi.lbm_step(s.handle, -1) == capi.LBM_ERR_INVALID_ARG
    rc, _ = capi.lbm_last_diagnostics(s.handle)
    assert rc == capi.LBM_ERR_STATE
    s.init_phi(np.full((32, 32), 0.5))
    assert capi.lbm_step(s.handle, 0) == capi.LBM_OK
    assert capi.lbm_debug_poke(s.handle, 2, 0, 0, 0.0) == capi.LBM_ERR_INVALID_ARG


@pytest.mark.parametrize("shape", [(192, 96), (256, 96), (128, 77)])
def test_fp32_against_oracle(gpu, oracle_mod, shape):
    """FP32 path vs the FP64 oracle on a droplet, 2000 steps (widths that are
    multiples of 128 fill every 128-column strip; 192 leaves a ragged one)."""
    s = gpu.Simulation(shape, precision="fp32", **PRM)
    o = oracle_mod.Oracle(shape, **PRM)
    phi0 = wl.droplet(shape[0], shape[1], 24.0, 4.0)
    s.init_phi(phi0)
    o.init_phi(phi0)
    s.step(2000)
    o.step(2000)
    mg, mo = s.moments(), o.macros()
    assert np.abs(mg["phi"] - mo["phi"]).max() < 1e-5
    assert np.abs(mg["u"] - mo["u"]).max() < 1e-6


@pytest.mark.parametrize("shape", [(257, 33), (256, 33), (128, 20), (384, 7), (640, 3)])
def test_fp32_one_step_from_same_state(gpu, oracle_mod, shape):
    """One step from an FP32-representable perturbed state: FP32 rounding only
    (several strips, a single strip, ragged rows, fewer rows than the halo)."""
    s = gpu.Simulation(shape, precision="fp32", **PRM)
    o = oracle_mod.Oracle(shape, **PRM)
    o.init_phi(wl.droplet(shape[0], shape[1], min(shape) / 3 + 1.0, 4.0))
    f, g, S = perturb(o, 21)
    f, g, S = (a.astype(np.float32).astype(np.float64) for a in (f, g, S))
    o.set_state(f, g, S, 0)
    s.set_state(f, g, S, 0)
    s.step(1)
    o.step(1)
    fg, gg, Sg = s.get_state()
    fo, go, So = o.get_state()
    close(fg, fo, 1e-6, "f")
    close(gg, go, 1e-5, "g")
    close(Sg, So, 1e-4, "S")
