"""D3Q19 with populations stored as 16-bit offsets from their equilibria
(FP16 / BF16, FP32 arithmetic) against the FP64 oracle and the FP64 GPU path.

The only approximation of the format is the rounding of each offset
(f_i - f_i^eq, g_i - g_i^eq) to the 16-bit format: half an ulp is 2^-11 of
the offset in FP16 and 2^-8 in BF16 (EPS below).  The state's equilibrium
part comes from FP32 macroscopic fields, and the rest population keeps
phi's FP32 rounding residual, so the bounds below are stated in units of
EPS times the size of the non-equilibrium populations."""
import numpy as np
import pytest

from paper_2311_10827_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

PRM = dict(W=5.0, M=0.05, alpha=1.0, sigma=1e-3, rho_l=10.0, rho_v=1.0, nu_l=1.0, nu_v=0.1)
EPS = {"f16off": 2.0 ** -11, "bf16off": 2.0 ** -8}
CODECS = ["f16off", "bf16off"]


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_10827_gb300 import build, sim
    build.build()
    return sim


def perturbed(O, shape, prm, seed):
    o = O.Oracle(shape, lattice_name="D3Q19", **prm)
    nx, ny, nz = shape
    o.init_phi(wl.two_droplets(nx, ny, min(shape) / 4 + 1.0, 5.0, nz=nz))
    f, g, S = o.get_state()
    g = g + wl.perturbed_state(g.shape, 1e-3, seed)
    f = f + wl.perturbed_state(f.shape, 1e-4, seed + 2)
    S = S + wl.perturbed_state(S.shape, 1e-4, seed + 1)
    return f, g, S


@pytest.mark.parametrize("codec", CODECS)
def test_offsets_state_round_trip(gpu, oracle_mod, codec):
    """set_state then get_state: every population comes back within one
    rounding of its offset (at most twice the largest moving population) and
    the FP32 rounding of the rest population's high word."""
    shape = (40, 20, 9)
    f, g, S = perturbed(oracle_mod, shape, PRM, 5)
    s = gpu.Simulation(shape, lattice="D3Q19", precision=codec, **PRM)
    s.set_state(f, g, S, 0)
    f2, g2, S2 = s.get_state()
    eps = EPS[codec]
    fmov = np.abs(f[1:]).max()
    assert np.abs(f2[1:] - f[1:]).max() <= 2 * eps * fmov
    assert np.abs(f2[0] - f[0]).max() <= 2 * eps * fmov + 2 ** -24 * np.abs(f[0]).max()
    assert np.abs(g2 - g).max() <= 4 * eps * np.abs(g).max()
    assert np.abs(S2 - S).max() <= 2 ** -24 * np.abs(S).max()


@pytest.mark.parametrize("codec", CODECS)
def test_offsets_one_step_vs_oracle(gpu, oracle_mod, codec):
    """One step from a state the format holds exactly (the round trip of a
    perturbed state) against the oracle's FP64 step: within a few roundings
    of the offsets plus FP32 arithmetic."""
    shape = (40, 24, 12)
    f, g, S = perturbed(oracle_mod, shape, PRM, 8)
    s = gpu.Simulation(shape, lattice="D3Q19", precision=codec, **PRM)
    s.set_state(f, g, S, 0)
    f, g, S = s.get_state()
    o = oracle_mod.Oracle(shape, lattice_name="D3Q19", **PRM)
    o.set_state(f, g, S, 0)
    s.step(1)
    o.step(1)
    fg, gg, Sg = s.get_state()
    fo, go, So = o.get_state()
    eps = EPS[codec]
    fmov = np.abs(fo[1:]).max()
    assert np.abs(fg - fo).max() <= 4 * eps * fmov + 1e-6 * np.abs(fo).max()
    assert np.abs(gg - go).max() <= 8 * eps * np.abs(go).max()
    assert np.abs(Sg - So).max() <= 1e-4 * np.abs(So).max()
    mg, mo = s.moments(), o.macros()
    assert np.abs(mg["phi"] - mo["phi"]).max() <= 19 * 4 * eps * fmov + 1e-6


@pytest.mark.parametrize("codec", CODECS)
def test_offsets_init_matches_oracle(gpu, oracle_mod, codec):
    shape = (24, 20, 16)
    phi0 = wl.droplet(24, 20, 6.0, 5.0, nz=16)
    s = gpu.Simulation(shape, lattice="D3Q19", precision=codec, **PRM)
    o = oracle_mod.Oracle(shape, lattice_name="D3Q19", **PRM)
    s.init_phi(phi0)
    o.init_phi(phi0)
    fg, gg, _ = s.get_state()
    fo, go, _ = o.get_state()
    fmov = np.abs(fo[1:]).max()
    assert np.abs(fg - fo).max() <= 2 * EPS[codec] * fmov + 2 ** -24 * np.abs(fo[0]).max()
    assert np.abs(gg).max() == 0.0
    # phi = sum of the pulled values: one offset rounding per population
    assert np.abs(s.moments()["phi"] - phi0).max() <= 19 * 2 * EPS[codec] * fmov + 1e-7


# 64^3 two-droplet coalescence (the 512^3 case scaled to the oracle: R = 8,
# W = 5, centres 2R + 3 apart), 120 steps against the oracle
TOL_COALESCENCE = {"f16off": (1e-5, 1e-6), "bf16off": (1e-4, 1e-5)}


@pytest.mark.parametrize("codec", CODECS)
def test_offsets_coalescence_64_vs_oracle(gpu, oracle_mod, codec):
    shape = (64, 64, 64)
    phi0 = wl.two_droplets(64, 64, 8.0, 5.0, gap=3.0, nz=64)
    s = gpu.Simulation(shape, lattice="D3Q19", precision=codec, **PRM)
    o = oracle_mod.Oracle(shape, lattice_name="D3Q19", **PRM)
    s.init_phi(phi0)
    o.init_phi(phi0)
    s.step(120)
    o.step(120)
    mg, mo = s.moments(), o.macros()
    tphi, tu = TOL_COALESCENCE[codec]
    assert np.abs(mg["phi"] - mo["phi"]).max() < tphi
    assert np.abs(mg["u"] - mo["u"]).max() < tu


@pytest.mark.parametrize("codec", CODECS)
def test_offsets_graph_checkpoint_and_refresh(gpu, codec):
    """Graph replays equal single steps bit for bit, a checkpoint restores
    bit-exactly, and diagnostics (which refresh the scales) leave a run that
    stays finite and close to the run without them."""
    shape = (36, 20, 18)
    phi0 = wl.two_droplets(36, 20, 6.0, 5.0, gap=3.0, nz=18)
    a = gpu.Simulation(shape, lattice="D3Q19", precision=codec, **PRM)
    b = gpu.Simulation(shape, lattice="D3Q19", precision=codec, **PRM)
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
    c = gpu.Simulation(shape, lattice="D3Q19", precision=codec, **PRM)
    c.load(ck)
    c.step(35)
    fc, gc, Sc = c.get_state()
    assert np.array_equal(fa, fc) and np.array_equal(ga, gc) and np.array_equal(Sa, Sc)
    d = gpu.Simulation(shape, lattice="D3Q19", precision=codec, diag_every=10, **PRM)
    d.init_phi(phi0)
    d.step(70)
    dd = d.diagnostics()
    assert not dd["nonfinite"]
    pa, pd = a.moments()["phi"], d.moments()["phi"]
    assert np.abs(pa - pd).max() < 100 * EPS[codec] * 1e-3


@pytest.mark.parametrize("codec", CODECS)
def test_offsets_nonfinite_is_reported(gpu, codec):
    shape = (16, 16, 8)
    s = gpu.Simulation(shape, lattice="D3Q19", precision=codec, diag_every=1, **PRM)
    s.init_phi(wl.droplet(16, 16, 4.0, 5.0, nz=8))
    s.step(2)
    s.sync()
    from paper_2311_10827_gb300 import capi
    capi.check(capi.lbm_debug_poke(s.handle, 0, 3, 100, float("nan")))
    s.step(2)
    with pytest.raises(capi.LbmError):
        s.sync()


@pytest.mark.parametrize("codec", CODECS)
def test_offsets_long_run_against_fp64(gpu, codec):
    """The 64^3 coalescence for 2000 steps: phi and u against the FP64 GPU
    path (itself in parity with the oracle at 1e-12) and the phi-mass drift
    against the FP64 drift."""
    shape = (64, 64, 64)
    phi0 = wl.two_droplets(64, 64, 8.0, 5.0, gap=3.0, nz=64)
    runs = {}
    for prec in ("fp64", codec):
        s = gpu.Simulation(shape, lattice="D3Q19", precision=prec, **PRM)
        s.init_phi(phi0)
        d0 = s.diagnostics()
        s.step(2000)
        d1 = s.diagnostics()
        runs[prec] = (s.moments(), d1["sum_phi"] - d0["sum_phi"], d0["sum_phi"])
    m64, drift64, mass = runs["fp64"]
    m, drift, _ = runs[codec]
    tphi, tu = TOL_LONG[codec]
    assert np.abs(m["phi"] - m64["phi"]).max() < tphi
    assert np.abs(m["u"] - m64["u"]).max() < tu
    assert abs(drift - drift64) < TOL_MASS[codec] * mass


# measured on GB300 at 2000 steps: phi 6.8e-8 / 9.6e-7, u 3.4e-9 / 2.3e-8, mass
# (relative to the FP64 drift) 3e-8 / 1e-7 for FP16 / BF16; bounds ~10x above
TOL_LONG = {"f16off": (1e-6, 1e-7), "bf16off": (1e-5, 1e-6)}
TOL_MASS = {"f16off": 1e-6, "bf16off": 2e-6}
