"""The library's discrete adjoint (C ABI lbm_adjoint_*, torch.autograd) against
the oracle's FP64 adjoint and against central finite differences of the GPU
forward map.  Loss: L = sum (phi^n - phi_target)^2 from the initial field."""
import numpy as np
import pytest

from paper_2311_10827_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

PRM = dict(W=4.0, alpha=1.0, rho_l=5.0, rho_v=1.0, nu_l=0.3, nu_v=0.1, Gx=2e-5, Gy=-1e-5)
SIGMA, MOB = 4e-3, 0.08


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_10827_gb300 import adjoint, build, capi, sim
    build.build()
    return torch, adjoint, capi, sim


def gpu_grads(env, shape, phi0, target, n, K, precision="fp64"):
    torch, adjoint, capi, sim = env
    p0 = torch.tensor(phi0, dtype=torch.float64, device="cuda", requires_grad=True)
    sg = torch.tensor(SIGMA, dtype=torch.float64, device="cuda", requires_grad=True)
    mo = torch.tensor(MOB, dtype=torch.float64, device="cuda", requires_grad=True)
    tg = torch.tensor(target, dtype=torch.float64, device="cuda")
    phiN = adjoint.rollout(p0, sg, mo, shape=shape, nsteps=n, checkpoint_every=K,
                           precision=precision, **PRM)
    L = ((phiN - tg) ** 2).sum()
    L.backward()
    return float(L.detach()), p0.grad.cpu().numpy(), float(sg.grad), float(mo.grad)


@pytest.mark.parametrize("shape,n,K", [((12, 10), 12, 5), ((40, 26), 30, 7)])
def test_gpu_adjoint_matches_oracle_adjoint(env, oracle_mod, shape, n, K):
    nx, ny = shape
    phi0 = wl.two_droplets(nx, ny, min(shape) / 4, 4.0, gap=1.0)
    target = np.roll(phi0, 1, axis=1) * 0.97 + 0.01
    Lo, go, so, mo = oracle_mod.phi_loss_gradients(shape, dict(PRM, sigma=SIGMA, M=MOB), phi0,
                                                   target, n)
    Lg, gg, sg, mg = gpu_grads(env, shape, phi0, target, n, K)
    assert np.isclose(Lg, Lo, rtol=1e-11)
    assert np.abs(gg - go).max() <= 1e-10 * np.abs(go).max()
    assert np.isclose(sg, so, rtol=1e-9) and np.isclose(mg, mo, rtol=1e-9)


def test_gpu_adjoint_finite_differences_32x32_50_steps(env):
    """The finite-difference check of the adjoint workload: 32 x 32, 50 steps, FP64."""
    torch, adjoint, capi, sim = env
    shape, n = (32, 32), 50
    phi0 = wl.two_droplets(32, 32, 5.0, 4.0)
    target = np.roll(phi0, 2, axis=0) * 0.98 + 0.01
    L, gphi0, gsig, gM = gpu_grads(env, shape, phi0, target, n, 10)

    def loss(phi, sigma=SIGMA, M=MOB):
        s = sim.Simulation(shape, precision="fp64", sigma=sigma, M=M, **PRM)
        s.init_phi(phi)
        s.step(n)
        return float(((s.moments()["phi"] - target) ** 2).sum())

    rng = np.random.default_rng(9)
    for _ in range(4):
        j, i = rng.integers(32), rng.integers(32)
        h = 1e-6
        pp, pm = phi0.copy(), phi0.copy()
        pp[j, i] += h
        pm[j, i] -= h
        fd = (loss(pp) - loss(pm)) / (2 * h)
        assert abs(fd - gphi0[j, i]) <= 1e-5 * max(abs(fd), 1e-4), (fd, gphi0[j, i])
    h = 1e-6 * SIGMA
    fd = (loss(phi0, sigma=SIGMA + h) - loss(phi0, sigma=SIGMA - h)) / (2 * h)
    assert abs(fd - gsig) <= 1e-5 * abs(fd)
    h = 1e-6 * MOB
    fd = (loss(phi0, M=MOB + h) - loss(phi0, M=MOB - h)) / (2 * h)
    assert abs(fd - gM) <= 1e-5 * abs(fd)


def test_gpu_adjoint_fp32_forward_close_to_fp64(env):
    """FP32 forward and FP32 reverse step on the same problem: gradients
    within FP32 rounding (accumulated over the run) of the FP64 ones."""
    shape, n = (64, 48), 60
    phi0 = wl.two_droplets(64, 48, 8.0, 4.0)
    target = np.roll(phi0, 3, axis=1) * 0.95 + 0.02
    L64, g64, s64, m64 = gpu_grads(env, shape, phi0, target, n, 20, "fp64")
    L32, g32, s32, m32 = gpu_grads(env, shape, phi0, target, n, 20, "fp32")
    assert np.isclose(L32, L64, rtol=1e-5)
    assert np.abs(g32 - g64).max() <= 1e-4 * np.abs(g64).max()
    assert np.isclose(s32, s64, rtol=1e-3) and np.isclose(m32, m64, rtol=1e-3)
