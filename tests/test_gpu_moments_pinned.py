"""lbm_moments into host arrays: when every given array is pinned host memory
the moments pass writes it directly through its device address; otherwise it
goes through a device staging buffer and copies.  Both routes, and a mix of
pinned and pageable arrays (which takes the staging route), give the same
values bit for bit, including the skipped (NULL) outputs, on a grid that is
not a whole number of tiles (FP32 and FP64)."""
import numpy as np
import pytest

from paper_2311_10827_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

BASE = dict(W=4.0, M=0.05, alpha=1.0, sigma=1e-3, rho_v=1.0, nu_l=1.0, nu_v=0.1)


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_10827_gb300 import build, sim
    build.build()
    return torch, sim


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_pinned_and_pageable_moments_agree(gpu, precision):
    torch, sim = gpu
    from paper_2311_10827_gb300 import capi
    nx, ny = 300, 70
    N = nx * ny
    s = sim.Simulation((nx, ny), precision=precision, **dict(BASE, rho_l=10.0))
    try:
        s.init_phi(wl.droplet(nx, ny, 20.0, 4.0))
        s.step(7)

        def pinned(m):
            return torch.empty(m * N, dtype=torch.float64).pin_memory().numpy()

        def pageable(m):
            return np.empty(m * N, dtype=np.float64)

        ref = {k: pageable(m) for k, m in (("phi", 1), ("p", 1), ("u", 2), ("mu", 1))}
        capi.check(capi.lbm_moments(s.handle, ref["phi"], ref["p"], ref["u"], ref["mu"], 0))
        pin = {k: pinned(m) for k, m in (("phi", 1), ("p", 1), ("u", 2), ("mu", 1))}
        capi.check(capi.lbm_moments(s.handle, pin["phi"], pin["p"], pin["u"], pin["mu"], 0))
        for k in ref:
            assert np.array_equal(ref[k], pin[k]), k
        # a mix takes the staging route; NULL outputs are skipped on both
        mix_phi, mix_u = pinned(1), pageable(2)
        capi.check(capi.lbm_moments(s.handle, mix_phi, None, mix_u, None, 0))
        assert np.array_equal(mix_phi, ref["phi"]) and np.array_equal(mix_u, ref["u"])
        only_mu = pinned(1)
        capi.check(capi.lbm_moments(s.handle, None, None, None, only_mu, 0))
        assert np.array_equal(only_mu, ref["mu"])
    finally:
        s.close()
