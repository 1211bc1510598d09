"""lbm_diagnostics_noalloc: diagnostics for callers that cannot allocate
device memory (a host framework's pool or a fixed arena, no cudaMalloc
allowed), with its scratch in a fixed device array inside the library.

The state is handed over in the library's storage layout (the population
payload of lbm_save) in buffers the test allocates; the entry point itself
allocates nothing.  Its output must match the context-based
lbm_diagnostics on the same state, on two calls in a row.
"""
import numpy as np
import pytest

from paper_2311_10827_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

PRM = dict(W=4.0, M=0.05, alpha=1.0, sigma=1e-3, rho_l=10.0, rho_v=1.0, nu_l=1.0, nu_v=0.1)
RTOL = 1e-12


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_10827_gb300 import build, capi, sim
    build.build()
    return torch, capi, sim


def device_state(torch, s):
    """(f, g, S) device tensors in storage layout, copied from a checkpoint."""
    buf = s.save()
    dt = np.float64 if s.precision == "fp64" else np.float32
    QN, N = s.Q * s.N, s.N
    FN = QN + (N if s.precision == "fp32" else 0)  # FP32 f carries the rest pair's low word
    payload = (FN + QN + N) * np.dtype(dt).itemsize
    raw = np.frombuffer(buf[len(buf) - payload:].tobytes(), dtype=dt)
    to = lambda a: torch.from_numpy(a.copy()).cuda()  # noqa: E731
    return to(raw[:FN]), to(raw[FN:FN + QN]), to(raw[FN + QN:])


def noalloc(torch, capi, s, f, g, S):
    out = torch.full((8,), -1.0, dtype=torch.float64, device="cuda")
    rc = capi.lbm_diagnostics_noalloc((s.nx, s.ny, 1), capi.LBM_D2Q9, s.params, f, g, S, out,
                                      torch.cuda.current_stream().cuda_stream)
    assert rc == capi.LBM_OK, capi.strerror(rc)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check_against_context(o, d):
    assert np.isclose(o[0], d["sum_phi"], rtol=RTOL, atol=0)
    assert np.isclose(o[1], d["kinetic_energy"], rtol=RTOL, atol=0)
    assert np.isclose(np.sqrt(o[2]), d["u_max"], rtol=RTOL, atol=0)
    assert np.isclose(o[3], d["mu_min"], rtol=RTOL, atol=0)
    assert np.isclose(o[4], d["mu_max"], rtol=RTOL, atol=0)
    assert np.isclose(o[5], d["budget"], rtol=RTOL, atol=1e-300)
    assert o[6] == float(d["nonfinite"]) and o[7] == 0.0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_context_diagnostics_twice(env, precision):
    torch, capi, sim = env
    s = sim.Simulation((384, 200), precision=precision,
                       stream=torch.cuda.current_stream().cuda_stream, **PRM)
    s.init_phi(wl.two_droplets(384, 200, 40.0, 4.0))
    s.step(30)
    for _ in range(2):  # two calls in a row, each on a fresh state
        f, g, S = device_state(torch, s)
        o = noalloc(torch, capi, s, f, g, S)
        d = s.diagnostics()
        check_against_context(o, d)
        assert d["kinetic_energy"] > 0.0
        s.step(17)


def test_noalloc_rejects_too_many_ctas_and_null(env):
    torch, capi, sim = env
    p = sim.make_params("fp32", **PRM)
    t = torch.zeros(64, dtype=torch.float64, device="cuda")
    # 8192 x 16448 nodes: a valid grid whose pass needs more than 4096 CTAs
    rc = capi.lbm_diagnostics_noalloc((8192, 16448, 1), capi.LBM_D2Q9, p, t, t, t, t)
    assert rc == capi.LBM_ERR_INVALID_ARG
    rc = capi.lbm_diagnostics_noalloc((64, 64, 1), capi.LBM_D2Q9, p, None, t, t, t)
    assert rc == capi.LBM_ERR_INVALID_ARG
