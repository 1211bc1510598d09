"""Batched ensemble: one launch per step over a tile table covering many
independent grids of uneven sizes and parameters.  Every grid must evolve as
it does alone, to rounding (the batched kernel and its tile-width variants
are separate compiled instantiations, so the compiler may contract the same
expressions into FMAs differently: agreement is at the parity tolerance, not
bit for bit), and the autotuner must leave the state untouched."""
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
    return sim


def ensemble(seeds):
    out = []
    for s in seeds:
        c = wl.ensemble_case(s)
        n = max(16, c["n"] // 4)  # scaled down for the test
        prm = dict(BASE, rho_l=c["rho_ratio"])
        out.append(((n, n + 7), prm, wl.droplet(n, n + 7, c["R"] / 4, 4.0)))
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_equals_single_grids(gpu, precision):
    cases = ensemble(range(7)) + [((300, 37), dict(BASE, rho_l=30.0), wl.droplet(300, 37, 10.0, 4.0))]
    b = gpu.Batch([(sh, prm) for sh, prm, _ in cases], precision=precision)
    singles = []
    for i, (sh, prm, phi0) in enumerate(cases):
        b.case(i).init_phi(phi0)
        s = gpu.Simulation(sh, precision=precision, **prm)
        s.init_phi(phi0)
        singles.append(s)
    b.step(1)
    b.step(77)  # odd start, graph replays, remainder
    for s in singles:
        s.step(78)
    rtol = 1e-12 if precision == "fp64" else 1e-5
    for i, s in enumerate(singles):
        fa, ga, Sa = b.case(i).get_state()
        fb, gb, Sb = s.get_state()
        scale = max(np.abs(fb).max(), np.abs(gb).max())
        for x, y in ((fa, fb), (ga, gb), (Sa, Sb)):
            assert np.abs(x - y).max() <= rtol * scale, i
        assert b.case(i).t == 78


def test_batch_tuning_keeps_state_and_reports_shape(gpu):
    cases = ensemble(range(5))
    b = gpu.Batch([(sh, prm) for sh, prm, _ in cases], precision="fp32")
    for i, (_, _, phi0) in enumerate(cases):
        b.case(i).init_phi(phi0)
    b.step(3)
    before = [b.case(i).get_state() for i in range(len(b))]
    w, r = b.tune()
    # the listed row counts (8 .. 128) or the one-wave count of a width (even)
    assert w in (64, 128) and r >= 2 and r % 2 == 0
    assert b.shape()[:2] == (w, r)
    for i in range(len(b)):
        for x, y in zip(before[i], b.case(i).get_state()):
            assert np.array_equal(x, y)


def test_multistep_tuning_keeps_state(gpu):
    """With multi-step launches on, tuning times multi-step launches of the
    grids' own state and puts the state back: the state, the time and the
    following steps are those of a batch that was never tuned that way."""
    cases = ensemble(range(4))
    runs = []
    for tune in (False, True):
        b = gpu.Batch([(sh, prm) for sh, prm, _ in cases], precision="fp32")
        try:
            for i, (_, _, phi0) in enumerate(cases):
                b.case(i).init_phi(phi0)
            b.set_shape(128, 16)
            b.set_persistent(True)
            b.step(5)
            before = [b.case(i).get_state() for i in range(len(b))]
            if tune:
                w, r = b.tune()
                assert w in (64, 128) and r >= 2 and r % 2 == 0
                for i in range(len(b)):
                    for x, y in zip(before[i], b.case(i).get_state()):
                        assert np.array_equal(x, y)
                    assert b.case(i).t == 5
            b.step(7)
            runs.append([b.case(i).get_state() for i in range(len(b))])
        finally:
            b.close()
    for sa, sb in zip(*runs):
        for x, y in zip(sa, sb):
            assert np.array_equal(x, y)


def test_batch_requires_lockstep(gpu):
    from paper_2311_10827_gb300 import capi
    cases = ensemble(range(3))
    b = gpu.Batch([(sh, prm) for sh, prm, _ in cases], precision="fp32")
    assert capi.lbm_batch_step(b.handle, 1) == capi.LBM_ERR_STATE  # not initialised
    for i, (_, _, phi0) in enumerate(cases):
        b.case(i).init_phi(phi0)
    b.step(2)
    b.case(1).step(1)  # desynchronise one grid
    assert capi.lbm_batch_step(b.handle, 1) == capi.LBM_ERR_STATE
    for i, (_, _, phi0) in enumerate(cases):
        b.case(i).init_phi(phi0)
    b.step(1)


def test_batch_fp64_matches_oracle(gpu, oracle_mod):
    cases = ensemble([11, 12])
    b = gpu.Batch([(sh, prm) for sh, prm, _ in cases], precision="fp64")
    oracles = []
    for i, (sh, prm, phi0) in enumerate(cases):
        b.case(i).init_phi(phi0)
        o = oracle_mod.Oracle(sh, **prm)
        o.init_phi(phi0)
        oracles.append(o)
    b.step(40)
    for i, o in enumerate(oracles):
        o.step(40)
        fg, gg, _ = b.case(i).get_state()
        fo, go, _ = o.get_state()
        atol = 1e-14 * max(np.abs(fo).max(), np.abs(go).max())
        assert np.abs(fg - fo).max() <= 1e-12 * np.abs(fo).max() + atol
        assert np.abs(gg - go).max() <= 1e-12 * np.abs(go).max() + atol
