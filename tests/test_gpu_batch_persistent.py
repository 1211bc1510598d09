"""Multi-step batch launches (lbm_batch_set_persistent): one cooperative
launch runs many time steps as a queue of (step, tile) pairs, each tile
waiting only for itself and the tiles its stencil reaches.  The arithmetic is
that of the per-step launches, so the states must agree bit for bit after
every chunk of steps.  Chunks of uneven length are interleaved with
diagnostics (which move the FP32 equilibrium shift between launches).  The
shapes cover:
- ragged strips and row tiles;
- a grid smaller than one tile, whose only neighbour is itself;
- both strip widths, and the bench's two 1024^2 grids at 128 x 28;
- batches with several times more tiles than resident CTAs (the tiles are
  walked as a queue every step).
A wait that timed out would leave NaN in S and set the batch's error word:
both are checked.  The fused batch diagnostics (lbm_batch_set_diag_every)
are checked against the on-demand diagnostics of the same states, and
against the exact phi budget of the step (reading R14)."""
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


def run_pair(sim, cases, precision, width, rows, chunks):
    """Two identical batches, per-step and multi-step; states after each chunk."""
    out = []
    batches = [sim.Batch([(sh, prm) for sh, prm, _ in cases], precision=precision)
               for _ in range(2)]
    try:
        for b in batches:
            for i, (_, _, phi) in enumerate(cases):
                b.case(i).init_phi(phi)
            b.set_shape(width, rows)
        batches[1].set_persistent(True)
        assert batches[1].persistent()[0] and not batches[0].persistent()[0]
        for n in chunks:
            states = []
            for b in batches:
                b.step(n)
                st = [b.case(i).get_state() for i in range(len(b))]
                for i in range(len(b)):
                    b.case(i).diagnostics()
                states.append(st)
            out.append(states)
        assert batches[1].persistent(read_timeout=True)[1] is False
    finally:
        for b in batches:
            b.close()
    return out


def assert_same(out):
    for k, (ref, per) in enumerate(out):
        for c, (sa, sb) in enumerate(zip(ref, per)):
            for name, x, y in zip(("f", "g", "S"), sa, sb):
                assert np.isfinite(y).all(), (k, c, name)
                assert np.array_equal(x, y), (k, c, name, float(np.abs(x - y).max()))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("width,rows", [(128, 28), (64, 16)])
def test_multistep_equals_per_step(gpu, precision, width, rows):
    cases = [((1024, 512), dict(BASE, rho_l=10.0), wl.droplet(1024, 512, 100.0, 4.0)),
             ((300, 37), dict(BASE, rho_l=30.0), wl.droplet(300, 37, 10.0, 4.0)),
             ((100, 9), dict(BASE, rho_l=3.0), wl.flat_interface(100, 9, 4.0))]
    assert_same(run_pair(gpu, cases, precision, width, rows, (2, 7, 40, 3)))


def test_multistep_equals_per_step_bench_config(gpu):
    """The default bench line's configuration: two 1024^2 droplets (density
    ratios 10 and 100), FP32, tiles 128 x 28 (592 CTAs, about one wave)."""
    phi = wl.droplet(1024, 1024, 128.0, 4.0)
    cases = [((1024, 1024), dict(BASE, rho_l=r), phi) for r in (10.0, 100.0)]
    assert_same(run_pair(gpu, cases, "fp32", 128, 28, (100, 201)))


def test_multistep_walks_more_tiles_than_resident_ctas(gpu):
    """64 grids of the ensemble recipe (seeds 0..63: N from U{64..512}, uneven
    sizes) at 128 x 28 and 64 x 8 tiles: thousands of tiles, several per
    resident CTA, walked as a queue every step.  Hundreds of steps: a CTA
    whose warps disagreed on their next pair (a race on the ticket) showed
    only after about a hundred steps of this batch."""
    cases = []
    for seed in range(64):
        c = wl.ensemble_case(seed)
        cases.append(((c["n"], c["n"]), dict(BASE, rho_l=c["rho_ratio"]),
                      wl.droplet(c["n"], c["n"], c["R"], 4.0)))
    assert_same(run_pair(gpu, cases, "fp32", 128, 28, (3, 30, 300)))
    small = cases[:16]
    assert_same(run_pair(gpu, small, "fp64", 64, 8, (5, 2)))


def test_long_call_splits_into_launches_of_at_most_1024_steps(gpu):
    """A call of more steps than one multi-step launch holds (1024, the size
    of the per-step completion counts) is split into launches of 1024 and 76
    steps; the state equals that of per-step launches bit for bit (FP32,
    staged pulls).  Without fused diagnostics: a diagnostics step inside a
    multi-step launch moves the FP32 equilibrium shift from the next launch
    on, per-step launches from the next step on, and the two differ by
    rounding (the shift is an exact symmetry of the step only in exact
    arithmetic)."""
    cases = [((128, 64), dict(BASE, rho_l=10.0), wl.droplet(128, 64, 15.0, 4.0)),
             ((128, 48), dict(BASE, rho_l=50.0), wl.droplet(128, 48, 12.0, 4.0))]
    batches = [gpu.Batch([(sh, prm) for sh, prm, _ in cases], precision="fp32") for _ in range(2)]
    try:
        for b in batches:
            for i, (_, _, phi) in enumerate(cases):
                b.case(i).init_phi(phi)
            b.set_shape(64, 16)
        batches[1].set_persistent(True)
        for b in batches:
            b.step(1100)
        assert batches[1].persistent(read_timeout=True)[1] is False
        for i in range(len(cases)):
            assert batches[1].case(i).t == 1100
            for x, y in zip(batches[0].case(i).get_state(), batches[1].case(i).get_state()):
                assert np.array_equal(x, y)
    finally:
        for b in batches:
            b.close()


def _start_at(b, cases, t0):
    """Every grid initialised from its phi0 (Eq. H_i initial condition), then
    set to time t0 (the state unchanged): the diagnostics cadence counts from
    there, so that no diagnostics step (and no FP32 shift move) comes before
    the one compared."""
    for i, (_, _, phi) in enumerate(cases):
        b.case(i).init_phi(phi)
        f, g, S = b.case(i).get_state()
        b.case(i).set_state(f, g, S, step=t0)


def _bench_like_cases():
    return [((300, 140), dict(BASE, rho_l=10.0), wl.droplet(300, 140, 30.0, 4.0)),
            ((256, 100), dict(BASE, rho_l=100.0), wl.droplet(256, 100, 25.0, 4.0)),
            ((70, 9), dict(BASE, rho_l=3.0), wl.flat_interface(70, 9, 4.0))]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fused_diagnostics_match_on_demand(gpu, precision):
    """Diagnostics every 10 steps from t = 1: the step from t = 10 carries
    them.  Against lbm_diagnostics of the same state at t = 10 (a separate
    pass, another tiling of the reduction): FP64 sums to 1e-12 relative,
    extrema identical.  Per-step and multi-step launches give identical
    records."""
    cases = _bench_like_cases()
    recs = {}
    for persistent in (False, True):
        b = gpu.Batch([(sh, prm) for sh, prm, _ in cases], precision=precision)
        try:
            _start_at(b, cases, 1)
            b.set_shape(128, 28)
            if persistent:
                b.set_persistent(True)
            b.set_diag_every(10)
            b.step(12)
            r = b.last_diagnostics()
            assert all(x["step"] == 10 for x in r)
            recs[persistent] = r
        finally:
            b.close()
    ref = gpu.Batch([(sh, prm) for sh, prm, _ in cases], precision=precision)
    try:
        _start_at(ref, cases, 1)
        ref.set_shape(128, 28)
        ref.step(9)
        want = [ref.case(i).diagnostics() for i in range(len(ref))]
    finally:
        ref.close()
    for got, w in zip(recs[False], want):
        assert w["step"] == 10
        for k in ("sum_phi", "kinetic_energy", "budget"):
            assert abs(got[k] - w[k]) <= 1e-12 * abs(w[k]) + 1e-300, (k, got[k], w[k])
        for k in ("u_max", "mu_min", "mu_max"):
            assert got[k] == w[k], (k, got[k], w[k])
        assert not got["nonfinite"]
    for a, b in zip(recs[False], recs[True]):
        assert a == b


@pytest.mark.parametrize("persistent", [False, True])
def test_fused_diagnostics_phi_budget(gpu, persistent):
    """Reading R14: sum phi^{t+1} - sum phi^t = -sum (1.5 S^t - 0.5 S^{t-1}),
    the budget of the step from t, exactly up to FP64 round-off.  Diagnostics
    every step, read after each call (FP64, three uneven grids); two-step
    calls put the records in multi-step launches too."""
    cases = _bench_like_cases()
    b = gpu.Batch([(sh, prm) for sh, prm, _ in cases], precision="fp64")
    try:
        for i, (_, _, phi) in enumerate(cases):
            b.case(i).init_phi(phi)
        b.set_shape(128, 28)
        if persistent:
            b.set_persistent(True)
        b.set_diag_every(1)
        b.step(6)
        prev = None
        for n in (1, 2, 1, 2, 1):
            b.step(n)
            r = b.last_diagnostics()
            if prev is not None and r[0]["step"] == prev[0]["step"] + 1:
                for x, y in zip(prev, r):
                    assert abs((y["sum_phi"] - x["sum_phi"]) + x["budget"]) <= \
                        1e-12 * abs(x["sum_phi"])
                    assert abs(x["budget"]) > 0.0
            prev = r
        # consecutive records: the last step of a call carries the diagnostics
        assert prev[0]["step"] == 6 + 7 - 1
    finally:
        b.close()


def test_stalled_tile_times_out_without_hanging(gpu):
    """Fault injection: tile 0 waits on a counter that nothing sets.  The
    launch must end by itself after the bounded wait (about 2 s of SM clock),
    report the timeout (the next batch step returns LBM_ERR_TIMEOUT, and
    keeps returning it until the tiles are rebuilt), and leave non-finite
    fields that the diagnostics flag; the GPU stays usable (the same batch,
    rebuilt and re-initialised, and a fresh batch then step normally)."""
    import time

    from paper_2311_10827_gb300 import capi
    cases = [((256, 128), dict(BASE, rho_l=10.0))] * 2
    phi = wl.droplet(256, 128, 30.0, 4.0)
    b = gpu.Batch(cases, precision="fp32")
    try:
        for i in range(len(b)):
            b.case(i).init_phi(phi)
        b.set_shape(128, 16)
        b.set_persistent(True)
        capi.check(capi.lbm_batch_debug_stall(b.handle, 0))
        t = time.perf_counter()
        b.step(4)
        on, timed_out = b.persistent(read_timeout=True)
        dt = time.perf_counter() - t
        assert timed_out is True
        assert 0.5 < dt < 30.0, dt
        assert capi.lbm_batch_step(b.handle, 2) == capi.LBM_ERR_TIMEOUT
        assert capi.lbm_batch_step(b.handle, 2) == capi.LBM_ERR_TIMEOUT
        assert capi.lbm_batch_sync(b.handle) == capi.LBM_ERR_TIMEOUT
        assert b.case(0).diagnostics()["nonfinite"]
        b.set_shape(128, 16)  # rebuilt tiles: the injection and the timeout are cleared
        assert b.persistent(read_timeout=True)[1] is False
        for i in range(len(b)):
            b.case(i).init_phi(phi)
        b.step(4)
        b.sync()
        assert not b.case(0).diagnostics()["nonfinite"]
    finally:
        b.close()
    fresh = gpu.Batch(cases, precision="fp32")
    try:
        for i in range(len(fresh)):
            fresh.case(i).init_phi(phi)
        fresh.set_shape(128, 16)
        fresh.set_persistent(True)
        fresh.step(4)
        assert fresh.persistent(read_timeout=True)[1] is False
        assert not fresh.case(0).diagnostics()["nonfinite"]
    finally:
        fresh.close()
