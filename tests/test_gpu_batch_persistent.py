"""Multi-step batch launches (lbm_batch_set_persistent): one cooperative
launch runs many time steps, each tile waiting only for the tiles its stencil
reaches.  The arithmetic is that of the per-step launches, so the states must
agree bit for bit after every chunk of steps.  Chunks of uneven length are
interleaved with diagnostics (which move the FP32 equilibrium shift between
launches).  The shapes cover:
- ragged strips and row tiles;
- a grid smaller than one tile, whose only neighbour is itself;
- both strip widths, and the bench's two 1024^2 grids at 128 x 28.
A wait that timed out would leave NaN in S and set the batch's error word:
both are checked."""
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


def test_set_persistent_rejects_shapes_that_do_not_fit(gpu):
    """Two 4096^2 grids at 64 x 8 tiles: 65536 tiles, far more than resident CTAs."""
    from paper_2311_10827_gb300 import capi
    cases = [((4096, 4096), dict(BASE, rho_l=10.0))] * 2
    b = gpu.Batch(cases, precision="fp32")
    try:
        b.set_shape(64, 8)
        with pytest.raises(capi.LbmError):
            b.set_persistent(True)
        assert b.persistent()[0] is False
    finally:
        b.close()


def test_stalled_tile_times_out_without_hanging(gpu):
    """Fault injection: tile 0 waits on a counter that nothing sets.  The
    launch must end by itself after the bounded wait (about 2 s of SM clock),
    report the timeout, and leave non-finite fields that the diagnostics flag;
    the GPU stays usable (a fresh batch then steps normally)."""
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
        assert b.case(0).diagnostics()["nonfinite"]
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
