"""The default bench line's kernel against the FP64 oracle directly, at the
tile shapes the bench runs: 64 x 16 (what the multi-step tuner picks for the
1024^2 pair: the staged multi-step kernel walks more tiles than resident
CTAs as a queue) and 128 x 28 (one tile per CTA; 14 two-row march
iterations per tile, so the phi/mu rings wrap and the two-stage copy
pipeline advances many times), on the bench's configuration scaled down:
two droplet grids (density ratios 10 and 100, viscosity ratio 10, W = 4,
sigma = 1e-3, M = 0.05) of 384 x 150 nodes (rows a multiple of 4 nodes, so
multi-step launches stage their pulls; ragged last row tiles of 6 and 10
rows), FP32, both launch forms (one multi-step launch per call, and
per-step launches), with the FP64 diagnostics fused every 20 steps as in
the bench (the diagnostics steps run the staged layout of their own).

* one step from a perturbed state that FP32 holds exactly (so both sides
  start from the same numbers): phi within 1e-5 and u within 1e-6;
* 2000 steps from the droplet: phi within 1e-5 and u within 1e-6 of the
  oracle, node by node (the FP32 targets)."""
import multiprocessing as mp

import numpy as np
import pytest

from paper_2311_10827_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SHAPE = (384, 150)
BASE = dict(W=4.0, M=0.05, alpha=1.0, sigma=1e-3, rho_v=1.0, nu_l=1.0, nu_v=0.1)
RATIOS = (10.0, 100.0)
STEPS = 2000


def _phi0():
    return wl.droplet(SHAPE[0], SHAPE[1], 40.0, 4.0)


def _oracle_run(args):
    """FP64 oracle, in its own process: (phi, u) after `steps` steps."""
    ratio, steps = args
    from oracle import oracle as O
    o = O.Oracle(SHAPE, **dict(BASE, rho_l=ratio))
    o.init_phi(_phi0())
    o.step(steps)
    m = o.macros()
    return m["phi"], m["u"]


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_10827_gb300 import build, sim
    build.build()
    return sim


@pytest.fixture(scope="module")
def oracle_long(oracle_mod):
    oracle_mod.build()
    with mp.get_context("spawn").Pool(len(RATIOS)) as pool:
        return pool.map(_oracle_run, [(r, STEPS) for r in RATIOS])


FORMS = [(True, (64, 16)), (True, (128, 28)), (False, (128, 28))]
IDS = ["multistep-64x16", "multistep-128x28", "perstep-128x28"]


def _batch(sim, persistent, tile):
    b = sim.Batch([(SHAPE, dict(BASE, rho_l=r)) for r in RATIOS], precision="fp32")
    b.set_shape(*tile)
    if persistent:
        b.set_persistent(True)
    b.set_diag_every(20)
    return b


@pytest.mark.parametrize("persistent,tile", FORMS, ids=IDS)
def test_headline_kernel_one_step_from_perturbed_state(gpu, oracle_mod, persistent, tile):
    b = _batch(gpu, persistent, tile)
    try:
        states = []
        for i, r in enumerate(RATIOS):
            o = oracle_mod.Oracle(SHAPE, **dict(BASE, rho_l=r))
            o.init_phi(_phi0())
            o.step(3)
            f, g, S = o.get_state()
            g = g + wl.perturbed_state(g.shape, 1e-3, 11 + i)
            S = S + wl.perturbed_state(S.shape, 1e-4, 21 + i)
            # values FP32 holds exactly (the rest population as a pair: hi only)
            f, g, S = (np.float32(x).astype(np.float64) for x in (f, g, S))
            o.set_state(f, g, S, 0)
            b.case(i).set_state(f, g, S, step=0)
            states.append(o)
        b.step(2)  # a multi-step launch needs two steps: compare after each
        for i, o in enumerate(states):
            o.step(2)
            m, mo = b.case(i).moments(), o.macros()
            assert np.abs(m["phi"] - mo["phi"]).max() <= 1e-5
            assert np.abs(m["u"] - mo["u"]).max() <= 1e-6
    finally:
        b.close()


@pytest.mark.parametrize("persistent,tile", FORMS, ids=IDS)
def test_headline_kernel_2000_steps_against_oracle(gpu, oracle_long, persistent, tile):
    b = _batch(gpu, persistent, tile)
    try:
        for i in range(len(b)):
            b.case(i).init_phi(_phi0())
        for _ in range(STEPS // 20):
            b.step(20)
        recs = b.last_diagnostics()
        assert all(not r["nonfinite"] and r["step"] == STEPS - 20 for r in recs)
        for i, (phi_o, u_o) in enumerate(oracle_long):
            m = b.case(i).moments()
            e_phi = np.abs(m["phi"] - phi_o).max()
            e_u = np.abs(m["u"] - u_o).max()
            assert e_phi <= 1e-5, (i, e_phi)
            assert e_u <= 1e-6, (i, e_u)
    finally:
        b.close()
