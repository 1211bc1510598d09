#!/usr/bin/env python
"""Throughput of the fused phase-field LBM step on GB300.

Workload: the 2D stationary droplet, 1024 x 1024 periodic, R = 128 centred,
W = 4, sigma = 1e-3, M = 0.05 (alpha = 1), viscosity ratio 10 (nu_l = 1,
nu_v = 0.1), D2Q9, FP32; one bench step advances both density-ratio cases
(rho_l/rho_v = 10 and 100) by one time step (two launches of the fused
kernel).  Synthetic input: the tanh droplet of the paper's stationary-droplet
test (Section 3.2), no dataset involved.

The step is the batched form: one kernel launch advances both grids
(tile shape from the library's autotuner, steps replayed from a CUDA graph),
and every --diag-every steps the FP64 diagnostics of both grids are reduced
and read back.

Metric: MLUPS (million node updates per second, both populations).  `value`
is device time (CUDA events on the launching stream around the timed
region), steps back to back: each step reads 2 x 84 MB, more than the 129 MB
L2, so reads come from HBM and every launch pays the write-backs of the one
before.  `e2e` is wall-clock through the C ABI with host buffers: pinned host
phi0 uploaded by lbm_init_phi, the same steps and diagnostics read-backs, the
final fields of both grids read back by lbm_moments.

Other workloads (--workload): ensemble (the 256-grid batch), coalescence3d
(the 512^3 D3Q19 run, --precision fp32 | f16off | bf16off) and adjoint (the
512^2 gradient).  Each line carries the same measurement keys: `roofline`
(algorithmic bytes over device time), `e2e` (through the C ABI with host
buffers), `clocks`, `gpu_launches` and `cpu_baseline` (the oracle on a
bounded sample of that workload).

Multi-GPU: replicas only (every rank runs its own pair of grids, weak
scaling; the only collectives are the timing barrier and max).

`cpu_baseline` is the FP64 oracle on one host core on a bounded sample of the
workload; `cpu_baseline_all_cores` runs one oracle process per host core.
--size 4096 runs the same line on two 4096 x 4096 grids (the out-of-L2 point).

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = NY = 1024
RATIOS = (10.0, 100.0)
# algorithmic bytes per node update: f and g each read once and written once
# (4 Q s) and S read + written (8 B FP32, 16 B FP64).  Anything else the
# kernels move (the FP32 rest population's low word, halo re-reads, phi work
# fields) is overhead and shows in the measured `traffic`.
BYTES_PER_NODE = {"fp32": 4 * 9 * 4 + 8, "fp64": 4 * 9 * 8 + 16}
# D3Q19 likewise; 16-bit offsets: 4 Q 2 + 2 x 24 (six FP32 macros read and
# written) + 8 (S)
BYTES_PER_NODE_3D = {"fp32": 4 * 19 * 4 + 8, "fp64": 4 * 19 * 8 + 16,
                     "f16off": 4 * 19 * 2 + 2 * 24 + 8, "bf16off": 4 * 19 * 2 + 2 * 24 + 8}
DTYPE = {"fp32": "f32", "fp64": "f64", "f16off": "f32 (f16 offset storage)",
         "bf16off": "f32 (bf16 offset storage)"}
KERNEL_SOURCES = ("paper_2311_10827_gb300/csrc/kernels_d2q9.cu",)
# DRAM bytes per step of the default line's kernel, from committed ncu
# summaries: the per-step launch and the multi-step cooperative launch
TRAFFIC_FILES = {
    "per_step": os.path.join(ROOT, "profiles", "traffic_d2q9_fp32_droplet1024.txt"),
    "multi_step": os.path.join(ROOT, "profiles", "traffic_d2q9_persist_fp32_droplet1024.txt"),
}


def params(ratio):
    from paper_2311_10827_gb300 import workloads as wl
    p = wl.physical(wl.DROPLET_1024)
    p["rho_l"] = ratio * p["rho_v"]
    return p


def phi0(n=NX):
    """The droplet on an n x n grid, R = 128 n / 1024 (R/L = 1/8)."""
    from paper_2311_10827_gb300 import workloads as wl
    return wl.droplet(n, n, wl.DROPLET_1024["R"] * n / NX, wl.DROPLET_1024["W"])


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_hash():
    """First 16 hex digits of the sha256 of the kernel sources with comments
    and blank lines removed: a traffic record belongs to the code it was
    taken on, whatever happens to the comments since."""
    import re
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel)) as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("\n".join(l.rstrip() for l in text.split("\n") if l.strip()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(mode="per_step"):
    """DRAM bytes per step from the committed ncu summary of the kernel that
    ran, if it was taken on the kernel source as it is now."""
    try:
        kv = {}
        with open(TRAFFIC_FILES[mode]) as fh:
            for line in fh:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_sha") != kernel_hash():
            return None
        return float(kv["dram_bytes_per_step"])
    except (OSError, KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms.  Started
    before the warm-up (its start-up must not fall in the timed region);
    summary() keeps the samples time-stamped inside the timed window."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.out = ""

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(1.0)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self, t_start=None, t_end=None):
        import datetime
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(f[2]), float(f[3]), f[6:10]))
            except ValueError:
                continue
        inside = [r for r in rows if t_start is None or t_start - 0.05 <= r[0] <= t_end + 0.05]
        if not inside and rows and t_start is not None:  # region shorter than the period
            inside = [min(rows, key=lambda r: abs(r[0] - 0.5 * (t_start + t_end)))]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in inside for k in range(4)
                          if r[3][k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[1] for r in inside),
                "sm_max_mhz": max(r[2] for r in inside), "reasons": reasons,
                "samples": len(inside)}


def cpu_baseline(steps=None, budget_s=12.0):
    """FP64 oracle on the host, on a bounded sample of the workload: whole
    1024 x 1024 grids (rho ratio 10), as many time steps as fit the budget."""
    from oracle import oracle as O
    O.build()
    o = O.Oracle((NX, NY), **params(RATIOS[0]))
    o.init_phi(phi0())
    o.step(1)
    n, t0 = 0, time.perf_counter()
    while (steps is None and time.perf_counter() - t0 < budget_s) or (steps is not None and n < steps):
        o.step(1)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": NX * NY * n / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"{n} time steps of one 1024x1024 D2Q9 droplet grid (rho ratio 10), FP64, "
                      f"single-threaded C oracle, {dt:.1f} s"}


def _oracle_worker(budget_s, barrier, out):
    """One oracle process of the all-cores timing: its own 1024 x 1024 grid
    (rho ratio 10), time steps until the budget is spent after a common start."""
    from oracle import oracle as O
    o = O.Oracle((NX, NY), **params(RATIOS[0]))
    o.init_phi(phi0())
    o.step(1)
    barrier.wait()
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        o.step(1)
        n += 1
    out.put((n, time.perf_counter() - t0))


def cpu_baseline_all_cores(budget_s=10.0):
    """The oracle on every host core at once: one single-threaded process per
    core (spawned), each stepping its own 1024 x 1024 grid; value = all node
    updates over the longest process's stepping time."""
    import multiprocessing as mp

    from oracle import oracle as O
    O.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(cores), ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(budget_s, barrier, out)) for _ in range(cores)]
    for pr in procs:
        pr.start()
    try:
        res = [out.get(timeout=budget_s + 300) for _ in procs]
    except Exception as e:  # a worker that died never reports
        for pr in procs:
            pr.terminate()
        return {"unavailable": f"all-cores oracle run failed: {type(e).__name__}"}
    for pr in procs:
        pr.join()
    steps = sum(n for n, _ in res)
    dt = max(t for _, t in res)
    return {"value": NX * NY * steps / dt / 1e6, "unit": "MLUPS", "cores": cores,
            "kind": "oracle",
            "sample": f"{cores} single-threaded oracle processes, each stepping its own "
                      f"1024x1024 D2Q9 droplet grid (rho ratio 10), FP64, {steps} time steps "
                      f"in all over {dt:.1f} s"}


def cpu_baseline_ensemble(budget_s=12.0, steps_each=5):
    """FP64 oracle on the ensemble's own grids in seed order (each initialised,
    then advanced steps_each time steps, only the steps timed) until the
    budget is spent."""
    from oracle import oracle as O
    from paper_2311_10827_gb300 import workloads as wl
    O.build()
    base = wl.physical(wl.DROPLET_1024)
    updates, dt, k = 0, 0.0, 0
    while dt < budget_s and k < 256:
        c = wl.ensemble_case(k)
        o = O.Oracle((c["n"], c["n"]), **dict(base, rho_l=c["rho_ratio"] * base["rho_v"]))
        o.init_phi(wl.droplet(c["n"], c["n"], c["R"], base["W"]))
        t = time.perf_counter()
        o.step(steps_each)
        dt += time.perf_counter() - t
        o.close()
        updates += c["n"] * c["n"] * steps_each
        k += 1
    return {"value": updates / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"{steps_each} time steps of each of the ensemble's grids 0..{k - 1} "
                      f"(seeds 0..{k - 1}), FP64, single-threaded C oracle, {dt:.1f} s"}


def cpu_baseline_coalescence3d(budget_s=12.0):
    """FP64 oracle (D3Q19) on the workload scaled to 64^3 (R = 8, same W,
    gap and parameters), as many time steps as fit the budget."""
    from oracle import oracle as O
    from paper_2311_10827_gb300 import workloads as wl
    O.build()
    cfg = wl.COALESCENCE_3D_SMALL
    n = cfg["shape"][0]
    o = O.Oracle((n, n, n), "D3Q19", **wl.physical(cfg))
    o.init_phi(wl.two_droplets(n, n, cfg["R"], cfg["W"], gap=cfg["gap"], nz=n))
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        o.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    o.close()
    return {"value": n ** 3 * steps / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"{steps} time steps of the two-droplet coalescence scaled to {n}^3 "
                      f"(R = {cfg['R']:g}), D3Q19, FP64, single-threaded C oracle, {dt:.1f} s"}


def cpu_baseline_adjoint(budget_s=12.0, n=128, steps=40):
    """FP64 oracle adjoint (forward run, then the reverse sweep) on the
    differentiated workload scaled to n^2 (R and the gap scaled, same W and
    parameters), gradients of steps-step runs repeated until the budget is
    spent; value in node updates of the differentiated run per second."""
    import numpy as np

    from oracle import oracle as O
    from paper_2311_10827_gb300 import workloads as wl
    O.build()
    cfg = wl.COALESCENCE_ADJ
    prm = wl.physical(cfg)
    R = cfg["R"] * n / cfg["shape"][0]
    phi0 = wl.two_droplets(n, n, R, cfg["W"])
    target = phi0 + 1e-3 * np.random.default_rng(0).standard_normal(phi0.shape)
    runs, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        O.phi_loss_gradients((n, n), prm, phi0, target, steps)
        runs += 1
    dt = time.perf_counter() - t0
    return {"value": n * n * steps * runs / dt / 1e6, "unit": "MLUPS", "cores": 1,
            "kind": "oracle",
            "sample": f"{runs} gradients of {steps}-step runs of the two-droplet coalescence "
                      f"scaled to {n}x{n} (R = {R:g}), FP64 forward + adjoint, "
                      f"single-threaded C oracle, {dt:.1f} s"}


def adjoint_bytes_per_node(esz):
    """Algorithmic bytes per node update of the differentiated run: the
    recorded forward step, the segment recomputation (which also writes the
    five moments), adj_local and adj_mu_phi (own-node values only;
    checkpoint copies, 2 % of the bytes at K = 100, are not counted)."""
    lo = 1 if esz == 4 else 0              # FP32 rest-pair low word
    fwd = (18 + lo) * 2 * esz + 2 * esz    # f, g (+ lo) read and written, S
    rec = fwd + 5 * esz                    # + phi, mu, p, ux, uy written
    local = (18 + lo + 5 + 10 + 9 + 1) * esz + 25 * esz
    mu_phi = 7 * esz + esz                 # lambda_mu, lambda_grad_mu, phi, lambda_phi, lambda_grad_phi; lpt
    return fwd + rec + local + mu_phi


def run_reference(args, rank, world, budget_s=90.0, est_mlups=2.0):
    """The oracle, as it stands, on rank 0.  Each step is one time step of a
    bounded sample of the workload: the full 1024 x 1024 droplet when K + W
    steps fit the budget, else a smaller square grid with the droplet scaled
    (R/L = 1/8) so that the whole run stays within a few minutes."""
    if rank != 0:
        return
    import math

    from oracle import oracle as O
    from paper_2311_10827_gb300 import workloads as wl
    O.build()
    nodes = est_mlups * 1e6 * budget_s / (args.steps + args.warmup)
    L = int(min(NX, max(32, math.isqrt(int(nodes)) // 32 * 32)))
    o = O.Oracle((L, L), **params(RATIOS[0]))
    o.init_phi(wl.droplet(L, L, L / 8.0, wl.DROPLET_1024["W"]))
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    v = L * L * args.steps / dt / 1e6
    sample = (f"{args.steps} time steps of a {L}x{L} periodic droplet grid (R = L/8, rho ratio "
              f"10), FP64 single-threaded C oracle")
    line = {"metric": "MLUPS (fused f+g step)", "value": v, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "2D stationary droplet 1024x1024, R=128, W=4, sigma=1e-3, "
                                   "M=0.05, nu_l/nu_v=10, rho ratio 10; bounded sample per step: "
                                   f"{L}x{L}"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# The stream is held by a short sleep kernel (torch's own, about 1 ms)
# between the synchronisation before a timed region and the region's first
# event, so that the host has enqueued the region's work by the time the
# first event fires: the events then time the device work of the steps, not
# the host's enqueue latency.  The sleep is outside the events.
GATE_CYCLES = 2_000_000


def gate():
    import torch
    torch.cuda._sleep(GATE_CYCLES)


def diag_cadence(args):
    """Diagnostics cadence of the timed runs: every --diag-every steps, and at
    least once in every timed region of --steps steps (any run of k
    consecutive steps holds exactly one multiple of k)."""
    return max(1, min(args.diag_every, args.steps))


def run_native(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2311_10827_gb300 import build as B
    B.build()
    from paper_2311_10827_gb300 import capi
    from paper_2311_10827_gb300 import workloads as wl
    from paper_2311_10827_gb300.sim import Batch

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    prec = args.precision
    de = diag_cadence(args)
    K = args.steps
    n = args.size or NX  # grid edge (1024: the headline; 4096: the out-of-L2 point)
    R = wl.DROPLET_1024["R"] * n / NX
    cases = [((n, n), params(r)) for r in RATIOS]
    nodes = n * n * len(cases)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return max_over_ranks_dist(x, world, dev)

    # ---- device-resident timing: the whole step (both grids) per launch,
    # diagnostics fused into the step that starts at each multiple of `de`
    batch = Batch(cases, precision=prec, stream=stream.cuda_stream)
    phi_d = torch.tensor(phi0(n), dtype=torch.float64, device=dev)
    for i in range(len(batch)):
        batch.case(i).init_phi(phi_d)
    # the tile shape: given, or tuned for the launches that will run
    multi = not args.per_step
    if args.tile:
        width, rows = (int(v) for v in args.tile.lower().split("x"))
        batch.set_shape(width, rows)
    if multi:
        batch.set_persistent(True)
    if not args.tile:
        width, rows = batch.tune()
    batch.set_diag_every(de)
    # The timed region (exactly K steps between two device synchronisations)
    # is repeated until about --min-time seconds of timed work, so that the
    # clock sampler sees it; `value` uses the mean over the repetitions.
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps_s = []
    with ClockSampler(local_rank) as clk:
        batch.step(args.warmup)
        barrier()
        t_wall = time.perf_counter()
        t_start = time.time()
        while True:
            barrier()
            gate()
            ev0.record(stream)
            batch.step(K)
            ev1.record(stream)
            barrier()
            reps_s.append(max_over_ranks(ev0.elapsed_time(ev1) / 1e3))
            if len(reps_s) >= args.repeat_min and (
                    sum(reps_s) >= args.min_time or len(reps_s) >= args.repeat_max):
                break
        t_wall = time.perf_counter() - t_wall
        t_end = time.time()
    recs = batch.last_diagnostics()
    if any(r["nonfinite"] for r in recs):
        raise RuntimeError("non-finite fields in the timed run")
    total_s = statistics.fmean(reps_s)
    value = nodes * K * world / total_s / 1e6
    ntiles = batch.shape()[2]
    batch.close()

    # ---- end to end through the C ABI with host buffers: phi0 of both grids
    # from pinned host memory, K steps with the fused diagnostics records read
    # on the host, final moments of both grids to pinned host memory
    hphi = torch.tensor(phi0(n), dtype=torch.float64).pin_memory()
    hphi_np = hphi.numpy()
    out_t = [{k: torch.empty(m * n * n, dtype=torch.float64).pin_memory()
              for k, m in (("phi", 1), ("p", 1), ("mu", 1), ("u", 2))} for _ in cases]
    outs = [{k: t.numpy() for k, t in o.items()} for o in out_t]  # views of pinned memory
    eb = Batch(cases, precision=prec, stream=stream.cuda_stream)
    eb.set_shape(width, rows)  # the tile shape tuned above (tuning is one-time setup)
    if multi:
        eb.set_persistent(True)
    eb.set_diag_every(de)
    e2e_runs = []
    for _ in range(args.e2e_runs):
        barrier()
        t_e = time.perf_counter()
        for i in range(len(eb)):
            capi.check(capi.lbm_init_phi(eb.case(i).handle, hphi_np, 0))
        capi.check(capi.lbm_batch_step(eb.handle, K))
        rc, erecs = capi.lbm_batch_last_diagnostics(eb.handle, len(eb))  # device -> host
        capi.check(rc)
        for i, o in enumerate(outs):
            capi.check(capi.lbm_moments(eb.case(i).handle, o["phi"], o["p"], o["u"], o["mu"], 0))
        barrier()
        e2e_runs.append(max_over_ranks(time.perf_counter() - t_e))
        if any(r.nonfinite for r in erecs):
            raise RuntimeError("non-finite fields in the end-to-end run")
    eb.close()
    e2e_s = statistics.fmean(e2e_runs)
    e2e_value = nodes * K * world / e2e_s / 1e6
    h2d = n * n * 8 * len(cases) / K
    n_diag = (K + de - 1) // de
    d2h = (n_diag * len(cases) * DIAG_RECORD_BYTES + 5 * n * n * 8 * len(cases)) / K

    if rank != 0:
        return
    # spurious velocity and phi of the e2e run's final state against the FP64
    # path (in parity with the FP64 oracle) after the same steps (not timed)
    accuracy = None
    if prec == "fp32" and not args.no_accuracy:
        ref = Batch(cases, precision="fp64", stream=stream.cuda_stream)
        ref.set_shape(width, rows)  # no tuning
        for i in range(len(ref)):
            ref.case(i).init_phi(phi_d)
        ref.step(K)
        accuracy = {"steps": K, "max_u_fp32": 0.0, "max_u_fp64": 0.0,
                    "max_abs_u_diff_vs_fp64": 0.0, "max_abs_phi_diff_vs_fp64": 0.0,
                    "reference": "FP64 GPU path (parity with the FP64 oracle at 1e-12), same "
                                 "phi0 and steps, both density ratios"}
        for i, o in enumerate(outs):
            m = ref.case(i).moments()
            u64 = m["u"].reshape(2, -1)
            u32 = o["u"].reshape(2, -1)
            accuracy["max_u_fp32"] = max(accuracy["max_u_fp32"], float(np.hypot(*u32).max()))
            accuracy["max_u_fp64"] = max(accuracy["max_u_fp64"], float(np.hypot(*u64).max()))
            accuracy["max_abs_u_diff_vs_fp64"] = max(accuracy["max_abs_u_diff_vs_fp64"],
                                                     float(np.abs(u32 - u64).max()))
            accuracy["max_abs_phi_diff_vs_fp64"] = max(
                accuracy["max_abs_phi_diff_vs_fp64"],
                float(np.abs(o["phi"] - m["phi"].reshape(-1)).max()))
        ref.close()
    peaks, src = measured_peaks()
    bpn = BYTES_PER_NODE[prec]
    achieved = bpn * nodes * K / total_s / 1e9
    traffic = (ncu_traffic("multi_step" if multi else "per_step")
               if prec == "fp32" and n == NX else None)
    launches = (launches_multi_step(args.warmup, K, de) if multi else K + (K + de - 1) // de)
    line = {
        "metric": "MLUPS (fused f+g step)", "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": K, "warmup": args.warmup,
        "ms_per_step": total_s / K * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64",
        "data": "synthetic",
        "config": {"workload": f"2D stationary droplet {n}x{n} periodic, R={R:g}, W=4, "
                               "sigma=1e-3, M=0.05, nu_l/nu_v=10, rho_l/rho_v=10 and 100 "
                               "(one step = both grids)",
                   "lattice": "D2Q9", "nodes_per_step": nodes, "diag_every": de,
                   "diagnostics": "FP64 diagnostics of both grids fused into the step that "
                                  "starts at each multiple of diag_every (one per timed region), "
                                  "reduced on the device, records read on the host after the "
                                  "timed regions",
                   "tile": {"width": width, "rows": rows, "ctas": ntiles},
                   "launch": ("one cooperative launch per timed region: a queue of "
                              "(step, tile) pairs, each tile synchronised with its neighbours"
                              if multi else "one launch per step, CUDA-graph replay"),
                   "timed_regions": {"count": len(reps_s), "steps_each": K,
                                     "start": "behind a ~1 ms sleep kernel issued after the "
                                              "synchronisation, so the events time the device "
                                              "work, not the host's enqueue",
                                     "ms_min": min(reps_s) * 1e3,
                                     "ms_median": statistics.median(reps_s) * 1e3,
                                     "ms_max": max(reps_s) * 1e3,
                                     "value_is": "mean over the regions"},
                   "l2": f"inputs larger than L2: 2 x {80 * n * n / 1e6:.0f} MB read per step, "
                         "back to back",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                     "traffic": traffic, "peak_source": f"{src} copy bandwidth (hbm_gbs)",
                     "algorithmic_bytes_per_node": bpn, "step_ms": total_s / K * 1e3,
                     "kernel": ("d2q9_batch_persist_kernel (both grids, one launch per timed "
                                "region; time of the whole region, per step; traffic per step)"
                                if multi else "d2q9_batch_kernel (both grids per launch)")},
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "runs": len(e2e_runs),
                "how": "wall clock through the C ABI, mean of the runs: lbm_init_phi of both "
                       "grids from pinned host phi0, lbm_batch_step of K steps with the fused "
                       "diagnostics (tile shape from the device-timed run's tuning, set "
                       "before the region), lbm_batch_last_diagnostics (the records, read on "
                       "the host), final lbm_moments of both grids to pinned host memory"},
        "accuracy": accuracy,
        "gpu_launches": launches,
        "clocks": clk.summary(t_start, t_end),
        "wall_s_timed_regions": t_wall,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
        line["cpu_baseline_all_cores"] = cpu_baseline_all_cores()
    print(json.dumps(line), flush=True)


DIAG_RECORD_BYTES = 64  # one FP64 record per grid: 8 doubles on the device


STEP_CAP = 1024  # steps per multi-step launch (the library splits longer calls)


def launches_multi_step(t0, k, de):
    """Kernel launches of one multi-step lbm_batch_step(k) call starting at
    time t0 with diagnostics every de steps: the launch is split so that it
    holds at most STEP_CAP steps and at most one diagnostics step (the
    library's rules)."""
    count, t, left = 0, t0, k
    while left > 0:
        m = min(left, STEP_CAP)
        d = (t + de - 1) // de * de
        if d < t + m and d + de < t + m:
            m = d + de - t
        count += 1
        t += m
        left -= m
    return count


def partition_cases(sizes, world):
    """Split independent cases over `world` ranks, balanced by node count:
    largest first, each to the rank with the fewest nodes so far (ties to the
    lowest rank).  Returns one sorted list of case indices per rank; every
    case lands on exactly one rank."""
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda j: (-sizes[j], j)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += sizes[i]
    return [sorted(p) for p in parts]


def combine_ranks(local_nodes, local_s, world, device):
    """Whole-job figures of a partitioned run: the node updates of all ranks
    over the slowest rank's time (the job ends when its last rank does)."""
    if world <= 1:
        return local_nodes, local_s
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_nodes)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item()), max_over_ranks_dist(local_s, world, device)


def run_ensemble(args, rank, world, local_rank):
    """The batched ensemble: 256 stationary droplets, N x N grids with N drawn
    from U{64..512}, R = U(0.15, 0.35) N, rho_l/rho_v = U(1, 100) (seeds 0..255,
    workloads.ensemble_case), W = 4, other parameters of the 1024^2 droplet.
    With N ranks the cases are partitioned across them (balanced by node
    count, no exchange: the cases are independent); each rank advances its
    share as one batch, one multi-step launch per call (the tiles walked as a
    queue), diagnostics fused every --diag-every steps."""
    import torch

    from paper_2311_10827_gb300 import build as B
    B.build()
    from paper_2311_10827_gb300 import workloads as wl
    from paper_2311_10827_gb300.sim import Batch
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    base = wl.physical(wl.DROPLET_1024)
    allc = [wl.ensemble_case(seed) for seed in range(256)]
    mine = partition_cases([c["n"] * c["n"] for c in allc], world)[rank]
    cases, phis = [], []
    for i in mine:
        c = allc[i]
        prm = dict(base, rho_l=c["rho_ratio"] * base["rho_v"])
        cases.append(((c["n"], c["n"]), prm))
        phis.append(wl.droplet(c["n"], c["n"], c["R"], base["W"]))
    de = diag_cadence(args)
    b = Batch(cases, precision=args.precision, stream=stream.cuda_stream)
    for i, phi in enumerate(phis):
        b.case(i).init_phi(phi)
    multi = not args.per_step
    if args.tile:
        width, rows = (int(v) for v in args.tile.lower().split("x"))
        b.set_shape(width, rows)
    if multi:
        b.set_persistent(True)
    if not args.tile:
        width, rows = b.tune()
    b.set_diag_every(de)
    ctas = b.shape()[2]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        b.step(args.warmup)
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        t_start = time.time()
        gate()
        e0.record(stream)
        b.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        t_end = time.time()
    if any(r["nonfinite"] for r in b.last_diagnostics()):
        raise RuntimeError("non-finite fields in the timed run")
    local_nodes = sum(sh[0] * sh[1] for sh, _ in cases)
    nodes, dt = combine_ranks(local_nodes, e0.elapsed_time(e1) / 1e3, world, dev)
    b.close()

    # end to end through the C ABI with host buffers: every grid's phi0 from
    # pinned host memory, the same steps, every grid's final phi to host
    import numpy as np

    from paper_2311_10827_gb300 import capi
    hphi = [torch.tensor(p, dtype=torch.float64).pin_memory() for p in phis]
    hout = [torch.empty(p.shape, dtype=torch.float64).pin_memory() for p in phis]
    eb = Batch(cases, precision=args.precision, stream=stream.cuda_stream)
    eb.set_shape(width, rows)  # the tuned shape (tuning is one-time setup)
    if multi:
        eb.set_persistent(True)
    eb.set_diag_every(de)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for i in range(len(eb)):
        capi.check(capi.lbm_init_phi(eb.case(i).handle, hphi[i].numpy(), 0))
    capi.check(capi.lbm_batch_step(eb.handle, args.steps))
    for i in range(len(eb)):
        capi.check(capi.lbm_moments(eb.case(i).handle, hout[i].numpy(), None, None, None, 0))
    rc, erecs = capi.lbm_batch_last_diagnostics(eb.handle, len(eb))
    capi.check(rc)
    torch.cuda.synchronize()
    _, e2e_s = combine_ranks(local_nodes, time.perf_counter() - t, world, dev)
    eb.close()
    if not all(np.isfinite(o.numpy()).all() for o in hout) or any(r.nonfinite for r in erecs):
        raise RuntimeError("non-finite phi in the end-to-end run")
    peaks, src = measured_peaks()
    bpn = BYTES_PER_NODE[args.precision]
    if rank == 0:
        v = nodes * args.steps / dt / 1e6
        n_diag = (args.steps + de - 1) // de
        line = {
            "metric": "MLUPS (fused f+g step)", "value": v, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": "batched ensemble: 256 stationary 2D droplets, grids "
                                   "64^2..512^2, seeds 0..255", "nodes_per_step": nodes,
                       "partition": f"cases split over {world} rank(s) by node count, no "
                                    "exchange (rank 0 holds "
                                    f"{len(mine)} cases, {local_nodes} nodes)",
                       "tile": {"width": width, "rows": rows, "ctas": ctas},
                       "launch": ("one cooperative launch per call: a queue of (step, tile) "
                                  "pairs over every grid's tiles" if multi
                                  else "one launch per step, CUDA-graph replay"),
                       "diag_every": de,
                       "l2": "inputs larger than L2: 27.5M nodes, 2.2 GB read per step"},
            "roofline": {"bound": "hbm", "achieved": bpn * v * 1e6 / 1e9 / world,
                         "peak": peaks["hbm_gbs"],
                         "frac": bpn * v * 1e6 / 1e9 / world / peaks["hbm_gbs"], "unit": "GB/s",
                         "traffic": None, "peak_source": f"{src} copy bandwidth (hbm_gbs)",
                         "algorithmic_bytes_per_node": bpn,
                         "kernel": ("d2q9_batch_persist_kernel" if multi else "d2q9_batch_kernel")
                                   + " (all of the rank's grids per launch)"},
            "e2e": {"value": nodes * args.steps / e2e_s / 1e6, "unit": "MLUPS",
                    "h2d_bytes_per_step": 8 * nodes / args.steps,
                    "d2h_bytes_per_step": (8 * nodes + n_diag * 256 * DIAG_RECORD_BYTES)
                                          / args.steps,
                    "how": "wall clock through the C ABI: lbm_init_phi of every grid from "
                           "pinned host phi0, lbm_batch_step (tuned shape set before the "
                           "region), lbm_moments of every grid's phi to pinned host memory, "
                           "the fused diagnostics records"},
            "gpu_launches": (launches_multi_step(args.warmup, args.steps, de) if multi
                             else args.steps + n_diag),
            "clocks": clk.summary(t_start, t_end),
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_ensemble()
        print(json.dumps(line), flush=True)


def run_coalescence3d(args, rank, world, local_rank):
    """3D coalescence (workloads.COALESCENCE_3D): 512^3 periodic, D3Q19 for
    both populations, two droplets R = 64, centres 2R + 3 apart, W = 5,
    density ratio 10.  One step = the phi pass and the fused pass; `value`
    and the roofline use the device time of whole steps (both kernels)."""
    import torch

    from paper_2311_10827_gb300 import build as B
    B.build()
    from paper_2311_10827_gb300 import capi
    from paper_2311_10827_gb300 import workloads as wl
    from paper_2311_10827_gb300.sim import Simulation
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    cfg = wl.COALESCENCE_3D
    n = args.size or cfg["shape"][0]
    R = cfg["R"] * n / cfg["shape"][0]
    sim = Simulation((n, n, n), lattice="D3Q19", precision=args.precision,
                     stream=stream.cuda_stream, **wl.physical(cfg))
    # phi0 of Section 3.3 in 3D, built on the device in FP64
    ax = torch.arange(n, dtype=torch.float64, device=dev)
    off = R + 0.5 * cfg["gap"]
    phi = torch.ones((), dtype=torch.float64, device=dev)
    for xk in (0.5 * n - off, 0.5 * n + off):
        d = torch.sqrt((ax[None, None, :] - xk) ** 2 + (ax[None, :, None] - 0.5 * n) ** 2
                       + (ax[:, None, None] - 0.5 * n) ** 2) - R
        phi = phi - torch.tanh(2 * d / cfg["W"])
        del d
    phi = (0.5 + 0.5 * phi).contiguous()
    sim.init_phi(phi)
    hphi = phi.cpu().pin_memory()  # host copy for the end-to-end run
    del phi
    torch.cuda.empty_cache()
    plan = []
    left = args.steps
    while left > 0:
        plan.append(min(args.diag_every, left))
        left -= plan[-1]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in plan]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d_first = None
    with ClockSampler(local_rank) as clk:
        sim.step(args.warmup)
        d_first = sim.diagnostics()
        torch.cuda.synchronize()
        t_start = time.time()
        gate()
        t0.record(stream)
        for (a, b), m in zip(ev, plan):
            a.record(stream)
            sim.step(m)
            b.record(stream)
            rc, d = capi.lbm_diagnostics(sim.handle)
            capi.check(rc)
            if d.nonfinite:
                raise RuntimeError("non-finite fields in the timed run")
        t1.record(stream)
        torch.cuda.synchronize()
        t_end = time.time()
    d_last = d.as_dict()
    total_s = max_over_ranks_dist(t0.elapsed_time(t1) / 1e3, world, dev)
    step_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3 / args.steps
    nodes = n ** 3
    sim.close()

    # end to end through the C ABI with host buffers: phi0 from pinned host
    # memory, the same steps and diagnostics read-backs, the final phi to host
    esim = Simulation((n, n, n), lattice="D3Q19", precision=args.precision,
                      stream=stream.cuda_stream, **wl.physical(cfg))
    hout = torch.empty_like(hphi).pin_memory()
    torch.cuda.synchronize()
    t = time.perf_counter()
    capi.check(capi.lbm_init_phi(esim.handle, hphi.numpy(), 0))
    n_diag = 0
    for m in plan:
        capi.check(capi.lbm_step(esim.handle, m))
        rc, d = capi.lbm_diagnostics(esim.handle)  # device -> host read
        capi.check(rc)
        n_diag += 1
    capi.check(capi.lbm_moments(esim.handle, hout.numpy(), None, None, None, 0))
    torch.cuda.synchronize()
    e2e_s = max_over_ranks_dist(time.perf_counter() - t, world, dev)
    esim.close()
    if not bool(torch.isfinite(hout).all()):
        raise RuntimeError("non-finite phi in the end-to-end run")
    del hphi, hout
    if rank != 0:
        return
    peaks, src = measured_peaks()
    bpn = BYTES_PER_NODE_3D[args.precision]
    achieved = bpn * nodes / step_s / 1e9
    line = {
        "metric": "MLUPS (fused f+g step)", "value": nodes * args.steps * world / total_s / 1e6,
        "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_s / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[args.precision],
        "data": "synthetic",
        "config": {"workload": f"3D coalescence of two droplets, D3Q19, {n}^3 periodic, "
                               f"R={R:g}, centres 2R+3 apart, W=5, rho_l/rho_v=10, "
                               "nu_l/nu_v=10, sigma=1e-3, M=0.05",
                   "lattice": "D3Q19", "nodes_per_step": nodes, "diag_every": args.diag_every,
                   "l2": "inputs larger than L2, steps back to back"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                     "peak_source": f"{src} copy bandwidth (hbm_gbs)",
                     "algorithmic_bytes_per_node": bpn, "step_ms": step_s * 1e3,
                     "kernel": ("d3q19_off_phi_kernel + d3q19_off_pass_kernel" if "off" in args.precision
                                else "d3q19_phi_kernel + d3q19_pass_kernel") + " (whole step)"},
        "e2e": {"value": nodes * args.steps * world / e2e_s / 1e6, "unit": "MLUPS",
                "h2d_bytes_per_step": 8 * nodes / args.steps,
                "d2h_bytes_per_step": (8 * nodes + n_diag * ctypes_sizeof_diag()) / args.steps,
                "how": "wall clock through the C ABI: lbm_init_phi from pinned host phi0, "
                       "lbm_step in chunks of diag_every steps each followed by "
                       "lbm_diagnostics (device-to-host read), final phi by lbm_moments to "
                       "pinned host memory"},
        "mass_drift_rel": (d_last["sum_phi"] - d_first["sum_phi"]) / d_first["sum_phi"],
        "u_max_final": d_last["u_max"],
        "clocks": clk.summary(t_start, t_end),
        # two passes per step; per chunk the diagnostics (both passes and the
        # reduction) plus the FP32 shift update or the offset-scale refresh
        "gpu_launches": 2 * args.steps + len(plan) * (
            4 if args.precision == "fp32" else (6 if "off" in args.precision else 3)),
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_coalescence3d()
    print(json.dumps(line), flush=True)


def run_adjoint(args, rank, world, local_rank):
    """Gradient of L = sum (phi_N - phi_target)^2 with respect to phi0, sigma
    and M through the discrete adjoint (workloads.COALESCENCE_ADJ: 512^2, two
    droplets R = 48, centres 2R + W apart; checkpoints every 100 steps).  The
    target is the final phi of a run from phi0 + 1e-3 N(0, 1), default_rng(0).
    `value` counts node updates of the differentiated run per second of
    forward + backward; the plain forward of the same run is timed beside it."""
    import numpy as np
    import torch

    from paper_2311_10827_gb300 import build as B
    B.build()
    from paper_2311_10827_gb300 import workloads as wl
    from paper_2311_10827_gb300.adjoint import rollout
    from paper_2311_10827_gb300.sim import Simulation
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    cfg = wl.COALESCENCE_ADJ
    nx, ny = cfg["shape"]
    prm = wl.physical(cfg)
    sigma0, M0 = prm.pop("sigma"), prm.pop("M")
    phi0 = wl.two_droplets(nx, ny, cfg["R"], cfg["W"])
    noisy = phi0 + 1e-3 * np.random.default_rng(0).standard_normal(phi0.shape)
    nsteps = args.steps
    ts = Simulation((nx, ny), precision=args.precision, sigma=sigma0, M=M0, **prm)
    ts.init_phi(noisy)
    ts.step(nsteps)
    target = torch.tensor(ts.moments()["phi"], device=dev)
    ts.close()
    p0 = torch.tensor(phi0, device=dev)

    def one():
        x = p0.clone().requires_grad_(True)
        sg = torch.tensor(sigma0, dtype=torch.float64, device=dev, requires_grad=True)
        mo = torch.tensor(M0, dtype=torch.float64, device=dev, requires_grad=True)
        phiN = rollout(x, sg, mo, shape=(nx, ny), nsteps=nsteps, checkpoint_every=100,
                       precision=args.precision, **prm)
        L = ((phiN - target) ** 2).sum()
        L.backward()
        return float(L.detach()), x.grad, float(sg.grad), float(mo.grad)

    stream = torch.cuda.current_stream()  # the library runs on it (adjoint.rollout)
    one()  # warm-up (builds graphs, touches allocations)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        t_start = time.time()
        t = time.perf_counter()
        e0.record(stream)
        L, g0, gs, gm = one()
        e1.record(stream)
        torch.cuda.synchronize()
        t_grad = max_over_ranks_dist(time.perf_counter() - t, world, dev)
        t_end = time.time()
    dev_s = max_over_ranks_dist(e0.elapsed_time(e1) / 1e3, world, dev)
    fs = Simulation((nx, ny), precision=args.precision, sigma=sigma0, M=M0, **prm)
    fs.init_phi(phi0)
    fs.step(args.warmup)
    torch.cuda.synchronize()
    t = time.perf_counter()
    fs.step(nsteps)
    fs.sync()
    t_fwd = max_over_ranks_dist(time.perf_counter() - t, world, dev)
    fs.close()

    # end to end through the C ABI with host buffers: phi0 from pinned host
    # memory, the final phi to host, dL/dphi = 2 (phi_N - target) on the host,
    # the backward pass from and to host memory
    import numpy as np

    from paper_2311_10827_gb300 import capi
    hphi0 = torch.tensor(phi0).pin_memory()
    hphiN = torch.empty_like(hphi0).pin_memory()
    hdl = torch.empty_like(hphi0).pin_memory()
    hgrad = torch.empty_like(hphi0).pin_memory()
    htarget = target.cpu().numpy()
    es = Simulation((nx, ny), precision=args.precision, stream=stream.cuda_stream, sigma=sigma0,
                    M=M0, **prm)
    rc, ha = capi.lbm_adjoint_create(es.handle, 100, nsteps)
    capi.check(rc, "lbm_adjoint_create")
    torch.cuda.synchronize()
    t = time.perf_counter()
    capi.check(capi.lbm_adjoint_forward(ha, hphi0.numpy(), 0, nsteps))
    capi.check(capi.lbm_moments(es.handle, hphiN.numpy(), None, None, None, 0))
    np.multiply(2.0, hphiN.numpy() - htarget, out=hdl.numpy())
    rc, eg = capi.lbm_adjoint_backward(ha, hdl.numpy(), 0, hgrad.numpy())
    capi.check(rc, "lbm_adjoint_backward")
    torch.cuda.synchronize()
    e2e_s = max_over_ranks_dist(time.perf_counter() - t, world, dev)
    capi.lbm_adjoint_destroy(ha)
    es.close()
    if not np.isfinite(hgrad.numpy()).all():
        raise RuntimeError("non-finite gradient in the end-to-end run")
    if rank != 0:
        return
    nodes = nx * ny
    peaks, src = measured_peaks()
    bpn = adjoint_bytes_per_node(4 if args.precision == "fp32" else 8)
    achieved = bpn * nodes * nsteps / dev_s / 1e9
    line = {
        "metric": "MLUPS (fused f+g step), differentiated: forward + adjoint",
        "value": nodes * nsteps * world / t_grad / 1e6, "unit": "MLUPS", "n_gpus": world,
        "steps": nsteps, "warmup": nsteps, "ms_per_step": t_grad / nsteps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f64",
        "data": "synthetic",
        "config": {"workload": f"2D two-droplet coalescence {nx}x{ny}, R=48, W=8, "
                               "sigma=5e-3, M=0.1, rho_l/rho_v=10, nu_l/nu_v=1; loss = "
                               "sum (phi_N - phi_target)^2, target from phi0 + 1e-3 N(0,1) "
                               "(default_rng(0)); checkpoint every 100 steps",
                   "warmup": "one whole gradient of the same run before the timed one",
                   "l2": "one step's state (2 x 21 MB) and adjoint fields fit the 129 MB L2"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                     "peak_source": f"{src} copy bandwidth (hbm_gbs)",
                     "algorithmic_bytes_per_node": bpn, "device_s": dev_s,
                     "kernel": "whole gradient (recorded forward, segment recomputation with "
                               "moments, adj_local + adj_mu_phi per reverse step); one "
                               "step's data (2 x 21 MB) fits the 129 MB L2"},
        "e2e": {"value": nodes * nsteps * world / e2e_s / 1e6, "unit": "MLUPS",
                "h2d_bytes_per_step": 2 * 8 * nodes / nsteps,
                "d2h_bytes_per_step": (2 * 8 * nodes + 32) / nsteps,
                "how": "wall clock through the C ABI: lbm_adjoint_forward from pinned host "
                       "phi0, lbm_moments of the final phi to host, dL/dphi on the host, "
                       "lbm_adjoint_backward from and to host memory"},
        "gradient_s": t_grad, "forward_only_s": t_fwd,
        "plain_step_MLUPS": nodes * nsteps / t_fwd / 1e6,
        "cost_vs_plain_forward": t_grad / t_fwd,
        "loss": L, "dL_dsigma": gs, "dL_dM": gm,
        "dL_dphi0_norm": float(g0.norm()),
        "e2e_dL_dsigma": eg[0],
        "clocks": clk.summary(t_start, t_end),
        # per gradient: initial condition (2), nsteps recorded steps, the
        # final phi (1), the seed, nsteps recomputation passes (one
        # moments-only per segment among them), 2 reverse kernels per step,
        # the initial-condition reverse (2)
        "gpu_launches": 4 * nsteps + 6,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_adjoint()
    print(json.dumps(line), flush=True)


def max_over_ranks_dist(x, world, device):
    """Max of a float over the ranks (identity for one rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def ctypes_sizeof_diag():
    import ctypes

    from paper_2311_10827_gb300 import capi
    return ctypes.sizeof(capi.lbm_diag)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--precision", choices=["fp32", "fp64", "f16off", "bf16off"], default="fp32",
                    help="f16off / bf16off: 16-bit offset storage (coalescence3d only)")
    ap.add_argument("--diag-every", type=int, default=100)
    ap.add_argument("--min-time", type=float, default=1.0,
                    help="droplet1024: repeat the timed region of --steps steps until about "
                         "this many seconds of timed work (clock samples)")
    ap.add_argument("--repeat-min", type=int, default=3)
    ap.add_argument("--repeat-max", type=int, default=2000)
    ap.add_argument("--e2e-runs", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the FP64 comparison run after the timed region (profiling)")
    ap.add_argument("--per-step", action="store_true",
                    help="droplet1024: one launch per step even when the tuned tiles fit the GPU "
                         "at once (default there: one cooperative launch per chunk of steps)")
    ap.add_argument("--tile", default="", help="WxR: fixed batch tile shape instead of the "
                    "autotuner (profiling commands use the shape the tuner picked)")
    ap.add_argument("--workload", choices=["droplet1024", "ensemble", "coalescence3d", "adjoint"],
                    default="droplet1024",
                    help="droplet1024: the headline line; ensemble: the 256-grid batch; "
                         "coalescence3d: the 512^3 D3Q19 run; adjoint: the 512^2 gradient")
    ap.add_argument("--size", type=int, default=0,
                    help="droplet1024: edge of the square grids (default 1024; 4096 is the "
                         "out-of-L2 point); coalescence3d: edge of the cube (default 512)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if "off" in args.precision and args.workload != "coalescence3d":
        ap.error("offset storage is built for the D3Q19 path (--workload coalescence3d)")
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        if args.workload == "ensemble":
            run_ensemble(args, rank, world, local_rank)
        elif args.workload == "coalescence3d":
            run_coalescence3d(args, rank, world, local_rank)
        elif args.workload == "adjoint":
            run_adjoint(args, rank, world, local_rank)
        else:
            run_native(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
