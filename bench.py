#!/usr/bin/env python
"""Throughput of the fused phase-field LBM step on GB300.

Workload: the 2D stationary droplet, 1024 x 1024 periodic, R = 128 centred,
W = 4, sigma = 1e-3, M = 0.05 (alpha = 1), viscosity ratio 10 (nu_l = 1,
nu_v = 0.1), D2Q9, FP32; one bench step advances both density-ratio cases
(rho_l/rho_v = 10 and 100) by one time step (two launches of the fused
kernel).  Synthetic input: the tanh droplet of the paper's stationary-droplet
test (Section 3.2), no dataset involved.

Metric: MLUPS (million node updates per second, both populations).  `value`
is device time (CUDA events around every timed step on the launching
stream), steps back to back: each step's inputs (2 x 79 MB) exceed the
129 MB L2 and each grid is re-read only after the other grid's pass, so
reads come from HBM and every kernel pays the write-backs of the one before
(--l2-flush instead writes and reads a 256 MiB buffer between timed steps,
outside the events).  `e2e` is wall-clock through the C ABI with host
buffers: pinned host phi0 uploaded by lbm_init_phi, every step followed by a
device-to-host read of the run's latest diagnostics record (refreshed by the
fused diagnostics every --diag-every steps), the final fields read back by
lbm_moments.

Multi-GPU: replicas only (every rank runs its own pair of grids, weak
scaling; the only collectives are the timing barrier and max).

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
# bytes moved per node update: f, g read + write (4 Q s) and S read + write;
# FP32 also moves the low word of the rest population pair (8 B)
BYTES_PER_NODE = {"fp32": 160, "fp64": 304}
L2_FLUSH_BYTES = 256 << 20
KERNEL_SOURCES = ("paper_2311_10827_gb300/csrc/kernels_d2q9.cu",)
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_d2q9_fp32_droplet1024.txt")


def params(ratio):
    from paper_2311_10827_gb300 import workloads as wl
    p = wl.physical(wl.DROPLET_1024)
    p["rho_l"] = ratio * p["rho_v"]
    return p


def phi0():
    from paper_2311_10827_gb300 import workloads as wl
    return wl.droplet(NX, NY, wl.DROPLET_1024["R"], wl.DROPLET_1024["W"])


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken
    on the kernel source as it is now."""
    try:
        kv = {}
        with open(TRAFFIC_FILE) as fh:
            for line in fh:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_sha") != kernel_hash():
            return None
        return float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for _, _, r in rows for k in range(4)
                          if r[k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


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


def run_native(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2311_10827_gb300 import build as B
    B.build()
    from paper_2311_10827_gb300 import capi
    from paper_2311_10827_gb300.sim import Simulation

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    prec = args.precision
    sims = [Simulation((NX, NY), precision=prec, stream=stream.cuda_stream,
                       diag_every=args.diag_every, **params(r)) for r in RATIOS]
    phi_d = torch.tensor(phi0(), dtype=torch.float64, device=dev)
    for s in sims:
        s.init_phi(phi_d)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def l2_flush(i):
        flush.fill_(float(i))
        flush.sum()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for i in range(args.warmup):
        if args.l2_flush:
            l2_flush(i)
        for s in sims:
            s.step(1)
    barrier()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(sims) + 1)]
           for _ in range(args.steps)]
    t_first = sims[0].t
    with ClockSampler(local_rank) as clk:
        t_wall = time.perf_counter()
        for k in range(args.steps):
            if args.l2_flush:
                l2_flush(k)
            starts[k].record(stream)
            kev[k][0].record(stream)
            for j, s in enumerate(sims):
                s.step(1)
                kev[k][j + 1].record(stream)
            ends[k].record(stream)
        barrier()
        t_wall = time.perf_counter() - t_wall
    step_ms = [starts[k].elapsed_time(ends[k]) for k in range(args.steps)]
    # single-kernel durations of plain steps (no fused diagnostics at that step)
    de = args.diag_every
    plain = [kev[k][j].elapsed_time(kev[k][j + 1]) for k in range(args.steps)
             for j in range(len(sims)) if de == 0 or (t_first + k) % de != 0]
    total_s = sum(step_ms) / 1e3
    if world > 1:
        t = torch.tensor([total_s], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    nodes = NX * NY * len(sims)
    value = nodes * args.steps * world / total_s / 1e6

    # ---- end to end through the C ABI with host buffers
    hphi = torch.tensor(phi0(), dtype=torch.float64).pin_memory()
    hphi_np = hphi.numpy()
    e2e_steps = args.steps
    outs = [dict(phi=np.empty(NX * NY), p=np.empty(NX * NY), mu=np.empty(NX * NY),
                 u=np.empty(2 * NX * NY)) for _ in sims]
    e2e_sims = [Simulation((NX, NY), precision=prec, stream=stream.cuda_stream,
                           diag_every=args.diag_every, **params(r)) for r in RATIOS]
    barrier()
    t0 = time.perf_counter()
    for s in e2e_sims:
        capi.check(capi.lbm_init_phi(s.handle, hphi_np, 0))
    for k in range(e2e_steps):
        for s in e2e_sims:
            capi.check(capi.lbm_step(s.handle, 1))
        for s in e2e_sims:
            rc, d = capi.lbm_last_diagnostics(s.handle)
            capi.check(rc)
    for s, o in zip(e2e_sims, outs):
        capi.check(capi.lbm_moments(s.handle, o["phi"], o["p"], o["u"], o["mu"], 0))
    barrier()
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = nodes * e2e_steps * world / e2e_s / 1e6
    diag_bytes = ctypes_sizeof_diag()
    h2d = NX * NY * 8 * len(sims) / e2e_steps
    d2h = diag_bytes * len(sims) + 5 * NX * NY * 8 * len(sims) / e2e_steps
    for s in e2e_sims:
        s.close()

    if rank != 0:
        return
    peaks, src = measured_peaks()
    avg_kernel_s = statistics.mean(plain) / 1e3 if plain else None
    bpn = BYTES_PER_NODE[prec]
    achieved = bpn * NX * NY / avg_kernel_s / 1e9 if avg_kernel_s else None
    traffic = ncu_traffic() if prec == "fp32" else None
    n_diag = sum(1 for k in range(args.steps) if de > 0 and (t_first + k) % de == 0)
    line = {
        "metric": "MLUPS (fused f+g step)", "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_s / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64",
        "data": "synthetic",
        "config": {"workload": "2D stationary droplet 1024x1024 periodic, R=128, W=4, "
                               "sigma=1e-3, M=0.05, nu_l/nu_v=10, rho_l/rho_v=10 and 100 "
                               "(one step = both grids)",
                   "lattice": "D2Q9", "nodes_per_step": nodes, "diag_every": de,
                   "l2": ("256 MiB write+read flush between timed steps, outside the events"
                          if args.l2_flush else
                          "inputs larger than L2: 2 x 79 MB per step, back to back"),
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"] if achieved else None,
                     "traffic": traffic, "peak_source": f"{src} copy bandwidth (hbm_gbs)",
                     "algorithmic_bytes_per_node": bpn,
                     "kernel_ms": avg_kernel_s * 1e3 if avg_kernel_s else None},
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "how": "lbm_init_phi from pinned host phi0, per step lbm_step + "
                       "lbm_last_diagnostics (D2H of the latest diagnostics record), final "
                       "lbm_moments to host; wall clock"},
        "gpu_launches": args.steps * len(sims) + n_diag * len(sims),
        "clocks": clk.summary(),
        "wall_s_timed_region": t_wall,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


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
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--diag-every", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--l2-flush", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        run_native(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
