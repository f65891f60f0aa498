#!/usr/bin/env python3
"""Benchmark of the Dirac Lanczos propagator: Lanczos H.psi site-updates/s.

One benchmark step is one time step of the propagator (all of: Lanczos passes
with fused stencil and reductions, the small exponential, the recombination)
on the laser-packet workload: 1024x1024 grid, dx = 0.05 au, Krylov m = 20,
dt = 2e-4 au, free Gaussian packet (width 1 au, p0 = (10, 0) au, positive
energy) in A_x(t) = 50 sin^2(pi t) sin(0.05 t), as in Sec. 7 of the paper
with a laser field.  value = sites * m * steps / time (whole job).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): every rank propagates its own packet (independent
replicas, weak scaling); only the timing is reduced across ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1407_7370_gb300 import workloads as wl  # noqa: E402

METRIC = "Lanczos H*psi site-updates/s (FP64 path)"
UNIT = "site-updates/s"
CFG = wl.LASER_PACKET_1024
SITE_BYTES = 32            # complex128 spinor
PASS_BYTES_PER_SITE = 3 * SITE_BYTES   # read q_i, read q_{i-1}, write q_{i+1} (V = 0)
PASS_FLOPS_PER_SITE = 80   # FP64 flops of one Lanczos iteration per site


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms (read-only)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 7:
                    rows.append(parts)
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# CPU oracle (the baseline and the reference arm only)
# ----------------------------------------------------------------------------
def oracle_site_updates(grid_side: int, steps: int):
    """Time the CPU oracle on `steps` time steps of the workload on a grid_side^2 crop."""
    from oracle import hamiltonian as ham
    from oracle import lanczos as lz
    g = wl.Grid(grid_side, grid_side, CFG["grid"].dx, CFG["grid"].dy)
    psi = wl.positive_energy_packet(g, p0=CFG["p0"], sigma_x=CFG["sigma_x"])
    op = ham.Operator(g.nx, g.ny, g.dx, g.dy)
    c0, w0 = os.times(), time.perf_counter()
    lz.propagate(op, psi, CFG["dt"], CFG["m"], steps, pulse=CFG["pulse"], t0=0.0)
    c1, w1 = os.times(), time.perf_counter()
    wall = w1 - w0
    cpu = (c1.user - c0.user) + (c1.system - c0.system)
    return g.n_sites * CFG["m"] * steps / wall, wall, max(1, round(cpu / wall))


def cpu_baseline():
    side = CFG["grid"].nx
    rate, wall, cores = oracle_site_updates(side, 2)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "2 time steps of the %dx%d laser-packet workload (m=%d), numpy FP64 oracle, "
                      "%.1f s wall" % (side, side, CFG["m"], wall)}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    # each step: one time step on a crop sized so (warmup + steps) fit in ~150 s
    rate0, wall0, _ = oracle_site_updates(64, 1)
    per_site_update = 1.0 / rate0
    budget = 150.0 / max(1, args.steps + args.warmup)
    side = int(math.sqrt(budget / (CFG["m"] * per_site_update)))
    side = max(32, min(CFG["grid"].nx, side - side % 8))
    oracle_site_updates(side, args.warmup) if args.warmup else None
    rate, wall, cores = oracle_site_updates(side, args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * wall / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": CFG["name"], "sample_grid": "%dx%d" % (side, side)},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d time steps on a %dx%d crop of the workload"
                                       % (args.steps, side, side)},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist
    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1407_7370_gb300 import build as bld
    if rank == 0 or world == 1:
        bld.build()
    if world > 1:
        dist.barrier()
    from paper_1407_7370_gb300 import Propagator
    from paper_1407_7370_gb300.propagator import pulse_schedule

    g, m, dt, pulse = CFG["grid"], CFG["m"], CFG["dt"], CFG["pulse"]
    psi0 = wl.positive_energy_packet(g, p0=CFG["p0"], sigma_x=CFG["sigma_x"])
    K, W = args.steps, args.warmup
    A = pulse_schedule(0.0, dt, W + 2 * K, pulse.a0, pulse.omega, pulse.duration)
    prop = Propagator(g.nx, g.ny, g.dx, g.dy, m_max=m)
    prop.set_fields(None, A=(0.0, 0.0))
    psi = torch.from_numpy(psi0).cuda()
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up
    prop.steps(psi, W, dt, m, A=A[:W])
    barrier()
    # timed region: K steps, device time by CUDA events on the launching stream
    clocks = ClockSampler(local)
    clocks.start()
    l0 = prop.kernel_launches
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    prop.steps(psi, K, dt, m, A=A[W:W + K])
    e1.record(stream)
    barrier()
    launches = prop.kernel_launches - l0
    clk = clocks.stop()
    t = e0.elapsed_time(e1) / 1e3
    if world > 1:
        tt = torch.tensor([t], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    value = world * g.n_sites * m * K / t

    # per-kernel device durations inside a second timed run of the same K steps
    prop.profile(True)
    info0 = prop.steps(psi, K, dt, m, A=A[W + K:W + 2 * K], info=True)
    prof = prop.profile_read()
    prop.profile(False)
    pass_ms, pass_n = prof["pass"]
    rec_ms, rec_n = prof["recombine"]
    pass_avg = pass_ms / pass_n / 1e3
    pk = peaks()
    # FP64 ALU roof: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
    fp64_peak = 152 * 2 * 2 * 2.07e9 / 1e12
    flops = PASS_FLOPS_PER_SITE * g.n_sites / pass_avg / 1e12
    hbm_peak = pk.get("hbm_gbs", 6800.0)
    gbs = PASS_BYTES_PER_SITE * g.n_sites / pass_avg / 1e9
    roofline = {"bound": "alu", "achieved": flops, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": flops / fp64_peak, "traffic": None,
                "kernel": "lanczos_pass", "kernel_avg_us": pass_avg * 1e6,
                "kernel_share": pass_ms / (pass_ms + rec_ms),
                "peak_source": "derived FP64 FMA rate (probe: 1.19 TFLOP/s measured)"}
    hbm = {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
           "bytes_per_site": PASS_BYTES_PER_SITE,
           "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in pk else "fallback"}

    # end to end through the host-buffer C-ABI call: pinned H2D + step + D2H per step
    host = torch.from_numpy(psi.cpu().numpy()).pin_memory()
    Ke = max(3, min(K, 200))
    barrier()
    w0 = time.perf_counter()
    for n in range(Ke):
        prop.propagate_host(host, 1, dt, m, A=A[W + (n % K):W + (n % K) + 1])
    w1 = time.perf_counter()
    te = w1 - w0
    if world > 1:
        tt = torch.tensor([te], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        te = float(tt.item())
    bytes_step = g.n_sites * SITE_BYTES
    e2e = {"value": world * g.n_sites * m * Ke / te, "unit": UNIT,
           "h2d_bytes_per_step": bytes_step, "d2h_bytes_per_step": bytes_step,
           "steps": Ke, "api": "dirac_propagate_host (pinned host buffer, 1 step per call)"}

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": W, "ms_per_step": 1e3 * t / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": CFG["name"], "grid": "%dx%d" % (g.nx, g.ny),
                           "dx": g.dx, "m": m, "dt": dt, "order": 2, "boundary": "periodic",
                           "pulse": "A_x = 50 sin^2(pi t) sin(0.05 t), T = 1",
                           "l2": "inputs larger than L2: Krylov basis %.0f MB per step"
                                 % (m * g.n_sites * SITE_BYTES / 1e6),
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": roofline, "hbm": hbm, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk,
                "diagnostics": {"k_used": info0.k_used, "err_est_last": info0.err_est,
                                "cum_err_est": info0.cum_err, "energy": info0.energy,
                                "recombine_avg_us": rec_ms / max(1, rec_n) * 1e3}}
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline()
        elif not args.no_cpu_baseline:
            line["cpu_baseline"] = None
        print(json.dumps(line), flush=True)
    prop.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
