"""Benchmark of the fused B-TriRT D2Q9 sweep on GB300.

Workload (N = 1): the linear anisotropic manufactured-solution problem at
8192 x 8192 nodes with half-way bounce-back walls, FP64, full diffusion tensor
R(pi/6) diag(0.05, 0.01) R(pi/6)^T, u = (0.05, 0.02), diffusive scaling
dt = 4 dx^2.  One bench step = one time step of the whole lattice (one fused
sweep launch).  Inputs (4.8 GB of populations) are far larger than L2, so no
flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs an independent replica (the method has
no exchange between independent solves); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "B-TriRT D2Q9 MLUPS & % HBM roofline; served solves/s + p50/p99 vs plain"
N_MAIN = 8192
BYTES_PER_UPDATE = {"f64": 160, "f32": 80, "f16": 44, "bf16": 44}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi sampling during the timed region (SM clock, throttle reasons)."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------- GPU arm
def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import workloads as w
    from paper_1902_09813_gb300 import Lattice

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    if args.workload == "mms":
        p = w.mms_sinsin(n=args.n, nsteps=args.steps)
        desc = (f"linear anisotropic CDE, manufactured solution, HBB walls, {p.nx}x{p.ny}, "
                f"{args.compute.upper()} compute, {args.storage.upper()} storage, {args.steps} steps")
    else:
        p = w.nonlinear_modes(n=args.n, nsteps=args.steps)
        p.phi_ref = 0.0
        desc = (f"nonlinear anisotropic CDE, 16 Fourier modes, periodic, {p.nx}x{p.ny}, "
                f"{args.compute.upper()} compute, {args.storage.upper()} storage, {args.steps} steps")
    phi0 = p.phi0()
    if args.workload != "mms":
        p.phi_ref = float(phi0.mean())
    nodes = p.nx * p.ny
    stream = torch.cuda.Stream()
    lat = Lattice.from_problem(p, compute=args.compute, storage=args.storage, stream=stream)
    lat.init(phi0)
    # warm-up
    lat.step(args.warmup)
    torch.cuda.synchronize()

    clocks = ClockSampler(local).start()
    time.sleep(0.3)
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    lat.step(args.steps)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    t_local = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if ws > 1:
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
    ms_max = float(t_local.item())
    lat.check()
    mlups = ws * nodes * args.steps / (ms_max * 1e-3) / 1e6

    # dominant kernel: the sweep, one launch per step on `stream`
    t_launch = ms / args.steps * 1e-3
    peak_hbm, peak_kind = _peaks()
    alg_bytes = BYTES_PER_UPDATE[args.storage] * nodes
    achieved_gbs = alg_bytes / t_launch / 1e9

    # end to end through the public API with host buffers: H2D of phi0 from pinned
    # memory, K steps, D2H of phi, all inside the timed region
    e2e_mlups = None
    if not args.no_e2e:
        phi0_pinned = torch.from_numpy(phi0).pin_memory()
        out_pinned = torch.empty((p.ny, p.nx), dtype=torch.float64).pin_memory()
        barrier()
        t0 = time.perf_counter()
        lat.init(phi0_pinned)
        lat.step(args.steps)
        lat.phi(out=out_pinned)
        stream.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e_t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        if ws > 1:
            dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
        e2e_mlups = ws * nodes * args.steps / float(e2e_t.item()) / 1e6

    extra = {}
    if rank == 0 and not args.no_cpu_baseline:
        extra["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(mlups, 2), "unit": "MLUPS",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.compute, "data": "synthetic",
            "config": {"workload": desc, "nx": p.nx, "ny": p.ny,
                       "parallelism": "replicas" if ws > 1 else "single",
                       "l2": f"inputs {alg_bytes / 2 / 1e9:.2f} GB read per step >> L2, no flush"},
            "roofline": {"bound": "hbm", "achieved": round(achieved_gbs, 1), "peak": peak_hbm,
                         "unit": "GB/s", "frac": round(achieved_gbs / peak_hbm, 4),
                         "traffic": None, "peak_kind": peak_kind,
                         "bytes_per_update": BYTES_PER_UPDATE[args.storage],
                         "kernel": f"sweep_kernel<{args.compute},{args.storage}>"},
            "e2e": None if e2e_mlups is None else {
                "value": round(e2e_mlups, 2), "unit": "MLUPS",
                "h2d_bytes_per_step": int(8 * nodes / args.steps),
                "d2h_bytes_per_step": int(8 * nodes / args.steps),
                "note": "one solve per K steps: phi0 in, phi out, amortised per step"},
            "gpu_launches": args.steps,
            "clocks": clk,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------- CPU oracle
def _oracle_sample(n_side: int):
    """A bounded patch of the benchmark workload: same dx, dt, coefficients and walls
    as the 8192^2 lattice, on an n_side x n_side sub-grid."""
    import workloads as w
    p = w.mms_sinsin(n=N_MAIN, nsteps=1)
    return p.replace(nx=n_side, ny=n_side)


def cpu_baseline(args, seconds: float = 12.0):
    import oracle
    cores = _cores()
    p = _oracle_sample(1024)
    lat = oracle.OracleLattice(p, nthreads=cores).init()
    lat.step(1)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        lat.step(2)
        steps += 2
    el = time.perf_counter() - t0
    return {"value": round(p.nx * p.ny * steps / el / 1e6, 3), "unit": "MLUPS", "cores": cores,
            "kind": "oracle",
            "sample": f"{p.nx}x{p.ny} patch of the benchmark lattice (same dx, dt, coefficients, "
                      f"walls), {steps} steps, {el:.1f} s, OpenMP over rows"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    cores = _cores()
    p = _oracle_sample(512)
    lat = oracle.OracleLattice(p, nthreads=cores).init()
    lat.step(args.warmup)
    t0 = time.perf_counter()
    lat.step(args.steps)
    el = time.perf_counter() - t0
    mlups = p.nx * p.ny * args.steps / el / 1e6
    sample = (f"{p.nx}x{p.ny} patch of the 8192x8192 benchmark lattice per step "
              f"(same dx, dt, coefficients, walls)")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(mlups, 3), "unit": "MLUPS",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(el / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "linear anisotropic CDE, manufactured solution, HBB walls, FP64 "
                               "(FP64 CPU oracle on a bounded patch)", "nx": p.nx, "ny": p.ny},
        "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="mms", choices=["mms", "nonlinear"])
    ap.add_argument("--n", type=int, default=N_MAIN)
    ap.add_argument("--compute", default="f64", choices=["f64", "f32"])
    ap.add_argument("--storage", default=None, choices=["f64", "f32", "f16", "bf16"])
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.storage is None:
        args.storage = args.compute
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
