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
BYTES_PER_UPDATE = {"f64": 160, "df64": 160, "f32": 80, "f16": 44, "bf16": 44}


def state_bytes(storage: str, shift: str = "auto") -> int:
    """Algorithmic bytes per update: one read and one write of the state (the 9
    populations and phi; a double-word phi adds its FP32 low words, the
    first-moment form its two 16-bit planes)."""
    extra = 8 if shift in ("local_dw", "local_dw_sr", "moment_sr") else 0
    return BYTES_PER_UPDATE[storage] + extra


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


CSRC = os.path.join(ROOT, "paper_1902_09813_gb300", "csrc")


def source_digest(names) -> str:
    """sha256 (first 16 hex digits) of kernel source files, in the given order."""
    import hashlib
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(CSRC, n), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _header_count(name: str) -> int:
    """An integer constant kept next to the kernel code it describes."""
    import re
    with open(os.path.join(CSRC, "btrt_sweep.cuh")) as fh:
        m = re.search(rf"constexpr int {name} = (\d+);", fh.read())
    return int(m.group(1))


# FP64 operations (add, mul or fma, one each) per node of the FP64 headline sweep,
# counted from the kernel source next to collide_fold, in total and by kind.
FP64_OPS_PER_UPDATE_LINEAR = _header_count("kFp64OpsPerNodeLinearTrig")
FP64_MIX_PER_UPDATE = {"add": _header_count("kFp64AddsPerNodeLinearTrig"),
                       "fma": _header_count("kFp64FmasPerNodeLinearTrig"),
                       "mul": _header_count("kFp64MulsPerNodeLinearTrig")}
# GB300's nominal FP64 rate, 1.25 TFLOP/s = 0.625 T FMA/s = 0.625 T FP64
# operations/s when every add, mul or fma takes one lane slot; reported beside the
# rate measured in the run (btrt_probe_fp64_rate), which is the roofline's peak.
FP64_NOMINAL_TOPS = 0.625
# DRAM bytes per node of one FP64 sweep launch measured by ncu
# (dram__bytes_read.sum + dram__bytes_write.sum) on the same kernel at 2048^2,
# scaled to the benchmark by node count.  The operation count and this capture
# hold for the kernel sources whose digest is FP64_SWEEP_DIGEST; after an edit
# to them both are re-taken and the digest updated (a CPU test checks it), and
# until then the traffic is reported as null.
FP64_SWEEP_SOURCES = ("btrt_sweep.cuh", "btrt_dw.cuh")   # the FP64 sweep's device code
FP64_SWEEP_DIGEST = "84f1a8f8aaf78b87"
FP64_TRAFFIC_PER_NODE = 149.3
# DRAM bytes per node and step of the two-step FP32-compute kernel measured by ncu,
# keyed by (storage, shift), for the sources with digest TB2_DIGEST.
TB2_SOURCES = ("btrt_sweep.cuh", "btrt_tb.cuh", "btrt_launch.cuh")
TB2_DIGEST = "a989bb60b344a85f"
TB2_DRAM_BYTES_PER_UPDATE = {("f32", "ref"): 38.6, ("f16", "local"): 20.9}
# DRAM bytes per node of one launch of the vector-access sweep measured by ncu,
# keyed by (storage, shift), for the sources with digest VEC_DIGEST.
VEC_SOURCES = ("btrt_sweep.cuh", "btrt_vec.cuh", "btrt_launch.cuh")
VEC_DIGEST = "253f0579e2e2edee"
VEC_DRAM_BYTES_PER_UPDATE = {("f16", "local"): 41.4, ("f16", "local_sr"): 41.2}


def measure_fp64_peak(iters: int = 2000):
    """FP64 operation rates of the probe kernel on the current device: for each kind
    (FMA, add, multiply) the best of 4, 8 and 16 independent chains per thread,
    and the peak of the FP64 sweep's own mix of kinds, FP64_MIX_PER_UPDATE:
    sum(n_k) / sum(n_k / rate_k) operations per second."""
    import ctypes

    import torch
    from paper_1902_09813_gb300 import _capi as C
    lib = C.load()
    sink = torch.zeros(8, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    rates = {}
    for name, kind in (("fma", C.PROBE_FMA), ("add", C.PROBE_ADD), ("mul", C.PROBE_MUL)):
        best = 0.0
        for chains in (4, 8, 16):
            rate, ms = ctypes.c_double(), ctypes.c_double()
            C.check(lib.btrt_probe_fp64_rate(ctypes.c_void_p(stream.cuda_stream), kind, chains, iters,
                                             ctypes.c_void_p(sink.data_ptr()), ctypes.byref(rate),
                                             ctypes.byref(ms)))
            best = max(best, rate.value)
        rates[name] = best
    n = sum(FP64_MIX_PER_UPDATE.values())
    mix = n / sum(FP64_MIX_PER_UPDATE[k] / rates[k] for k in FP64_MIX_PER_UPDATE)
    return {"tops": round(mix / 1e12, 4),
            "by_kind_tops": {k: round(v / 1e12, 4) for k, v in rates.items()},
            "mix": dict(FP64_MIX_PER_UPDATE),
            "kernel": "fp64_chains (4/8/16 independent chains per thread, whole waves, best per kind)"}


def kernel_form(args) -> str:
    """The kernel form of the timed steps: what the library's AUTO resolves to for
    FP32 compute (the vector form for FP16/BF16 storage on lattices of 2^21 nodes
    or more, two steps per launch otherwise), the form asked for, or the plain
    sweep."""
    if args.compute != "f32" or args.shift in ("local_dw", "local_dw_sr"):
        return "plain"
    if args.sweep != "auto":
        return args.sweep
    large = args.n * args.n >= 1 << 21
    if args.shift in ("local_sr", "moment_sr"):
        return "vec" if large else "plain"
    return "vec" if args.storage in ("f16", "bf16") and large else "tb2"


def two_step_form(args) -> bool:
    """Pairs of steps in one launch (the scalar or the vector two-step kernel)."""
    return kernel_form(args) in ("tb2", "tb2v")



def roofline(args, nodes, t_launch, achieved_gbs, peak_hbm, peak_kind, fp64_peak=None):
    hbm = {"bound": "hbm", "achieved": round(achieved_gbs, 1), "peak": peak_hbm, "unit": "GB/s",
           "frac": round(achieved_gbs / peak_hbm, 4), "peak_kind": peak_kind,
           "frac_of_nominal_8tbs": round(achieved_gbs / 8000.0, 4),
           "bytes_per_update": state_bytes(args.storage, args.shift)}
    if two_step_form(args):
        # algorithmic bytes count one read and one write of the state per step; the
        # two-step kernel moves about half of that through DRAM, so this fraction
        # can exceed 1 (the DRAM bytes it measured are in `dram_bytes_per_update`)
        shift = args.shift if args.shift != "auto" else ("local" if args.storage in ("f16", "bf16") else "ref")
        key = (args.storage, shift)
        fresh = source_digest(TB2_SOURCES) == TB2_DIGEST
        per_update = TB2_DRAM_BYTES_PER_UPDATE.get(key) if fresh else None
        # DRAM bytes of one launch (two steps), from the capture scaled by node count
        traffic = None if per_update is None else round(per_update * 2 * nodes)
        return dict(hbm, traffic=traffic, kernel=f"sweep_tb2_kernel<f32,{args.storage}>",
                    dram_bytes_per_update=per_update,
                    note="two steps per launch; achieved = algorithmic bytes of the steps / time")
    kernel = f"sweep_kernel<{args.compute},{args.storage}>"
    if kernel_form(args) == "vec":
        shift = args.shift if args.shift != "auto" else ("local" if args.storage in ("f16", "bf16") else "ref")
        fresh = source_digest(VEC_SOURCES) == VEC_DIGEST
        per_update = VEC_DRAM_BYTES_PER_UPDATE.get((args.storage, shift)) if fresh else None
        return dict(hbm, traffic=None if per_update is None else round(per_update * nodes),
                    dram_bytes_per_update=per_update, kernel=f"sweep_vec_kernel<f32,{args.storage}>")
    if args.compute != "f64" or args.workload != "mms":
        return dict(hbm, traffic=None, kernel=kernel)
    # the FP64 sweep is bound by GB300's FP64 pipe, not by HBM
    tops = FP64_OPS_PER_UPDATE_LINEAR * nodes / t_launch / 1e12
    fresh = source_digest(FP64_SWEEP_SOURCES) == FP64_SWEEP_DIGEST
    traffic = round(FP64_TRAFFIC_PER_NODE * nodes) if fresh else None
    if fp64_peak:
        peak, kind = fp64_peak["tops"], (f"measured in this run: probe rates by kind {fp64_peak['by_kind_tops']} "
                                         f"T op/s combined over the sweep's mix {fp64_peak['mix']} "
                                         f"(GB300 nominal FP64 1.25 TFLOP/s = {FP64_NOMINAL_TOPS} T op/s)")
    else:
        peak, kind = FP64_NOMINAL_TOPS, "GB300 nominal FP64 1.25 TFLOP/s = 0.625 T op/s (not measured)"
    return {"bound": "alu", "achieved": round(tops, 4), "peak": peak,
            "unit": "T FP64 op/s", "frac": round(tops / peak, 4), "traffic": traffic,
            "ops_per_update": FP64_OPS_PER_UPDATE_LINEAR, "peak_kind": kind,
            "frac_of_nominal": round(tops / FP64_NOMINAL_TOPS, 4),
            "kernel": kernel, "hbm_view": hbm}


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


def aggregate(ms_local: float, units_per_rank: float, device):
    """Whole-job timing across replicas: the slowest rank's time (MAX over ranks)
    and the throughput of all ranks' units over that time.  One process: as is."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return ms, ws * units_per_rank / (ms * 1e-3)


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
    lat = Lattice.from_problem(p, compute=args.compute, storage=args.storage, stream=stream, shift=args.shift)
    if args.compute == "f32":
        lat.set_sweep_variant(args.sweep)
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
    ms_max, lups = aggregate(ms, nodes * args.steps, "cuda")
    lat.check()
    mlups = lups / 1e6

    # dominant kernel: the sweep, one launch per step on `stream`
    t_launch = ms / args.steps * 1e-3
    peak_hbm, peak_kind = _peaks()
    alg_bytes = state_bytes(args.storage, args.shift) * nodes
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
        _, e2e_lups = aggregate(e2e_s * 1e3, nodes * args.steps, "cuda")
        e2e_mlups = e2e_lups / 1e6

    extra = {}
    del lat
    torch.cuda.empty_cache()
    # the FP64 pipe's rate on this GPU, the FP64 sweep's roofline peak
    fp64_peak = measure_fp64_peak() if args.compute == "f64" else None
    if ws > 1:
        # the per-GPU characterisations (variants, accuracy, batching, serving, CPU oracle)
        # are reported at N = 1; replicas only time the headline sweep
        args.no_variants = args.no_accuracy = args.no_batched = args.no_serving = True
        args.no_cpu_baseline = True
    if not args.no_variants:
        extra["variants"] = run_variants(args)
    if not args.no_accuracy:
        extra["accuracy"] = run_accuracy(args)
    if not args.no_batched:
        torch.cuda.empty_cache()
        extra["batched"] = run_batched(args)
    if not args.no_serving:
        extra["serving"] = run_serving(args)
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
            "roofline": roofline(args, nodes, t_launch, achieved_gbs, peak_hbm, peak_kind, fp64_peak),
            "e2e": None if e2e_mlups is None else {
                "value": round(e2e_mlups, 2), "unit": "MLUPS",
                "h2d_bytes_per_step": int(8 * nodes / args.steps),
                "d2h_bytes_per_step": int(8 * nodes / args.steps),
                "note": "one solve per K steps: phi0 in, phi out, amortised per step"},
            "gpu_launches": (args.steps // 2 + args.steps % 2) if two_step_form(args) else args.steps,
            "clocks": clk,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------- variants
def _time_single(p, phi0, compute, storage, steps, warmup, variant="plain", shift="ref"):
    import torch
    from paper_1902_09813_gb300 import Lattice
    stream = torch.cuda.Stream()
    lat = Lattice.from_problem(p, compute=compute, storage=storage, stream=stream, shift=shift)
    if compute == "f32":
        lat.set_sweep_variant(variant)
    lat.init(phi0)
    lat.step(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    lat.check()
    ms = e0.elapsed_time(e1)
    nodes = p.nx * p.ny
    mlups = nodes * steps / (ms * 1e-3) / 1e6
    peak, _ = _peaks()
    gbs = state_bytes(storage, shift) * mlups * 1e6 / 1e9
    del lat
    torch.cuda.empty_cache()
    return {"mlups": round(mlups, 1), "ms_per_step": round(ms / steps, 4),
            "algorithmic_gbs": round(gbs, 1), "hbm_frac": round(gbs / peak, 4)}


def run_variants(args, steps=200, warmup=5):
    """The other compute/storage paths at 8192^2: double-word (FP32-pair) arithmetic
    on the manufactured-solution workload, FP32 compute with FP32/FP16/BF16 shifted
    storage (both shifts: one step per launch plain and with vector access, two
    steps per launch; reference shift: TMA-staged too) on the manufactured-solution
    and nonlinear workloads."""
    import workloads as w
    out = {}
    p = w.mms_sinsin(n=args.n, nsteps=steps)
    phi0 = p.phi0()
    out["mms_df64"] = _time_single(p, phi0, "df64", "df64", steps, warmup)
    q = w.nonlinear_modes(n=args.n, nsteps=steps)
    q_phi0 = q.phi0()
    q.phi_ref = float(q_phi0.mean())
    for name, prob, a in (("mms", p, phi0), ("nonlinear", q, q_phi0)):
        for st in ("f32", "f16", "bf16"):
            for sh, tag in (("ref", ""), ("local", "_local")):
                # one step per launch (plain and vector access), and two
                out[f"{name}_f32_{st}{tag}"] = _time_single(prob, a, "f32", st, steps, warmup, shift=sh)
                out[f"{name}_f32_{st}{tag}_vec"] = _time_single(prob, a, "f32", st, steps, warmup, variant="vec",
                                                               shift=sh)
                out[f"{name}_f32_{st}{tag}_tb2"] = _time_single(prob, a, "f32", st, steps, warmup, variant="tb2",
                                                               shift=sh)
                out[f"{name}_f32_{st}{tag}_tb2v"] = _time_single(prob, a, "f32", st, steps, warmup,
                                                                variant="tb2v", shift=sh)
            out[f"{name}_f32_{st}_tma"] = _time_single(prob, a, "f32", st, steps, warmup, variant="tma")
            # phi as a double-word pair (plain form)
            out[f"{name}_f32_{st}_local_dw"] = _time_single(prob, a, "f32", st, steps, warmup, shift="local_dw")
            if st != "f32":
                # stochastically rounded 16-bit storage: vector form, and with a double-word phi
                out[f"{name}_f32_{st}_local_sr_vec"] = _time_single(prob, a, "f32", st, steps, warmup,
                                                                    variant="vec", shift="local_sr")
                out[f"{name}_f32_{st}_local_dw_sr"] = _time_single(prob, a, "f32", st, steps, warmup,
                                                                   shift="local_dw_sr")
                out[f"{name}_f32_{st}_moment_sr"] = _time_single(prob, a, "f32", st, steps, warmup,
                                                                 shift="moment_sr")
                out[f"{name}_f32_{st}_moment_sr_vec"] = _time_single(prob, a, "f32", st, steps, warmup,
                                                                     variant="vec", shift="moment_sr")
    out["nonlinear_f64"] = _time_single(q, q_phi0, "f64", "f64", 50, 3)
    out.update(run_d3q19(args))
    out.update(run_extended(args))
    return out


def run_extended(args, n=4096, steps=100):
    """The extended coefficient paths at n^2 in the default kernel form (two steps
    per launch for FP32 compute): per-node diffusion tensor and source fields (the
    variable-tensor problem, Eqs. 73-76; 4 field planes read per update), and the
    Burgers-Fisher power-law flux with the reaction source (Eq. 67, periodic copy
    of the problem; products and a square root per node)."""
    import workloads as w
    out = {}
    vt = w.variable_tensor(n=n, alpha=1e-2, walls=True, t_end=0.0)
    vt = vt.replace(dt=20.0 * vt.dx ** 2)
    phi0 = vt.phi0()
    for comp, st in (("f64", "f64"), ("f32", "f32")):
        r = _time_single(vt, phi0, comp, st, steps, 3, variant="auto")
        field_b = 4 * (8 if comp == "f64" else 4)
        gbs = (BYTES_PER_UPDATE[st] + field_b) * r["mlups"] * 1e6 / 1e9
        peak, _ = _peaks()
        r.update(bytes_per_update=BYTES_PER_UPDATE[st] + field_b, algorithmic_gbs=round(gbs, 1),
                 hbm_frac=round(gbs / peak, 4))
        out[f"fields_{n}_{comp}_{st}"] = r
    # Burgers-Fisher coefficients on a periodic square with a smooth periodic field in [0.1, 0.9]
    bf = w.burgers_fisher(n=n, a=2.0, alpha=0.05).replace(
        bc=(0, 0, 0, 0), wall_fn=None,
        phi0_fn=lambda X, Y: 0.5 + 0.4 * np.sin(2 * np.pi * X / 3.0) * np.sin(2 * np.pi * Y / 3.0))
    phi0 = bf.phi0()
    for comp, st in (("f64", "f64"), ("f32", "f32"), ("f32", "f16")):
        out[f"burgers_fisher_{n}_{comp}_{st}"] = _time_single(bf, phi0, comp, st, steps, 3, variant="auto",
                                                             shift="local" if st == "f16" else "ref")
    return out


BYTES_PER_UPDATE_3D = {"f64": 2 * (19 * 8 + 8), "f32": 2 * (19 * 4 + 4), "f16": 2 * (19 * 2 + 4),
                       "bf16": 2 * (19 * 2 + 4)}
N_3D = 384


def _time_single3(p, compute, storage, steps, warmup, shift="auto"):
    import torch
    from paper_1902_09813_gb300 import Lattice3
    stream = torch.cuda.Stream()
    lat = Lattice3.from_problem(p, compute=compute, storage=storage, stream=stream, shift=shift)
    lat.init(p.phi0())
    lat.step(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    lat.check()
    ms = e0.elapsed_time(e1)
    nodes = p.nx * p.ny * p.nz
    mlups = nodes * steps / (ms * 1e-3) / 1e6
    peak, _ = _peaks()
    gbs = BYTES_PER_UPDATE_3D[storage] * mlups * 1e6 / 1e9
    lat.close()
    del lat
    torch.cuda.empty_cache()
    return {"mlups": round(mlups, 1), "ms_per_step": round(ms / steps, 4), "algorithmic_gbs": round(gbs, 1),
            "hbm_frac": round(gbs / peak, 4), "bytes_per_update": BYTES_PER_UPDATE_3D[storage]}


def run_d3q19(args, n=N_3D):
    """The D3Q19 sweep on an n^3 periodic box (advected anisotropic Gaussian hill,
    lattice units): FP64, FP32 storage, FP16 storage with the local shift."""
    import workloads as w
    p = w.gaussian_hill3(n=n, sigma0=n / 16.0, u=(0.05, -0.03, 0.02),
                         A0=(0.02, 0.004, 0.0, 0.015, -0.003, 0.01), nsteps=0)
    return {f"d3q19_{n}_f64": _time_single3(p, "f64", "f64", 30, 3),
            f"d3q19_{n}_f32_f32": _time_single3(p, "f32", "f32", 100, 5),
            f"d3q19_{n}_f32_f16_local": _time_single3(p, "f32", "f16", 100, 5, shift="local")}


# ---------------------------------------------------------------------------- accuracy
def _final_phi(p, phi0, compute, storage, steps, shift="ref"):
    import torch
    from paper_1902_09813_gb300 import Lattice
    lat = Lattice.from_problem(p, compute=compute, storage=storage, shift=shift)
    lat.init(phi0, t0=p.t0).step(steps)
    out = lat.phi_host()
    lat.check()
    del lat
    torch.cuda.empty_cache()
    return out


REDUCED = [("df64", "df64", "ref"), ("f32", "f32", "ref"), ("f32", "f32", "local"), ("f32", "f16", "ref"),
           ("f32", "f16", "local"), ("f32", "bf16", "ref"), ("f32", "bf16", "local"),
           ("f32", "f32", "local_dw"), ("f32", "f16", "local_dw"), ("f32", "bf16", "local_dw"),
           ("f32", "f16", "local_sr"), ("f32", "bf16", "local_sr"), ("f32", "f16", "local_dw_sr"),
           ("f32", "bf16", "local_dw_sr"), ("f32", "f16", "moment_sr"), ("f32", "bf16", "moment_sr")]


def _fmt_key(c, s, sh):
    return c if c in ("f64", "df64") else f"{c}_{s}_{sh}"


# The reduced-precision bar: a format's GRE against the closed form may differ
# from the FP64 sweep's by at most this fraction of it.
GRE_BAR = 0.01
CONV_SIDES = (64, 128, 256, 512, 1024, 2048)


def run_convergence(sides=CONV_SIDES, formats=None):
    """Config-2 convergence sweep under diffusive scaling (dt = 4 dx^2, T_end = 0.1,
    HBB walls, manufactured solution): the GRE against the closed form per grid
    and format, the observed order log2(GRE(N/2) / GRE(N)), each format's GRE
    relative to the FP64 sweep's, and the finest N at which a format stays within
    GRE_BAR of it (all coarser grids too)."""
    import workloads as w
    formats = formats or [("f64", "f64", "ref")] + REDUCED
    out = {"sides": list(sides), "kappa": 4.0, "t_end": 0.1, "bar": GRE_BAR, "formats": {}}
    gre = {}
    t_fmt = {}
    for n in sides:
        p = w.mms_sinsin(n=n)
        phi0 = p.phi0()
        ex = w.mms_sinsin_exact(p, p.t0 + p.nsteps * p.dt)
        for c, s, sh in formats:
            t0 = time.perf_counter()
            g = w.gre(_final_phi(p, phi0, c, s, p.nsteps, sh), ex)
            k = _fmt_key(c, s, sh)
            gre.setdefault(k, []).append(g)
            t_fmt[k] = t_fmt.get(k, 0.0) + time.perf_counter() - t0
    out["steps"] = [int(w.mms_sinsin(n=n).nsteps) for n in sides]
    base = gre["f64"]
    for k, g in gre.items():
        order = [None] + [round(math.log2(g[i - 1] / g[i]), 3) for i in range(1, len(g))]
        rel = [round(g[i] / base[i] - 1.0, 5) for i in range(len(g))]
        finest = None
        for i, r in enumerate(rel):
            if abs(r) > GRE_BAR:
                break
            finest = sides[i]
        out["formats"][k] = {"gre": [float(f"{v:.5e}") for v in g], "order": order,
                             "rel_to_f64": rel, "finest_n_within_bar": finest,
                             "seconds": round(t_fmt[k], 2)}
    return out


def run_accuracy(args):
    """Error of each reduced-precision path: relative L2 against the FP64 sweep on
    the nonlinear 16-mode workload (2048^2 and 8192^2, 1000 steps; the FP64 sweep
    matches the FP64 oracle to 1e-11 in the parity tests, at 8192^2 on sampled
    nodes), the discretisation error (GRE) against the closed forms of the
    Gaussian hill (64^2, 500 steps) and the manufactured solution (128^2) next to
    the FP64 sweep's, and the config-2 convergence sweep (run_convergence)."""
    import workloads as w

    out = {"reference": "FP64 sweep (= FP64 oracle to 1e-11)"}
    for n in (2048, 8192):
        q = w.nonlinear_modes(n=n, nsteps=1000)
        phi0 = q.phi0()
        q.phi_ref = float(phi0.mean())
        ref = _final_phi(q, phi0, "f64", "f64", 1000)
        out[f"nonlinear_{n}_1000_rel_l2"] = {
            _fmt_key(c, s, sh): float(f"{w.rel_l2(_final_phi(q, phi0, c, s, 1000, sh), ref):.3e}")
            for c, s, sh in REDUCED}
        del ref
    closed = {"hill_64": (w.gaussian_hill(), lambda p: w.gaussian_hill_exact(p, p.nsteps * p.dt)),
              "mms_128": (w.mms_sinsin(n=128), lambda p: w.mms_sinsin_exact(p, p.t0 + p.nsteps * p.dt))}
    for name, (p, exact) in closed.items():
        phi0 = p.phi0()
        p.phi_ref = float(phi0.mean())
        ex = exact(p)
        g = {"f64": float(f"{w.gre(_final_phi(p, phi0, 'f64', 'f64', p.nsteps), ex):.4e}")}
        for c, s, sh in REDUCED:
            g[_fmt_key(c, s, sh)] = float(f"{w.gre(_final_phi(p, phi0, c, s, p.nsteps, sh), ex):.4e}")
        out[f"{name}_gre"] = g
    out["mms_convergence"] = run_convergence()
    return out


# ---------------------------------------------------------------------------- batched
def run_batched(args, count=512, nsteps=2000, seed=0, plain=True):
    """Config-4 style batch: `count` instances, side log-uniform in [32, 1024], half
    periodic Gaussian hills / half HBB manufactured solutions, FP32 compute + FP16
    shifted storage, `nsteps` steps each: one batched launch form per call (CUDA
    graph) with an autotuned tile shape (or the one `--batch-tile` names), against
    plain per-instance launches."""
    import torch

    import workloads as w
    from paper_1902_09813_gb300 import Batch, Lattice

    probs = w.batched_instances(count=count, seed=seed, nsteps=nsteps)
    stream = torch.cuda.current_stream()
    phi0s = [p.phi0() for p in probs]
    for p, a in zip(probs, phi0s):
        p.phi_ref = float(a.mean())
    nodes = sum(p.nx * p.ny for p in probs)

    def make():
        lats = []
        for p, a in zip(probs, phi0s):
            lat = Lattice.from_problem(p, compute="f32", storage="f16", stream=stream)
            lat.init(a)
            lats.append(lat)
        return lats

    # batched: autotune on a throw-away copy (its steps are real steps), then time
    shape = tuple(getattr(args, "batch_tile", None) or ())
    if not shape:
        lats = make()
        b = Batch(lats, stream=stream)
        shape = b.autotune(steps_per_trial=3)
        b.close()
        del lats, b
    lats = make()
    b = Batch(lats, stream=stream)
    b.set_tiles(*shape)
    b.step(2)                      # warm-up, not timed
    b.prepare(nsteps - 2, residual=False)   # capture the timed call's graph outside the timed region
    graphs = b.graphs()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    b.step(nsteps - 2)
    ev1.record(stream)
    torch.cuda.synchronize()
    b.check()
    t_batch = ev0.elapsed_time(ev1) * 1e-3 * nsteps / (nsteps - 2)
    batched = [l.phi_host() for l in lats[:8]]
    b.close()
    del lats, b

    if not plain:
        return {"instances": count, "steps": nsteps, "nodes": nodes, "tile": list(shape),
                "batched_s": round(t_batch, 4),
                "batched_mlups": round(nodes * nsteps / t_batch / 1e6, 1)}
    # plain: every instance alone, one launch per step, sequentially
    lats = make()
    torch.cuda.synchronize()
    ev0.record(stream)
    for l in lats:
        l.step(nsteps)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_plain = ev0.elapsed_time(ev1) * 1e-3
    same = all(np.array_equal(a, l.phi_host()) for a, l in zip(batched, lats[:8]))
    del lats
    return {"instances": count, "steps": nsteps, "nodes": nodes, "tile": list(shape),
            "batched_s": round(t_batch, 4), "plain_s": round(t_plain, 4),
            "batched_solves_per_s": round(count / t_batch, 2),
            "plain_solves_per_s": round(count / t_plain, 2),
            "batched_mlups": round(nodes * nsteps / t_batch / 1e6, 1),
            "plain_mlups": round(nodes * nsteps / t_plain / 1e6, 1),
            "speedup": round(t_plain / t_batch, 3),
            "batched_equals_plain_bitwise_first8": same,
            "launch": ("one launch per step" if shape[3] in (1, 3) else "two steps per launch" if shape[3] == 2
                       else "persistent cooperative") + (", CUDA graph" if graphs > 0 else ", direct launches"),
            "dtype": "f32 compute, f16 storage (local shift)"}


# ---------------------------------------------------------------------------- serving
def run_serving(args, rates=(100.0, 500.0, 2000.0), count=96, seed=1):
    """Config-5 style serving: Poisson arrivals of batched-config instances, each
    run to ||phi^{n+1} - phi^n||_2 < 1e-8 (checked every 100 steps) or 20000 steps,
    150 GB admission budget; continuous batching vs sequential plain solves of the
    same requests (the highest-rate trace), with each served phi compared to its
    sequential counterpart.  Per rate: the device's idle share of the run (wall
    time without a slice on the GPU), batch rebuilds, host time admitting and
    rebuilding (with the graph capture; both while queued slices run) and waiting
    for the oldest queued slice, and how many requests stopped at the tolerance or
    the cap."""
    import workloads as w
    from paper_1902_09813_gb300.serve import Server, depth_series, poisson_trace, serve_sequential, summarize

    import torch

    from paper_1902_09813_gb300 import Batch, Lattice

    count = args.serve_count or count
    probs = w.batched_instances(count=count, seed=seed, nsteps=0)
    for p in probs:
        p.phi_ref = float(p.phi0().mean())
    # tile shape of the server's batches: the autotuner on a throw-away batch of all
    # the requests (its trial steps advance only these copies), before any trace runs
    lats = [Lattice.from_problem(p, compute="f32", storage="f16").init(p.phi0(), t0=p.t0) for p in probs]
    b = Batch(lats)
    shape = b.autotune(steps_per_trial=3)
    b.close()
    del lats, b
    torch.cuda.empty_cache()
    out = {"requests_per_rate": count, "slice_steps": 100, "max_steps": 20000, "tol": 1e-8,
           "budget_gb": 150, "dtype": "f32 compute, f16 storage (local shift)", "tile": list(shape),
           "rates": {}}
    served = None
    for lam in rates:
        trace = poisson_trace(probs, rate=lam, seed=seed)
        srv = Server(budget_bytes=150e9, slice_steps=100, max_steps=20000, tol=1e-8, tiles=shape)
        res = srv.run(trace)
        st = srv.stats
        out["rates"][str(int(lam))] = dict(
            summarize(res), peak_active=st["peak_active"], slices=st["slices"], rebuilds=st["rebuilds"],
            gpu_idle_fraction=round(srv.idle_fraction(), 4), gpu_busy_s=round(st["gpu_busy_s"], 3),
            admit_s=round(st["admit_s"], 3), rebuild_s=round(st["rebuild_s"], 3),
            wait_s=round(st["wait_s"], 3), stopped_at_tol=st["tol_hits"], stopped_at_cap=st["cap_hits"], rejected=st["rejected"],
            unstable=st["unstable"], depth_t_active_waiting=depth_series(srv.depth))
        served = res
    # plain sequential baseline on the same requests as the highest-rate trace
    trace = poisson_trace(probs, rate=max(rates), seed=seed)
    seq = serve_sequential(trace, slice_steps=100, max_steps=20000, tol=1e-8)
    out["sequential_plain"] = dict(summarize(seq), requests_same_as_served=True,
                                   stopped_at_tol=sum(1 for r in seq if r.steps < 20000))
    diffs = [float(np.max(np.abs(a.phi - b_.phi)) / max(np.max(np.abs(b_.phi)), 1e-300))
             for a, b_ in zip(served, seq) if a.phi is not None and a.steps == b_.steps]
    out["served_vs_sequential"] = {
        "same_steps": sum(1 for a, b_ in zip(served, seq) if a.steps == b_.steps),
        "bitwise_equal": sum(1 for a, b_ in zip(served, seq)
                             if a.phi is not None and a.steps == b_.steps and np.array_equal(a.phi, b_.phi)),
        "max_rel_diff": float(f"{max(diffs):.3e}") if diffs else None,
        "requests": len(seq)}
    return out


# ---------------------------------------------------------------------------- CPU oracle
def _oracle_sample(n_side: int):
    """A bounded patch of the benchmark workload: same dx, dt, coefficients and walls
    as the 8192^2 lattice, on an n_side x n_side sub-grid."""
    import workloads as w
    p = w.mms_sinsin(n=N_MAIN, nsteps=1)
    return p.replace(nx=n_side, ny=n_side)


def _oracle_rate(n_side: int, threads: int, seconds: float):
    import oracle
    p = _oracle_sample(n_side)
    lat = oracle.OracleLattice(p, nthreads=threads).init()
    lat.step(1)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        lat.step(2)
        steps += 2
    el = time.perf_counter() - t0
    return p, steps, el, p.nx * p.ny * steps / el / 1e6


def cpu_baseline(args, seconds: float = 12.0):
    """The FP64 oracle on the host cores (all of them, OpenMP over rows), plus a
    short single-thread sample."""
    cores = _cores()
    p, steps, el, mlups = _oracle_rate(1024, cores, seconds)
    _, steps1, el1, mlups1 = _oracle_rate(256, 1, 4.0)
    return {"value": round(mlups, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "single_thread_mlups": round(mlups1, 3),
            "sample": f"{p.nx}x{p.ny} patch of the benchmark lattice (same dx, dt, coefficients, "
                      f"walls), {steps} steps, {el:.1f} s, OpenMP over rows; single thread: 256x256 patch, "
                      f"{steps1} steps, {el1:.1f} s"}


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


def run_batched_only(args):
    import torch
    torch.cuda.set_device(0)
    print(json.dumps({"batched": run_batched(args, count=args.batch_count, nsteps=args.batch_steps,
                                             plain=False)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--serve-count", type=int, default=0,
                    help="requests per serving trace (0: the default 96)")
    ap.add_argument("--serving-only", action="store_true", help="only the serving comparison")
    ap.add_argument("--accuracy-only", action="store_true",
                    help="only the accuracy study (reduced formats, closed forms, convergence sweep)")
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched persistent launch (for profiling small batches)")
    ap.add_argument("--d3q19-only", action="store_true",
                    help="only the D3Q19 sweep on an n^3 box (--n, --compute, --storage, --shift, --steps)")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--batch-steps", type=int, default=2000)
    ap.add_argument("--batch-tile", type=lambda v: tuple(int(x) for x in v.split(",")), default=None,
                    help="block_x,block_y,rows,form of the batch instead of the autotuner's pick")
    ap.add_argument("--workload", default="mms", choices=["mms", "nonlinear"])
    ap.add_argument("--n", type=int, default=N_MAIN)
    ap.add_argument("--compute", default="f64", choices=["f64", "df64", "f32"])
    ap.add_argument("--storage", default=None, choices=["f64", "df64", "f32", "f16", "bf16"])
    ap.add_argument("--shift", default="auto",
                    choices=["auto", "ref", "local", "local_dw", "local_sr", "local_dw_sr", "moment_sr"],
                    help="stored form of F32/F16/BF16 populations")
    ap.add_argument("--sweep", default="auto", choices=["auto", "plain", "tma", "tb2", "vec", "tb2v"],
                    help="kernel form of FP32-compute sweeps")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.storage is None:
        args.storage = args.compute
    if args.impl == "reference":
        run_reference(args)
    elif args.accuracy_only:
        import torch
        torch.cuda.set_device(0)
        t0 = time.perf_counter()
        acc = run_accuracy(args)
        print(json.dumps({"accuracy": acc, "seconds": round(time.perf_counter() - t0, 1)}), flush=True)
    elif args.batched_only:
        run_batched_only(args)
    elif args.serving_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"serving": run_serving(args)}), flush=True)
    elif args.d3q19_only:
        import workloads as w
        p = w.gaussian_hill3(n=args.n, sigma0=args.n / 16.0, u=(0.05, -0.03, 0.02),
                             A0=(0.02, 0.004, 0.0, 0.015, -0.003, 0.01), nsteps=0)
        r = _time_single3(p, args.compute, args.storage, args.steps, args.warmup, shift=args.shift)
        print(json.dumps({"d3q19": r, "n": args.n, "compute": args.compute, "storage": args.storage}), flush=True)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
