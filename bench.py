#!/usr/bin/env python3
"""Benchmark of the fused MRT lattice Boltzmann step (MLUPS and HBM roofline).

One bench "step" is one pass of the whole hot path over the cavity: DELTA
fused time steps (pull streaming, moments, porous solve, strain-rate power
law, forced MRT flow and thermal collisions), then the wall Nusselt
reduction and the convergence residual.  The default workload is the
4096 x 4096 cavity of the paper's sweep corner (n = 0.6, Da = 1e-3,
Ra = 1e5, Pr = 6.2, porosity 0.6) with FP32 storage; FP64 and the two
16-bit deviation storages are measured beside it.  The device state
(1 GB in FP32) is far larger than the 129 MB L2, so no flush is needed.

Multi-GPU: independent cavities per rank (weak scaling, no collective on the
data path); value = all ranks' node updates / max-over-ranks time.

``--impl reference`` times the FP64 CPU oracle (the test checker) on the host
cores instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_NODE = {"f64": 240, "f32": 120, "bf16d": 64, "f16d": 64}
CASE = dict(n=0.6, Da=1e-3, Ra=1e5, Pr=6.2, porosity=0.6)
FALLBACK_HBM_GBS = 6800.0
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.txt")


def kernel_source_hash():
    """Hash of the CUDA sources: a traffic figure taken from another build of
    the kernel is reported as null."""
    import glob
    import hashlib
    h = hashlib.sha256()
    for fn in sorted(glob.glob(os.path.join(ROOT, "paper_2011_15073_gb300", "csrc", "*"))):
        with open(fn, "rb") as fh:
            h.update(os.path.basename(fn).encode() + fh.read())
    return h.hexdigest()[:16]


def recorded(key, N=None):
    """A figure from the committed ncu summary ``profiles/traffic.txt``
    (lines: key N value source_hash), or None if absent or taken from other
    CUDA sources.  N=None accepts any grid size."""
    try:
        with open(TRAFFIC_FILE) as fh:
            for line in fh:
                parts = line.split()
                if len(parts) == 4 and not line.startswith("#") and parts[0] == key and \
                        (N is None or int(parts[1]) == N):
                    if parts[3] == kernel_source_hash():
                        return float(parts[2])
    except OSError:
        pass
    return None


def recorded_traffic(prec, N):
    """DRAM bytes per launch of the step kernel at this grid, or None."""
    return recorded(prec, N)


# FP64 pipe of this part: 2 FP64 lanes per SM per cycle (measured in
# profiles/step_kernel_f64_1536.md), 152 SMs.
FP64_LANES_PER_SM, N_SM = 2, 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=4096)
    ap.add_argument("--delta", type=int, default=1000,
                    help="fused time steps per bench step (the convergence-check interval)")
    ap.add_argument("--variant-delta", type=int, default=200)
    ap.add_argument("--prec", default="f32")
    ap.add_argument("--variants", default="f64,bf16d,f16d",
                    help="other storage precisions measured beside the headline ('' for none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        for k in ("hbm_gbs", "hbm_GBps", "hbm"):
            if k in d:
                return float(d[k]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi sampler for the SM clock and throttle reasons (read-only)."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def clk_summary_max(clk):
    try:
        return clk.summary()["sm_max_mhz"]
    except Exception:
        return None


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def time_ours(lbm, torch, N, prec, steps, warmup, delta, stream):
    """Device-resident run: returns (seconds for `steps` bench steps, avg fused
    kernel seconds, kernels launched in the timed region, Nu)."""
    cav = lbm.Cavity(N, N, prec=prec, cuda_stream=stream, **CASE)
    try:
        cav.residual()   # first call stores the snapshot
        for _ in range(warmup):
            cav.step(delta)
            cav.nusselt()
            cav.residual()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        nu = None
        for s in range(steps):
            ev[s][0].record(stream)
            cav.step(delta)
            ev[s][1].record(stream)
            nu = cav.nusselt()[0]
            cav.residual()
        t1.record(stream)
        torch.cuda.synchronize()
        total = t0.elapsed_time(t1) / 1e3
        kern = sum(a.elapsed_time(b) for a, b in ev) / 1e3 / (steps * delta)
        launches = steps * (delta + 1 + 2)
        return total, kern, launches, nu
    finally:
        cav.close()


def time_e2e(lbm, torch, N, prec, steps, warmup, delta, stream):
    """End to end through the C ABI with host buffers: each bench step uploads
    the state from pinned host memory, runs `delta` fused steps and reads the
    hot-wall Nusselt number back."""
    cav = lbm.Cavity(N, N, prec=prec, cuda_stream=stream, **CASE)
    try:
        nbytes = cav.state_bytes()
        host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        cav.get_state(host)
        for _ in range(warmup):
            cav.set_state(host)
            cav.step(delta)
            cav.nusselt()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(steps):
            cav.set_state(host)
            cav.step(delta)
            cav.nusselt()
        dt = time.perf_counter() - t
        return dt, nbytes, 8
    finally:
        cav.close()


def cpu_baseline(N_sample=1024, steps=150):
    """The FP64 oracle as it stands, on all host cores (OpenMP), on a bounded
    sample of the workload: an N_sample^2 cavity with the same parameters."""
    import oracle
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    oracle.build()
    c = oracle.Cavity.from_params(N_sample, N_sample, CASE["n"], CASE["Da"], CASE["Ra"], CASE["Pr"],
                                  porosity=CASE["porosity"])
    c.step(1)
    t = time.perf_counter()
    c.step(steps)
    dt = time.perf_counter() - t
    mlups = N_sample * N_sample * steps / dt / 1e6
    return {"value": mlups, "unit": "MLUPS", "cores": int(os.environ["OMP_NUM_THREADS"]), "kind": "oracle",
            "sample": f"FP64 oracle, {N_sample}x{N_sample} cavity, {steps} steps, same (n, Da, Ra, Pr, porosity)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    steps_each = 10
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    Ns = 1024
    c = oracle.Cavity.from_params(Ns, Ns, CASE["n"], CASE["Da"], CASE["Ra"], CASE["Pr"], porosity=CASE["porosity"])
    for _ in range(args.warmup):
        c.step(steps_each)
    t = time.perf_counter()
    for _ in range(args.steps):
        c.step(steps_each)
    dt = time.perf_counter() - t
    mlups = Ns * Ns * steps_each * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": "fused MRT step MLUPS", "value": mlups, "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"cavity {args.N}x{args.N} (timed on a {Ns}x{Ns} sample), "
                                   f"n={CASE['n']}, Da={CASE['Da']}, Ra={CASE['Ra']}, Pr={CASE['Pr']}, "
                                   f"porosity={CASE['porosity']}",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": int(os.environ["OMP_NUM_THREADS"]),
                             "kind": "oracle",
                             "sample": f"{Ns}x{Ns} cavity, {steps_each} steps per bench step"},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2011_15073_gb300 import lbm
    lbm.lib()
    stream = torch.cuda.Stream()
    N, prec, delta = args.N, args.prec, args.delta

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    barrier()
    with Clocks(local) as clk:
        total, kern, launches, nu = time_ours(lbm, torch, N, prec, args.steps, max(3, args.warmup), delta, stream)
    barrier()
    if world > 1:
        t = torch.tensor([total], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total = float(t.item())
    units = world * N * N * delta * args.steps
    mlups = units / total / 1e6
    peak, peak_src = hbm_peak()
    achieved = BYTES_PER_NODE[prec] * N * N / kern / 1e9
    variants = {}
    for v in [p for p in args.variants.split(",") if p and p != prec]:
        vs, vd = 2, args.variant_delta
        tv, kv, _, nuv = time_ours(lbm, torch, N, v, vs, 1, vd, stream)
        av = BYTES_PER_NODE[v] * N * N / kv / 1e9
        variants[v] = {"MLUPS": N * N * vd * vs / tv / 1e6, "kernel_MLUPS": N * N / kv / 1e6,
                       "fused_steps_per_bench_step": vd,
                       "bytes_per_node": BYTES_PER_NODE[v], "achieved_GBs": av, "frac_of_hbm": av / peak,
                       "nu_hot": nuv}
        if v == "f64":
            ipn = recorded("f64_fp64_inst_per_node")
            clk = clk_summary_max(clk)
            if ipn and clk:
                peak_inst = FP64_LANES_PER_SM * N_SM * clk * 1e6
                ach = N * N / kv * ipn
                variants[v]["roofline"] = {"bound": "alu", "unit": "FP64 inst/s", "achieved": ach,
                                           "peak": peak_inst, "frac": ach / peak_inst,
                                           "fp64_inst_per_node": ipn,
                                           "peak_source": "2 FP64 lanes/SM/cycle x 152 SMs x max SM clock"}
    e2e = None
    if not args.no_e2e:
        es = max(2, args.steps // 2)
        te, hb, db = time_e2e(lbm, torch, N, prec, es, 1, delta, stream)
        e2e = {"value": N * N * delta * es / te / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": hb,
               "d2h_bytes_per_step": db}
    if rank != 0:
        return
    cpu = None if args.no_cpu_baseline else cpu_baseline()
    line = {
        "metric": "fused MRT step MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": prec,
        "data": "synthetic",
        "config": {"workload": f"cavity {N}x{N}, n={CASE['n']}, Da={CASE['Da']}, Ra={CASE['Ra']}, "
                               f"Pr={CASE['Pr']}, porosity={CASE['porosity']}, {prec} storage; "
                               f"bench step = {delta} fused steps + Nu + residual",
                   "grid": [N, N], "fused_steps_per_bench_step": delta,
                   "l2": "state larger than L2 (no flush needed)", "parallelism": f"independent cavity per GPU x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": recorded_traffic(prec, N),
                     "peak_source": peak_src, "kernel": f"step_kernel<{prec}>",
                     "bytes_per_node": BYTES_PER_NODE[prec], "avg_launch_us": kern * 1e6},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "nu_hot": nu,
        "variants": variants,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
