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

BYTES_PER_NODE = {"f64": 240, "f32": 120, "f32d": 120, "bf16d": 64, "f16d": 64, "f16s": 64, "bf16s": 64}
# bytes of the stored lagged tau in those figures (read + write); the
# node-local implicit tau (tau_iters > 0) moves none
STORAGE_NAMES = {"f64": "FP64", "f32": "FP32", "f32d": "FP32 deviation-from-rest", "bf16d": "BF16 deviation",
                 "f16d": "FP16 deviation", "f16s": "FP16 deviation (x2^15, stochastic rounding)",
                 "bf16s": "BF16 deviation (stochastic rounding)"}
TAU_BYTES = {"f64": 16, "f32": 8, "f32d": 8, "bf16d": 8, "f16d": 8, "f16s": 8, "bf16s": 8}
STAGING_NAMES = {1: "registers, two nodes per thread", 3: "registers, four nodes per thread"}


def parse_variant(v):
    """'prec[@aa][@tauK][@reg|@quad]' -> (prec, layout, tau_iters, staging)."""
    parts = v.split("@")
    layout, tau_iters, staging = 0, 0, 0
    for m in parts[1:]:
        if m == "aa":
            layout = 1
        elif m.startswith("tau") and m[3:].isdigit():
            tau_iters = int(m[3:])
        elif m in ("reg", "quad"):
            staging = {"reg": 1, "quad": 3}[m]
        else:
            raise ValueError(f"unknown variant modifier {m!r} in {v!r}")
    return parts[0], layout, tau_iters, staging


def resolved_staging(prec, tau_iters, staging, N):
    """The step-kernel mode the library runs for lbm_opts.staging (0 = auto:
    four nodes per thread for the 16-bit storages on grids of at least
    2048 x 2048, 4096 x 4096 with the implicit tau, else two; the rule of
    lbm_opts.staging)."""
    if staging:
        return staging
    return 3 if prec in ("bf16d", "f16d", "f16s", "bf16s") and N >= (4096 if tau_iters else 2048) else 1


def staging_label(prec, layout, tau_iters, staging, N):
    if layout:
        return "in-place kernels (no staging choice)"
    if prec == "f64":
        return "registers, one node per thread"
    return ("auto: " if staging == 0 else "") + STAGING_NAMES[resolved_staging(prec, tau_iters, staging, N)]


def step_kernel_name(prec, layout, tau_iters, staging, N):
    if layout:
        return "aa_even/aa_odd kernels (alternating)"
    if prec == "f64":
        return "step_kernel"
    return {1: "step2_kernel", 3: "step4_kernel"}[resolved_staging(prec, tau_iters, staging, N)]


def bytes_per_node(prec, tau_iters=0):
    return BYTES_PER_NODE[prec] - (TAU_BYTES[prec] if tau_iters else 0)
CASE = dict(n=0.6, Da=1e-3, Ra=1e5, Pr=6.2, porosity=0.6)
FALLBACK_HBM_GBS = 6800.0
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.txt")
PRECISION_FILE = os.path.join(ROOT, "profiles", "precision_study_512.txt")


# The CUDA sources the recorded figures depend on: the single-context step
# kernels (two- and four-node tiles, FP64), their launchers, lbm_step and its
# step graphs, the Nu and residual reductions.  The batch, adjoint, in-place
# and staged kernels are not among them.
# the files that define the step kernels' arithmetic and which kernel runs
# (host-only files are left out: they do not change a measured figure)
RECORD_SOURCES = ("lbm_device.cuh", "lbm_round.cuh", "lbm_step.cuh", "lbm_kernels.cu")


def kernel_source_hash():
    """Hash of RECORD_SOURCES: a figure taken from another build of those
    kernels is reported as null."""
    import hashlib
    h = hashlib.sha256()
    for fn in sorted(RECORD_SOURCES):
        with open(os.path.join(ROOT, "paper_2011_15073_gb300", "csrc", fn), "rb") as fh:
            h.update(fn.encode() + fh.read())
    return h.hexdigest()[:16]


def recorded(key, N=None, path=None):
    """A figure from a committed measurement summary (default
    ``profiles/traffic.txt``; lines: key N value source_hash), or None if
    absent or taken from other CUDA sources.  N=None accepts any grid size."""
    try:
        with open(path or TRAFFIC_FILE) as fh:
            for line in fh:
                parts = line.split()
                if len(parts) == 4 and not line.startswith("#") and parts[0] == key and \
                        (N is None or int(parts[1]) == N):
                    if parts[3] == kernel_source_hash():
                        return float(parts[2])
    except OSError:
        pass
    return None


def recorded_dnu(storage):
    """Largest |relative Nu difference| to FP64 storage at steady state over
    the precision study's cases (512^2, n = 0.6 and 1.0; mean of the last 20
    samples; for the stochastic storages the largest over four rounding
    streams) for this storage, from ``profiles/precision_study_512.txt``."""
    return recorded(storage, None, PRECISION_FILE)


def recorded_dnu_detail(storage):
    """The per-n spread line of the precision record for this storage (text), or None."""
    try:
        with open(PRECISION_FILE) as fh:
            for line in fh:
                parts = line.split(None, 2)
                if len(parts) == 3 and parts[0] == "detail" and parts[1] == storage:
                    return parts[2].strip()
    except OSError:
        pass
    return None


def recorded_traffic(prec, N):
    """DRAM bytes per launch of the step kernel at this grid, or None."""
    return recorded(prec, N)



def alu_peaks(lbm):
    """Measured FMA throughput of this GPU (lbm_bench_fma_peak): thread-level
    instructions per second for FP64, FP32 and packed FP32x2 FMAs."""
    out = {}
    for kind in ("f64", "f32", "f32x2"):
        fma, inst = lbm.bench_fma_peak(kind, reps=20)
        out[kind] = {"fma_per_s": fma, "inst_per_s": inst, "flop_per_s": 2 * fma}
    return out


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
    ap.add_argument("--prec", default="f32d",
                    help="storage of the headline run (f32d: FP32 deviations from the rest state)")
    ap.add_argument("--layout", type=int, default=0, choices=[0, 1],
                    help="0: two buffers (pull); 1: one buffer, in-place AA-pattern streaming")
    ap.add_argument("--staging", type=int, default=0, choices=[0, 1, 3],
                    help="step-kernel inputs: 0 auto, 1 straight to registers (two nodes per thread), "
                         "3 straight to registers (four nodes per thread)")
    ap.add_argument("--tau-iters", type=int, default=0,
                    help="0: lagged tau (stored per node); K > 0: node-local implicit tau, K Newton steps")
    ap.add_argument("--variants", default=DEFAULT_VARIANTS,
                    help="other storage precisions measured beside the headline ('' for none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--study", choices=["tables", "precision", "batch", "adjoint", "plain", "throughput", "grid",
                                        "sensitivity"],
                    default=None,
                    help="physics studies instead of the throughput bench (one JSON line per case)")
    ap.add_argument("--study-N", type=int, default=None)
    ap.add_argument("--study-max-steps", type=int, default=3_000_000)
    ap.add_argument("--study-prec", default="f32d", help="storage of --study sensitivity")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="weak: an independent cavity per rank; strong: one cavity in row slabs over the ranks")
    ap.add_argument("--sr-runs", type=int, default=4,
                    help="rounding streams per stochastic-rounding storage in --study precision")
    ap.add_argument("--study-ref", default=None,
                    help="--study precision: take the FP64 reference from this earlier output (same N)")
    ap.add_argument("--h-sweep", type=lambda t: [float(x) for x in t.split(",") if x], default=[],
                    help="comma-separated difference steps (log Da) for --study adjoint's single-node sweep")
    ap.add_argument("--readings", default="", help="';'-separated labels of --study sensitivity (all if empty)")
    return ap.parse_args()


# Average Nusselt numbers the paper prints (Table 1: clear fluid, Ra = 1e5,
# Pr = 100; Table 2: 160 x 160 grid, Pr = 6.2).
PAPER_TABLES = [
    ("table1", dict(n=0.6, Da=None, Ra=1e5, Pr=100.0), 12.95289),
    ("table1", dict(n=1.0, Da=None, Ra=1e5, Pr=100.0), 4.69148),
    ("table1", dict(n=1.4, Da=None, Ra=1e5, Pr=100.0), 2.44821),
    ("case1", dict(n=0.6, Da=1e-3, Ra=1e5, Pr=6.2), 9.249539),
    ("case1", dict(n=1.0, Da=1e-3, Ra=1e5, Pr=6.2), 2.430419),
    ("case1", dict(n=1.4, Da=1e-3, Ra=1e5, Pr=6.2), 1.300101),
    ("case2", dict(n=0.6, Da=1e-2, Ra=1e5, Pr=6.2), 12.835687),
    ("case2", dict(n=0.6, Da=1e-1, Ra=1e5, Pr=6.2), 13.316177),
    ("case3", dict(n=0.6, Da=1e-2, Ra=1e3, Pr=6.2), 1.068697),
    ("case3", dict(n=0.6, Da=1e-2, Ra=1e4, Pr=6.2), 4.411946),
]


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


def reduced_storage_summary(variants, prec, mlups):
    """The fastest reduced-storage form (fewer bytes per node than FP64)
    whose recorded steady-state |dNu|/Nu is at most 1e-3, against FP64
    storage measured in the same run."""
    f64 = variants.get("f64")
    if not f64:
        return None
    cands = [(v["MLUPS"], k, v.get("dnu_rel_vs_f64_512")) for k, v in variants.items()
             if k != "f64" and v.get("dnu_rel_vs_f64_512") is not None and v["dnu_rel_vs_f64_512"] <= 1e-3]
    main_dnu = recorded_dnu(prec)
    if main_dnu is not None and main_dnu <= 1e-3:
        cands.append((mlups, prec, main_dnu))
    if not cands:
        return None
    best = max(cands)
    return {"variant": best[1], "MLUPS": best[0], "dnu_rel_vs_f64": best[2],
            "dnu_detail": recorded_dnu_detail(best[1]), "dnu_grid": [512, 512],
            "speedup_vs_f64_storage": best[0] / f64["MLUPS"], "f64_MLUPS": f64["MLUPS"],
            "dnu_source": "recorded: bench.py --study precision --study-N 512 (512^2 steady state, n = 0.6 and 1.0, "
                          "max over 4 rounding streams of the 20-sample mean), against FP64 storage on the GPU, "
                          "whose steps equal the FP64 CPU oracle's to 1e-12 (parity tests)"}


def max_over_ranks(value, world, device):
    """The largest value over the ranks (the slowest rank's time): one
    all-reduce of a scalar, nothing on the data path."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_units(world, N, delta, steps):
    """Node updates of the whole job: every rank runs its own N x N cavity
    for steps x delta time steps (weak scaling)."""
    return world * N * N * delta * steps


def time_ours(lbm, torch, N, prec, steps, warmup, delta, stream, layout=0, tau_iters=0, staging=0, graph_steps=0):
    """Device-resident run: returns (seconds for `steps` bench steps, avg fused
    kernel seconds, kernels launched in the timed region, Nu)."""
    cav = lbm.Cavity(N, N, prec=prec, cuda_stream=stream, layout=layout, tau_iters=tau_iters, staging=staging,
                     graph_steps=graph_steps, **CASE)
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
            "sample": f"FP64 oracle, {N_sample}x{N_sample} cavity, {steps} steps, same (n, Da, Ra, Pr, porosity)",
            "single_thread": oracle_single_thread(), "cpu_model": cpu_model()}


def cpu_model():
    """The host CPU's model string (x86 'model name', or the Arm implementer
    and part numbers), for the CPU baseline's record."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return None
    for key in ("model name", "Model"):
        for ln in info:
            if ln.startswith(key):
                return ln.split(":", 1)[1].strip()
    parts = sorted({ln.split(":", 1)[1].strip() for ln in info if ln.startswith(("CPU implementer", "CPU part"))})
    return "arm " + " ".join(parts) if parts else None


def oracle_single_thread(N=64, steps=2000):
    """The oracle on one host core (a child process with OMP_NUM_THREADS=1),
    on an N^2 cavity of the same parameters."""
    import subprocess
    code = ("import time, oracle; oracle.build(); "
            f"c = oracle.Cavity.from_params({N}, {N}, {CASE['n']}, {CASE['Da']}, {CASE['Ra']}, {CASE['Pr']}, "
            f"porosity={CASE['porosity']}); c.step(1); t = time.perf_counter(); c.step({steps}); "
            "print(time.perf_counter() - t)")
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    if r.returncode != 0:
        return None
    dt = float(r.stdout.strip().splitlines()[-1])
    return {"value": N * N * steps / dt / 1e6, "unit": "MLUPS", "cores": 1,
            "sample": f"FP64 oracle, {N}x{N} cavity, {steps} steps"}


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


def run_until_nu_settles(cav, max_steps, chunk=20000, window=6, rel=1e-6):
    """Advance until the residual falls below 1e-10 or the hot-wall Nu of the
    last `window` chunks spreads by less than `rel` (the literal power law can
    leave a small limit cycle at nodes sitting on the gamma_1 jump, so the
    residual need not vanish), or until max_steps."""
    cav.residual()
    hist, done = [], 0
    while done < max_steps:
        cav.step(chunk)
        done += chunk
        r = cav.residual()
        nu = cav.nusselt()[0]
        hist.append(nu)
        if r < 1e-10:
            return done, r, "tol"
        last = hist[-window:]
        if len(last) == window and (max(last) - min(last)) <= rel * abs(last[-1]):
            return done, r, "nu_settled"
    return done, r, "max_steps"


def study_tables(args):
    """The paper's cases (Tables 1 and 2) with its own Darcy model (porosity
    1, no Forchheimer term) and its literal modified power law on its
    160 x 160 grid, run as one batch (the clear-fluid cases of Table 1 as
    Da = 1e12, so that the drag vanishes) until every case's Nu has settled;
    FP64 storage unless --study-prec names another."""
    N = args.study_N or 160
    prec = args.study_prec if args.study_prec != "f32d" else "f64"
    t = time.perf_counter()
    res = batched_tables([c for _, c, _ in PAPER_TABLES], N, dict(prec=prec, Ma=0.1, clamp_mode=0),
                         args.study_max_steps, rel=1e-6 if prec == "f64" else 2e-5)
    secs = time.perf_counter() - t
    for (table, c, nu_paper), (m, spread, steps) in zip(PAPER_TABLES, res):
        print(json.dumps({"study": "tables", "table": table, "N": N, "prec": prec, **c,
                          "nu_hot_mean": m, "spread": spread, "nu_paper": nu_paper,
                          "rel_diff": (m - nu_paper) / nu_paper, "steps": steps, "batch_seconds": secs}),
              flush=True)


def batched_tables(cases, N, opts, max_steps, chunk=20000, window=6, rel=2e-5):
    """Run table cases as one batch (each a cavity of N x N nodes with the
    paper's Darcy model; clear fluid as Da = 1e12) in chunks of `chunk` steps
    until the hot-wall Nu of every case spreads by at most `rel` over the last
    `window` chunks, or max_steps.  Returns per case (mean Nu over the window,
    relative spread, steps); the mean is the time average of a limit cycle."""
    import numpy as np

    from paper_2011_15073_gb300 import lbm
    cl = [dict(nx=N, ny=N, n=c["n"], Da=c["Da"] if c["Da"] is not None else 1e12, Ra=c["Ra"], Pr=c["Pr"],
               porosity=1.0) for c in cases]
    hist = [[] for _ in cl]
    done = 0
    with lbm.Batch(cl, porous_model=0, **opts) as b:
        while done < max_steps:
            b.step(chunk)
            done += chunk
            hot, _ = b.nusselt()
            if not np.all(np.isfinite(hot)):
                raise RuntimeError("non-finite Nu in the table batch")
            for h, v in zip(hist, hot):
                h.append(float(v))
            if all(len(h) >= window and max(h[-window:]) - min(h[-window:]) <= rel * abs(h[-1]) for h in hist):
                break
    out = []
    for h in hist:
        w = h[-window:]
        m = sum(w) / len(w)
        out.append((m, (max(w) - min(w)) / abs(m), done))
    return out


# Extra cases beside the paper's: the clear fluid at the porous cases' Pr, and
# the most permeable porous case at Table 1's Pr (do Pr and drag separate?).
SENSITIVITY_EXTRA = [
    ("diag", dict(n=0.6, Da=None, Ra=1e5, Pr=6.2), None),
    ("diag", dict(n=0.6, Da=1e-1, Ra=1e5, Pr=100.0), None),
]
SENSITIVITY_READINGS = [
    # (label, options, N, Ma)
    ("literal clamp, lagged tau", dict(clamp_mode=0), 160, 0.1),
    ("continuous clamp, lagged tau", dict(clamp_mode=1), 160, 0.1),
    ("literal clamp, implicit tau", dict(clamp_mode=0, tau_iters=2), 160, 0.1),
    ("literal clamp, Ma 0.05", dict(clamp_mode=0), 160, 0.05),
    ("continuous clamp, Ma 0.05", dict(clamp_mode=1), 160, 0.05),
    ("literal clamp, 256^2", dict(clamp_mode=0), 256, 0.1),
    ("continuous clamp, 256^2", dict(clamp_mode=1), 256, 0.1),
]


def study_sensitivity(args):
    """Which reading of the unstated parts moves the paper's table values:
    the clamp of Eq. (MPL) (literal jump at gamma_1 or continuous), the
    lagged or node-local implicit tau, the Mach number of the velocity scale,
    and the grid.  FP32-deviation storage (its steady states are within 1e-4
    of FP64's), the paper's Darcy model, the batched API, one batch per
    reading."""
    cases = PAPER_TABLES + SENSITIVITY_EXTRA
    sel = [r for r in SENSITIVITY_READINGS if not args.readings or r[0] in args.readings.split(";")]
    for label, opts, N, Ma in sel:
        N = args.study_N or N
        max_steps = int(args.study_max_steps * (0.1 / Ma) * (N / 160))
        t = time.perf_counter()
        res = batched_tables([c for _, c, _ in cases], N, dict(prec=args.study_prec, Ma=Ma, **opts), max_steps)
        secs = time.perf_counter() - t
        for (table, c, nu_paper), (m, spread, steps) in zip(cases, res):
            print(json.dumps({"study": "sensitivity", "reading": label, "N": N, "Ma": Ma, **opts,
                              "prec": args.study_prec, "table": table, **c, "nu_hot_mean": m,
                              "spread": spread, "nu_paper": nu_paper,
                              "rel_diff": None if nu_paper is None else (m - nu_paper) / nu_paper,
                              "steps": steps, "batch_seconds": secs}), flush=True)


def study_grid(args):
    """Grid independence of the average hot-wall Nu at 128^2, 160^2 and
    192^2 (the paper reports choosing 160^2 without showing the study): three
    of its cases (Table 1 n = 1; Table 2 Case 1 n = 1.0 and 1.4), its Darcy
    model and literal law, FP64, each run until Nu settles."""
    from paper_2011_15073_gb300 import lbm
    cases = [PAPER_TABLES[1], PAPER_TABLES[4], PAPER_TABLES[5]]
    for table, c, nu_paper in cases:
        nus = {}
        for N in (128, 160, 192):
            Da = c["Da"] if c["Da"] is not None else 1e12
            with lbm.Cavity(N, N, c["n"], Da, c["Ra"], c["Pr"], 1.0, prec="f64", porous_model=0) as cav:
                steps, resid, why = run_until_nu_settles(cav, args.study_max_steps)
                nus[N] = cav.nusselt()[0]
        d1, d2 = nus[160] - nus[128], nus[192] - nus[160]
        print(json.dumps({"study": "grid", "table": table, **c, "nu_hot": nus, "nu_paper_160": nu_paper,
                          "rel_change_128_160": d1 / nus[160], "rel_change_160_192": d2 / nus[192],
                          "rel_diff_160_vs_paper": (nus[160] - nu_paper) / nu_paper}), flush=True)


DEFAULT_VARIANTS = "f64,f32,f32d@aa,f32d@tau2,bf16d,f16d,f16s,f16s@reg,bf16s,f16s@tau2"
PRECISION_VARIANTS = ("f64", "f64@tau4", "f32", "f32@tau2", "f32d", "f16d", "bf16d", "f16s", "bf16s")


def recorded_fp64_reference(path, N):
    """The FP64 rows of an earlier --study precision output at grid N, by
    power-law index n (JSON lines; other lines of the file are skipped)."""
    out = {}
    with open(path) as fh:
        for line in fh:
            d = json.loads(line) if line.startswith("{") else {}
            if d.get("study") == "precision" and d.get("variant") == "f64" and d.get("N") == N:
                out[d["n"]] = d
    return out


def study_precision(args):
    """Storage formats and tau schemes against FP64 storage (lagged tau) at
    the FP64 steady state: the FP64 run goes to a residual of 1e-10 in S steps
    (continuous power law, so the steady state is unique); every other
    variant then runs the same S steps from the same rest state, sampling the
    hot-wall Nu every 1000 steps over the last 20,000 (stochastic rounding
    leaves a noise of its own on any one snapshot).  Reported: the relative
    L2 errors of u_x, u_y, T at the end, the relative Nu difference at the end
    and of the mean of the samples.  --study-ref FILE takes the FP64 run (its
    Nu and step count) from an earlier run's output at the same N instead of
    repeating it; the field errors are then not reported."""
    import numpy as np
    from paper_2011_15073_gb300 import lbm
    N = args.study_N or 512
    variants = [v for v in (args.variants.split(",") if args.variants != DEFAULT_VARIANTS else PRECISION_VARIANTS)
                if v]
    recorded_ref = recorded_fp64_reference(args.study_ref, N) if args.study_ref else {}
    for n in (0.6, 1.0):
        case = dict(n=n, Da=1e-2, Ra=1e5, Pr=6.2, porosity=0.6)
        res = {}
        S = None
        # the stochastic-rounding storages run once per rounding stream
        # (lbm_opts.seed), labelled variant#seed beyond the default stream
        runs = []
        for v in ["f64"] + [x for x in variants if x != "f64"]:
            runs.append(v)
            if parse_variant(v)[0] in ("f16s", "bf16s"):
                runs += [f"{v}#{s}" for s in range(1, args.sr_runs)]
        for v in runs:
            if v == "f64" and n in recorded_ref:
                d = recorded_ref[n]
                S = d["steps"]
                res[v] = dict(nu=d["nu_hot"], nu_cold=d["nu_cold"], nu_mean=d["nu_hot"], nu_std=0.0, fl=None,
                              steps=S, resid=d["residual"], stop="recorded", sec=0.0)
                continue
            prec, layout, tau_iters, staging = parse_variant(v.split("#")[0])
            seed = int(v.split("#")[1]) if "#" in v else 0
            t = time.perf_counter()
            with lbm.Cavity(N, N, prec=prec, resid_interval=1000, clamp_mode=1, layout=layout, tau_iters=tau_iters,
                            staging=staging, seed=seed, **case) as cav:
                samples = []
                if v == "f64":
                    S, resid, why = cav.run_to_steady(1e-10, args.study_max_steps)
                    stop = ["tol", "stagnated", "max_steps"][why]
                    samples.append(cav.nusselt()[0])
                else:
                    tail = min(20, S // 1000 - 1)
                    cav.step(S - 1000 * tail)
                    cav.residual()
                    for _ in range(tail):
                        cav.step(1000)
                        samples.append(cav.nusselt()[0])
                    resid, stop = cav.residual(), "same_steps"
                hot, cold, _ = cav.nusselt()
                fl = cav.fields()
            res[v] = dict(nu=hot, nu_cold=cold, nu_mean=float(np.mean(samples)), nu_std=float(np.std(samples)),
                          fl=fl, steps=S, resid=resid, stop=stop, sec=time.perf_counter() - t)
        ref = res["f64"]
        for v, r in res.items():
            err = None if r["fl"] is None or ref["fl"] is None else {
                k: float(np.linalg.norm(r["fl"][k] - ref["fl"][k]) / np.linalg.norm(ref["fl"][k]))
                for k in ("ux", "uy", "T")}
            print(json.dumps({"study": "precision", "N": N, **case, "clamp_mode": 1, "variant": v,
                              "nu_hot": r["nu"], "nu_cold": r["nu_cold"], "nu_hot_mean": r["nu_mean"],
                              "nu_hot_std": r["nu_std"],
                              "dnu_rel": (r["nu"] - ref["nu"]) / ref["nu"],
                              "dnu_mean_rel": (r["nu_mean"] - ref["nu"]) / ref["nu"], "l2_rel": err,
                              "steps": r["steps"], "residual": r["resid"], "stop": r["stop"],
                              "seconds": r["sec"]}), flush=True)
        for v in variants:
            reps = [r for k, r in res.items() if k.split("#")[0] == v]
            if len(reps) > 1:
                d = [(r["nu_mean"] - ref["nu"]) / ref["nu"] for r in reps]
                print(json.dumps({"study": "precision", "N": N, **case, "clamp_mode": 1, "variant": v,
                                  "streams": len(reps), "dnu_mean_rel_per_stream": d,
                                  "dnu_mean_rel_mean": float(np.mean(d)), "dnu_mean_rel_spread": float(np.std(d)),
                                  "dnu_mean_rel_max_abs": float(np.max(np.abs(d)))}), flush=True)


def study_plain(args):
    """The plain method in FP64 on a 64^2 cavity (n = 1, Da = 0.1, Ra = 1e3,
    porosity 0.6; Pr = 10 and 6.2): average hot-wall Nu after 20,000 steps,
    on the GPU and from the FP64 oracle, and at convergence (r < 1e-10)."""
    import oracle
    from paper_2011_15073_gb300 import lbm
    oracle.build()
    for Pr in (10.0, 6.2):
        case = dict(n=1.0, Da=1e-1, Ra=1e3, Pr=Pr, porosity=0.6)
        ref = oracle.Cavity.from_params(64, 64, case["n"], case["Da"], case["Ra"], Pr, porosity=0.6)
        t = time.perf_counter()
        ref.step(20_000)
        t_orc = time.perf_counter() - t
        nu_orc = ref.nusselt()[0]
        with lbm.Cavity(64, 64, prec="f64", **case) as cav:
            cav.step(20_000)
            nu_20k = cav.nusselt()[0]
            steps, r, why = cav.run_to_steady(1e-10, 2_000_000)
            nu_ss = cav.nusselt()[0]
        print(json.dumps({"study": "plain", "N": 64, **case, "prec": "f64", "nu_hot_20000": nu_20k,
                          "oracle_nu_hot_20000": nu_orc, "rel_diff_vs_oracle": (nu_20k - nu_orc) / nu_orc,
                          "oracle_seconds": t_orc, "steady_steps": 20_000 + steps, "steady_residual": r,
                          "nu_hot_steady": nu_ss}), flush=True)


def study_throughput(args):
    """Single cases at 1024^2 and 4096^2 (n = 0.6, Da = 1e-3, Ra = 1e5):
    200 warm-up steps, then five timed runs of 2000 steps each (CUDA events
    on the library's stream); best and median MLUPS per storage."""
    import statistics
    import torch
    from paper_2011_15073_gb300 import lbm
    stream = torch.cuda.Stream()
    for N in (1024, 4096):
        for prec in ("f64", "f32", "f32d"):
            with lbm.Cavity(N, N, prec=prec, cuda_stream=stream, **CASE) as cav:
                cav.step(200)
                rates = []
                for _ in range(5):
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    cav.step(2000)
                    b.record(stream)
                    b.synchronize()
                    rates.append(N * N * 2000 / (a.elapsed_time(b) / 1e3) / 1e6)
            print(json.dumps({"study": "throughput", "N": N, "prec": prec, "best_MLUPS": max(rates),
                              "median_MLUPS": statistics.median(rates),
                              "GBs_at_median": statistics.median(rates) * 1e6 * BYTES_PER_NODE[prec] / 1e9}),
                  flush=True)


def study_batch(args):
    """The paper's kind of sweep (27 cases, n x Da x Ra, grids 128^2-512^2 drawn
    by seed) run to steady state as one batched workload -- one CUDA graph
    launch looping on the device, execution plan from the autotuner --
    against the same cases run one after another with lbm_run_to_steady.
    FP32 storage cannot bring the residual to 1e-8 (its rounding floor is
    near 1e-5), so a case also retires on stagnation: no new minimum over 10
    checks while below 1e-4.  Reported per case: steps, final residual, stop
    rule, Nu, the Nu drift over 10,000 further steps of the retired state,
    and for the three smallest cases the hot-wall Nu of an FP64 run to
    r < 1e-8."""
    from paper_2011_15073_gb300 import inputs, lbm
    max_steps = args.study_max_steps if args.study_max_steps != 3_000_000 else 1_000_000
    cl = [dict(nx=c["N"], ny=c["N"], n=c["n"], Da=c["Da"], Ra=c["Ra"], Pr=6.2, porosity=0.6)
          for c in inputs.sweep_cases(2011)]
    floor = 1e-4
    opts = dict(prec="f32", clamp_mode=1, resid_interval=1000, stag_floor=floor)
    with lbm.Batch(cl, **opts) as b:
        t = time.perf_counter()
        threads = b.tune(200)
        t_tune = time.perf_counter() - t
        plan = b.plan()
        t = time.perf_counter()
        steps, res, why = b.run_to_steady(1e-8, max_steps, graph_mode=1)
        t_batch = time.perf_counter() - t
        hot, _ = b.nusselt()
        b.step(10_000)
        hot_later, _ = b.nusselt()
    t = time.perf_counter()
    seq = []
    for c in cl:
        with lbm.Cavity(c["nx"], c["ny"], c["n"], c["Da"], c["Ra"], c["Pr"], c["porosity"], **opts) as cav:
            s_, r, w = cav.run_to_steady(1e-8, max_steps)
            seq.append((s_, r, w, cav.nusselt()[0]))
    t_seq = time.perf_counter() - t
    # FP64 reference of the smallest grids, to r < 1e-8
    small = sorted(range(len(cl)), key=lambda i: (cl[i]["nx"], i))[:3]
    f64 = {}
    for i in small:
        c = cl[i]
        with lbm.Cavity(c["nx"], c["ny"], c["n"], c["Da"], c["Ra"], c["Pr"], c["porosity"], prec="f64",
                        clamp_mode=1, resid_interval=1000) as cav:
            s_, r, w = cav.run_to_steady(1e-8, 3_000_000)
            f64[i] = dict(steps=s_, resid=r, stop=["tol", "stagnated", "max_steps"][w], nu=cav.nusselt()[0])
    updates = sum(c["nx"] * c["ny"] * s_ for c, s_ in zip(cl, steps))
    print(json.dumps({
        "study": "batch", "cases": len(cl), "prec": "f32", "tol": 1e-8, "max_steps": max_steps,
        "stop_rule": f"r < 1e-8, or no new minimum over 10 checks while r < {floor}, or {max_steps} steps",
        "tol_met": sum(1 for w in why if w == 0),
        "tuned_plan": plan, "tuned_threads": threads, "tune_seconds": t_tune,
        "batched": {"seconds": t_batch, "cases_per_s": len(cl) / t_batch, "MLUPS": updates / t_batch / 1e6,
                    "graph_launches": 1},
        "sequential": {"seconds": t_seq, "cases_per_s": len(cl) / t_seq,
                       "MLUPS": sum(c["nx"] * c["ny"] * q[0] for c, q in zip(cl, seq)) / t_seq / 1e6},
        "speedup": t_seq / t_batch,
        "same_steps": all(s_ == q[0] for s_, q in zip(steps, seq)),
        "max_rel_nu_diff": max(abs(h - q[3]) / abs(q[3]) for h, q in zip(hot, seq)),
        "stop_reasons": {k: sum(1 for w in why if w == k) for k in (0, 1, 2, 3)},
        "max_rel_nu_drift_10k": max(abs(a - h) / abs(h) for a, h in zip(hot_later, hot)),
        "fp64_r1e-8": [dict(case=i, N=cl[i]["nx"], n=cl[i]["n"], Da=cl[i]["Da"], Ra=cl[i]["Ra"],
                            nu_f32_retired=float(hot[i]), **f64[i],
                            rel_diff=(float(hot[i]) - f64[i]["nu"]) / f64[i]["nu"]) for i in small],
        "per_case": [dict(N=c["nx"], n=c["n"], Da=c["Da"], Ra=c["Ra"], steps=s_, resid=float(r), stop=w,
                          nu=float(h), rel_nu_drift_10k=float(abs(a - h) / abs(h)))
                     for c, s_, r, w, h, a in zip(cl, steps, res, why, hot, hot_later)],
    }), flush=True)


def study_adjoint(args):
    """Gradient of the hot-wall Nusselt number after 10,000 FP32 steps of a
    256^2 cavity (n = 0.8, Ra = 1e4, Pr = 6.2, porosity 0.6) with a per-node
    Darcy field log-uniform in [1e-3, 1e-1] (seed 2011), by the discrete
    adjoint with checkpoints every 500 steps; checked against FP64 central
    differences (h = 1e-4 in log Da) on 16 random nodes and one random
    direction, and against the FP64 adjoint.  The continuous clamp of the
    power law is used: the literal law jumps at gamma_1, so J is not
    differentiable and a difference quotient across a jump is meaningless."""
    import numpy as np
    from paper_2011_15073_gb300 import inputs, lbm
    N = args.study_N or 256
    steps, ckpt = 10_000, 500
    case = dict(n=0.8, Ra=1e4, Pr=6.2, porosity=0.6)
    Da = inputs.darcy_field(2011, N, N)

    def cav(prec):
        c = lbm.Cavity(N, N, case["n"], 1e-2, case["Ra"], case["Pr"], case["porosity"], prec=prec, clamp_mode=1)
        c.set_darcy_field(Da)
        return c

    res = {}
    for prec in ("f32", "f64"):
        with cav(prec) as c:       # forward alone, same steps
            c.step(10)
            c.synchronize()
            t = time.perf_counter()
            c.step(steps)
            c.synchronize()
            t_fwd = time.perf_counter() - t
        with cav(prec) as c:
            t = time.perf_counter()
            J, dDa, dn, dRa, peak = c.adjoint_nu(steps, ckpt, from_rest=True)
            t_adj = time.perf_counter() - t
        res[prec] = dict(J=J, dDa=dDa, dn=dn, dRa=dRa, peak=peak, t_fwd=t_fwd, t_adj=t_adj)

    def J_of(D):
        with lbm.Cavity(N, N, case["n"], 1e-2, case["Ra"], case["Pr"], case["porosity"], prec="f64",
                        clamp_mode=1) as c:
            c.set_darcy_field(D)
            c.step(steps)
            return c.nusselt()[0]

    h = 1e-4
    rng = np.random.default_rng(2011)
    nodes = [(int(rng.integers(0, N)), int(rng.integers(0, N))) for _ in range(16)]
    fd_rel = []
    for (j, i) in nodes:
        Dp, Dm = Da.copy(), Da.copy()
        Dp[j, i] *= np.exp(h)
        Dm[j, i] *= np.exp(-h)
        fd = (J_of(Dp) - J_of(Dm)) / (2 * h)
        for prec in ("f64", "f32"):
            ad = res[prec]["dDa"][j, i] * Da[j, i]
            fd_rel.append(dict(node=[j, i], prec=prec, fd=fd, adjoint=ad,
                               rel=abs(ad - fd) / max(abs(fd), 1e-300)))
    # step sweep of the single-node differences: truncation shrinks with h^2,
    # the rounding of J (FP64, 10,000 steps) grows with 1/h
    sweep = {}
    for hs in args.h_sweep:
        rel64, rel32 = [], []
        for (j, i) in nodes:
            Dp, Dm = Da.copy(), Da.copy()
            Dp[j, i] *= np.exp(hs)
            Dm[j, i] *= np.exp(-hs)
            fd = (J_of(Dp) - J_of(Dm)) / (2 * hs)
            for prec, out in (("f64", rel64), ("f32", rel32)):
                ad = res[prec]["dDa"][j, i] * Da[j, i]
                out.append(abs(ad - fd) / max(abs(fd), 1e-300))
        sweep[repr(hs)] = {"max_rel_f64": max(rel64), "median_rel_f64": float(np.median(rel64)),
                           "max_rel_f32": max(rel32), "median_rel_f32": float(np.median(rel32)),
                           "rel_f64_per_node": rel64}
    v = rng.standard_normal((N, N))
    fd_dir = (J_of(Da * np.exp(h * v)) - J_of(Da * np.exp(-h * v))) / (2 * h)
    dir_ad = {p_: float(np.sum(res[p_]["dDa"] * Da * v)) for p_ in ("f64", "f32")}
    f32, f64 = res["f32"], res["f64"]
    print(json.dumps({
        "study": "adjoint", "N": N, "steps": steps, "ckpt_every": ckpt, **case,
        "J": {"f32": f32["J"], "f64": f64["J"]},
        "dJ_dn": {"f32": f32["dn"], "f64": f64["dn"]}, "dJ_dRa": {"f32": f32["dRa"], "f64": f64["dRa"]},
        "time_forward_s": {"f32": f32["t_fwd"], "f64": f64["t_fwd"]},
        "time_adjoint_s": {"f32": f32["t_adj"], "f64": f64["t_adj"]},
        "adjoint_over_forward": {"f32": f32["t_adj"] / f32["t_fwd"], "f64": f64["t_adj"] / f64["t_fwd"]},
        "peak_device_bytes": {"f32": f32["peak"], "f64": f64["peak"]},
        "fd_nodes_max_rel": {p_: max(r["rel"] for r in fd_rel if r["prec"] == p_) for p_ in ("f64", "f32")},
        "fd_direction": {"fd": fd_dir, "adjoint_f64": dir_ad["f64"], "adjoint_f32": dir_ad["f32"],
                         "rel_f64": abs(dir_ad["f64"] - fd_dir) / abs(fd_dir),
                         "rel_f32": abs(dir_ad["f32"] - fd_dir) / abs(fd_dir)},
        "f32_vs_f64_dDa_rel_l2": float(np.linalg.norm(f32["dDa"] - f64["dDa"]) / np.linalg.norm(f64["dDa"])),
        "fd_nodes": fd_rel,
        "fd_nodes_h_sweep": sweep,
    }), flush=True)


def run_strong(args, torch, lbm, rank, world, local):
    """Strong scaling: ONE N x N cavity split into row slabs over the ranks
    (paper_2011_15073_gb300.slabs.DistributedSlab): every fused step is
    followed by the halo exchange with the ranks above and below (NCCL
    send/recv of 4 x N values per cut each way), the Nusselt number and the
    residual by an all-reduce of their sums.  A bench step is `delta` fused
    steps + Nu + residual; value = N^2 x delta x steps / max-over-ranks time."""
    import socket

    import torch.distributed as dist
    from paper_2011_15073_gb300 import slabs
    N, prec, delta = args.N, args.prec, args.delta
    own_group = not dist.is_initialized()
    if own_group:   # one rank: a group of one, so the same slab path runs
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    slab = slabs.DistributedSlab(N, N, CASE["n"], CASE["Da"], CASE["Ra"], CASE["Pr"], CASE["porosity"], prec=prec)

    def bench_step():
        slab.step(delta)
        return slab.nusselt()[0], slab.residual()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(3, args.warmup)):
        bench_step()
    barrier()
    with Clocks(local) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(args.steps):
            nu, _r = bench_step()
        t1.record()
        barrier()
    total = max_over_ranks(t0.elapsed_time(t1) / 1e3, world, "cuda")
    slab.ops.close()
    if own_group:
        dist.destroy_process_group()
    if rank != 0:
        return
    y0, y1 = slabs.partition(N, world)[0]
    line = {
        "metric": "fused MRT step MLUPS", "value": N * N * delta * args.steps / total / 1e6, "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f64" if prec == "f64" else "f32", "data": "synthetic",
        "config": {"workload": f"one cavity {N}x{N} in {world} row slabs (rank 0: rows {y0}-{y1}), "
                               f"{STORAGE_NAMES[prec]} storage; halo exchange every fused step",
                   "grid": [N, N], "fused_steps_per_bench_step": delta, "parallelism": f"row slabs x{world}",
                   "halo_bytes_per_cut_per_step": 2 * 4 * N * {"f64": 8}.get(prec, 2 if "16" in prec else 4)},
        "gpu_launches": args.steps * (delta * (3 if world > 1 else 1) + 3),
        "clocks": clk.summary(),
        "nu_hot": nu,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.study == "adjoint":
        study_adjoint(args)
        return
    if args.study == "batch":
        study_batch(args)
        return
    if args.study == "tables":
        study_tables(args)
        return
    if args.study == "precision":
        study_precision(args)
        return
    if args.study == "plain":
        study_plain(args)
        return
    if args.study == "grid":
        study_grid(args)
        return
    if args.study == "sensitivity":
        study_sensitivity(args)
        return
    if args.study == "throughput":
        study_throughput(args)
        return
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
    if args.scaling == "strong":
        run_strong(args, torch, lbm, rank, world, local)
        return
    stream = torch.cuda.Stream()
    N, prec, delta = args.N, args.prec, args.delta

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    barrier()
    with Clocks(local) as clk:
        total, kern, launches, nu = time_ours(lbm, torch, N, prec, args.steps, max(3, args.warmup), delta, stream,
                                              layout=args.layout, tau_iters=args.tau_iters, staging=args.staging)
    barrier()
    total = max_over_ranks(total, world, "cuda")
    units = whole_job_units(world, N, delta, args.steps)
    mlups = units / total / 1e6
    peak, peak_src = hbm_peak()
    bpn_main = bytes_per_node(prec, args.tau_iters)
    achieved = bpn_main * N * N / kern / 1e9
    key_main = prec + (f"@tau{args.tau_iters}" if args.tau_iters else "") + \
        {0: "", 1: "@reg", 3: "@quad"}[args.staging] + ("@aa" if args.layout else "")
    peaks = alu_peaks(lbm)
    variants = {}
    for v in [p for p in args.variants.split(",") if p and p != key_main]:
        vs, vd = 2, args.variant_delta
        vp, vl, vt, vg = parse_variant(v)
        tv, kv, _, nuv = time_ours(lbm, torch, N, vp, vs, 1, vd, stream, layout=vl, tau_iters=vt, staging=vg)
        bpn = bytes_per_node(vp, vt)
        av = bpn * N * N / kv / 1e9
        variants[v] = {"MLUPS": N * N * vd * vs / tv / 1e6, "kernel_MLUPS": N * N / kv / 1e6,
                       "fused_steps_per_bench_step": vd,
                       "bytes_per_node": bpn, "achieved_GBs": av, "frac_of_hbm": av / peak,
                       "layout": "aa (in place)" if vl else "ab (two buffers)",
                       "tau": f"implicit, {vt} Newton steps" if vt else "lagged (stored)",
                       "dnu_rel_vs_f64_512": recorded_dnu(vp),
                       "staging": staging_label(vp, vl, vt, vg, N),
                       "kernel": step_kernel_name(vp, vl, vt, vg, N),
                       "nu_hot": nuv}
        if v == "f64":
            ipn = recorded("f64_fp64_inst_per_node")
            if ipn:
                peak_inst = peaks["f64"]["inst_per_s"]
                ach = N * N / kv * ipn
                variants[v]["roofline"] = {"bound": "alu", "unit": "FP64 inst/s", "achieved": ach,
                                           "peak": peak_inst, "frac": ach / peak_inst,
                                           "fp64_inst_per_node": ipn,
                                           "peak_source": "measured: lbm_bench_fma_peak FP64 FMA throughput"}
    # launch-bound small grid: one launch per step against replayed step graphs
    small = {"grid": [256, 256], "storage": "f32d", "fused_steps": 2 * 5000}
    for key, gs in (("MLUPS_one_launch_per_step", -1), ("MLUPS_replayed_graphs", 0)):
        ts, _, _, _ = time_ours(lbm, torch, 256, "f32d", 2, 1, 5000, stream, graph_steps=gs)
        small[key] = 256 * 256 * 5000 * 2 / ts / 1e6
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
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == "f64" else "f32",
        "data": "synthetic",
        "config": {"workload": f"cavity {N}x{N}, n={CASE['n']}, Da={CASE['Da']}, Ra={CASE['Ra']}, "
                               f"Pr={CASE['Pr']}, porosity={CASE['porosity']}, {STORAGE_NAMES[prec]} storage, "
                               + (f"implicit tau ({args.tau_iters} Newton steps)" if args.tau_iters
                                  else "lagged tau") +
                               f"; bench step = {delta} fused steps + Nu + residual",
                   "grid": [N, N], "fused_steps_per_bench_step": delta,
                   "l2": "state larger than L2 (no flush needed)", "parallelism": f"independent cavity per GPU x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": recorded_traffic(key_main, N),
                     "peak_source": peak_src,
                     "kernel": step_kernel_name(prec, args.layout, args.tau_iters, args.staging, N) +
                               f"<{key_main}>",
                     "bytes_per_node": bpn_main, "avg_launch_us": kern * 1e6,
                     # the arithmetic side of the same kernel: FMA-pipe activity (ncu, 2048^2)
                     "fma_pipe_active": recorded(key_main + "_fma_pipe_active")},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "nu_hot": nu,
        "variants": variants,
        "reduced_storage": reduced_storage_summary(variants, prec, mlups),
        "small_grid": small,
        "alu_peaks": peaks,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    try:
        main()
    finally:
        _dist = sys.modules.get("torch.distributed")
        if _dist is not None and _dist.is_available() and _dist.is_initialized():
            _dist.destroy_process_group()
