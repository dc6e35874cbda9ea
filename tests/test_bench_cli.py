"""bench.py keeps its command-line contract (CPU part): the reference arm
runs and prints one JSON line with the keys the benchmark contract names."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0


def test_bench_defines_every_leg():
    src = open(os.path.join(ROOT, "bench.py")).read()
    for fn in ("def time_ours", "def time_e2e", "def cpu_baseline", "def run_reference", "def hbm_peak",
               "def dist_env", "class Clocks", "def study_tables", "def study_precision", "def study_batch",
               "def study_adjoint", "def study_plain", "def study_throughput", "def study_grid", "def main"):
        assert fn in src, fn


def test_variant_names():
    import bench
    assert bench.parse_variant("f32") == ("f32", 0, 0, 0)
    assert bench.parse_variant("f32@aa") == ("f32", 1, 0, 0)
    assert bench.parse_variant("f32@tau2") == ("f32", 0, 2, 0)
    assert bench.parse_variant("f32d@aa@tau3") == ("f32d", 1, 3, 0)
    assert bench.parse_variant("bf16d@tau2@reg") == ("bf16d", 0, 2, 1)
    assert bench.parse_variant("f16s@quad") == ("f16s", 0, 0, 3)
    # the auto rule of lbm_opts.staging: four nodes per thread for the 16-bit
    # storages from 2048^2 on (4096^2 with the implicit tau)
    assert bench.step_kernel_name("f16s", 0, 0, 0, 4096) == "step4_kernel"
    assert bench.step_kernel_name("f16s", 0, 0, 0, 2048) == "step4_kernel"
    assert bench.step_kernel_name("f16s", 0, 0, 0, 1024) == "step2_kernel"
    assert bench.step_kernel_name("f16s", 0, 2, 0, 4096) == "step4_kernel"
    assert bench.step_kernel_name("f16s", 0, 2, 0, 2048) == "step2_kernel"
    assert bench.step_kernel_name("f16s", 0, 0, 1, 4096) == "step2_kernel"
    assert bench.step_kernel_name("f32d", 0, 0, 0, 4096) == "step2_kernel"
    assert bench.step_kernel_name("f64", 0, 0, 0, 4096) == "step_kernel"
    assert bench.bytes_per_node("f32", 2) == 112 and bench.bytes_per_node("f64", 1) == 224
    with pytest.raises(ValueError):
        bench.parse_variant("f32@bogus")
    with pytest.raises(ValueError):
        bench.parse_variant("f32d@tma")   # the staged kernel is not built


def test_reduced_storage_summary_picks_fastest_within_the_bar():
    import bench
    v = {"f64": {"MLUPS": 2000.0},
         "f16s": {"MLUPS": 69000.0, "dnu_rel_vs_f64_512": 7.6e-4},
         "bf16s": {"MLUPS": 71000.0, "dnu_rel_vs_f64_512": 2.4e-3},    # faster, misses the bar
         "f16d": {"MLUPS": 74000.0, "dnu_rel_vs_f64_512": 0.14},
         "f32": {"MLUPS": 54000.0, "dnu_rel_vs_f64_512": None}}       # no record: not a candidate
    s = bench.reduced_storage_summary(v, "f32d", 57000.0)
    assert s["variant"] == "f16s" and s["speedup_vs_f64_storage"] == 69000.0 / 2000.0
    assert bench.reduced_storage_summary({"f16s": v["f16s"]}, "f32d", 1.0) is None   # no FP64 run to compare


def test_recorded_fp64_reference_reads_the_committed_1024_rows():
    """--study-ref takes the FP64 rows (Nu and step count per n) of the grid
    asked for from an earlier output, skipping comment and other lines."""
    import bench
    ref = bench.recorded_fp64_reference(os.path.join(ROOT, "profiles", "precision_study_1024.txt"), 1024)
    assert sorted(ref) == [0.6, 1.0]
    assert ref[0.6]["steps"] == 1836000 and ref[1.0]["steps"] == 2512000
    assert abs(ref[0.6]["nu_hot"] - 8.124632) < 1e-6 and abs(ref[1.0]["nu_hot"] - 3.673356) < 1e-6
    assert bench.recorded_fp64_reference(os.path.join(ROOT, "profiles", "precision_study_1024.txt"), 512) == {}
