"""The FMA-throughput probe that gives the ALU rooflines a measured peak.

Checked against what the hardware's structure fixes, not against a number:
each kind returns a finite positive rate below the nominal ceiling of 152 SMs
x 128 FP32 lanes x 2 (packed) x 2.07 GHz, FP32 runs many times faster than
FP64 on this part, and a packed FP32x2 instruction does two FMAs.
"""
import math

import pytest

pytestmark = pytest.mark.gpu

CEILING = 152 * 128 * 2 * 2.07e9 * 1.05   # packed FP32 FMAs per second, with margin


def test_fma_probe_rates_are_ordered_and_bounded():
    from paper_2011_15073_gb300 import lbm
    r = {k: lbm.bench_fma_peak(k, reps=5) for k in ("f64", "f32", "f32x2")}
    for k, (fma, inst) in r.items():
        assert math.isfinite(fma) and 0 < fma < CEILING, (k, fma)
        assert inst > 0
    assert r["f32x2"][0] == pytest.approx(2 * r["f32x2"][1])
    assert r["f32"][0] == pytest.approx(r["f32"][1])
    assert r["f32"][0] > 8 * r["f64"][0]

