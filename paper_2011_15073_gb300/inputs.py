"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds random numbers and workload descriptions only -- none of
the method's arithmetic.  The paper has no dataset: every input is the
differentially heated cavity itself, described by its grid and the paper's
non-dimensional groups.  Two kinds of synthetic data are produced here:

* relative perturbations ``delta`` of the initial populations, uniform in
  ``[-amp, amp)``, so that shear-dependent viscosity and the clamp are
  exercised from the first step (the rest state has zero strain rate);
* the case list of the paper's (n, Da, Ra) sweep (abstract: 0.6 <= n <= 1,
  1e-3 <= Da <= 1e-1, 1e3 <= Ra <= 1e5) with seeded grid sizes, and a
  seeded log-uniform per-node Darcy field.
"""
from __future__ import annotations

import numpy as np


def perturbation(seed: int, nx: int, ny: int, amp: float = 1e-3):
    """Relative perturbations (dF[9][ny][nx], dG[5][ny][nx]) in [-amp, amp)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dF = rng.uniform(-amp, amp, size=(9, ny, nx))
    dG = rng.uniform(-amp, amp, size=(5, ny, nx))
    return dF, dG


def perturbed_state(state, seed: int, amp: float = 1e-3):
    """Multiply a rest state (f, g, tau) elementwise by (1 + delta)."""
    f, g, tau = state
    ny, nx = tau.shape
    dF, dG = perturbation(seed, nx, ny, amp)
    return f * (1.0 + dF), g * (1.0 + dG), tau.copy()


SWEEP_N = (0.6, 0.8, 1.0)
SWEEP_DA = (1e-3, 1e-2, 1e-1)
SWEEP_RA = (1e3, 1e4, 1e5)
SWEEP_GRIDS = (128, 192, 256, 384, 512)


def splitmix64(x: int) -> int:
    """SplitMix64 output function (Steele, Lea & Flood 2014), 64-bit wrap."""
    mask = (1 << 64) - 1
    z = (x + 0x9E3779B97F4A7C15) & mask
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
    return z ^ (z >> 31)


def sweep_cases(seed: int = 2011):
    """27 cases n x Da x Ra; grid drawn from SWEEP_GRIDS by splitmix64(seed ^ case)."""
    cases = []
    idx = 0
    for n in SWEEP_N:
        for Da in SWEEP_DA:
            for Ra in SWEEP_RA:
                N = SWEEP_GRIDS[splitmix64(seed * 1000003 + idx) % len(SWEEP_GRIDS)]
                cases.append(dict(case=idx, N=N, n=n, Da=Da, Ra=Ra))
                idx += 1
    return cases


def darcy_field(seed: int, nx: int, ny: int, lo: float = 1e-3, hi: float = 1e-1):
    """Per-node Darcy numbers, log-uniform in [lo, hi], shape [ny][nx]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return 10.0 ** rng.uniform(np.log10(lo), np.log10(hi), size=(ny, nx))
