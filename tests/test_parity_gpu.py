"""GPU parity: the CUDA library against the FP64 oracle on the same seeded inputs.

Tolerances (element by element):
* FP64 storage and arithmetic: relative 1e-12 on f and g after 100 steps and
  1e-10 on the average Nusselt number (the stated FP64 bar); tau below.  Both sides
  compute the same real-number expression in a different order, so the gap
  is a few ulps per step and does not grow in a dissipative scheme.
* FP32 storage and arithmetic: the input is rounded to FP32 before either side
  sees it.  Each step rounds every population once on store and about ten
  times in the arithmetic (unit roundoff 6e-8, special functions within
  2 ulp), so after 100 steps the population error is bounded by
  100 x 10 x 6e-8 = 6e-5 relative in the worst (all-aligned) case; the test
  uses 5e-5 of the population scale (rest weight).  The wall Nusselt number
  amplifies the temperature error by about 3 L (a one-sided difference times
  L), so Nu gets 1e-4 relative.
* The literal modified power law (Eq. MPL) jumps at gamma_1, so a node whose
  strain rate lies within rounding of gamma_1 may take either branch in FP32,
  changing its viscosity several-fold; through the Darcy drag that changes
  the node's velocity, and over many steps the difference spreads.  Results
  are then not unique, so multi-step FP32 and 16-bit parity uses the
  continuous clamp (clamp_mode 1), and the literal law is checked one step
  at a time from identical inputs (a branch flip then only changes the
  relaxation of the tiny p_xx, p_xy non-equilibrium moments, < 1e-6 w) and
  by the sampled full-size test.
* 16-bit deviation storage (FP32 arithmetic): each store rounds the deviation
  f - w_i (or g - w_i T_m) to 8 (BF16) or 11 (FP16) significant bits, i.e.
  to 2^-9 or 2^-12 of the deviation.  Deviations reach 2e-2 w for the flow
  populations and 0.5 w for the thermal ones (T spans [0, 1] around
  T_m = 1/2).  One step: BF16 f 1e-4 w, g 2e-3 w; FP16 f 1e-5 w, g 2.5e-4 w.
  After 100 steps (rounding errors add as a random walk, x 10): BF16 f 2e-3 w,
  g 2e-2 w; FP16 f 2e-4 w, g 2.5e-3 w.
* The relaxation time tau and the apparent viscosity are not populations:
  they come from the strain rate, a small difference of O(1) moments, through
  the modified power law, whose literal form jumps at gamma_1.  They are
  checked node by node with ``parity_util.check_tau``: unique (to the
  propagated strain-rate error) where the oracle's strain rate is resolved,
  and otherwise the law's value at a strain rate within the error band.
"""
import math

import numpy as np
import pytest

from parity_util import check_tau

pytestmark = pytest.mark.gpu

CASES = {
    # sweep corner of the paper's abstract: shear-thinning, porous, high Ra
    "thinning": dict(n=0.6, Da=1e-2, Ra=1e5, Pr=6.2, porosity=0.6, porous_model=1, clamp_mode=0),
    # the plain Newtonian cavity at low Ra, porosity 0.6, Pr 10
    "newtonian": dict(n=1.0, Da=1e-1, Ra=1e3, Pr=10.0, porosity=0.6, porous_model=1, clamp_mode=0),
    # the paper's own Darcy model, continuous clamp
    "darcy": dict(n=0.8, Da=1e-3, Ra=1e4, Pr=6.2, porosity=1.0, porous_model=0, clamp_mode=1),
    # shear-thickening case of the paper's tables
    "thickening": dict(n=1.4, Da=1e-3, Ra=1e5, Pr=6.2, porosity=0.6, porous_model=1, clamp_mode=0),
}
SIZES = [(8, 8), (17, 13), (64, 64), (130, 67), (2, 2), (3, 70)]


@pytest.fixture(scope="module")
def mods():
    import oracle
    from paper_2011_15073_gb300 import inputs, lbm
    oracle.build()
    lbm.lib()
    return oracle, inputs, lbm


def oracle_for(oracle, nx, ny, c):
    return oracle.Cavity.from_params(nx, ny, c["n"], c["Da"], c["Ra"], c["Pr"], porosity=c["porosity"],
                                     porous_model=c["porous_model"], clamp_mode=c["clamp_mode"])


def gpu_for(lbm, nx, ny, c, prec, layout=0):
    return lbm.Cavity(nx, ny, c["n"], c["Da"], c["Ra"], c["Pr"], c["porosity"], prec=prec,
                      porous_model=c["porous_model"], clamp_mode=c["clamp_mode"], layout=layout)


LAYOUTS = pytest.mark.parametrize("layout", [0, 1], ids=["ab", "aa"])


def rel_err(a, b, scale):
    return float(np.max(np.abs(a - b) / scale))


W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
W5 = np.array([1 / 3] + [1 / 6] * 4)[:, None, None]


def test_lattice_mapping_matches_oracle(mods):
    oracle, _, lbm = mods
    for c in CASES.values():
        ref = oracle_for(oracle, 64, 48, c).lat
        with gpu_for(lbm, 64, 48, c, "f64") as cav:
            L = cav.lattice()
        for k in ("nu_ref", "gamma_scale", "gamma1", "gamma2", "K", "eps", "Feps", "gbeta", "Tm",
                  "tauT", "s_e", "s_p", "T_hot", "T_cold", "L", "tau0", "n"):
            a, b = getattr(L, k), getattr(ref, k)
            assert a == pytest.approx(b, rel=1e-15, abs=0), k
        assert L.clamp_mode == ref.clamp_mode


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16d", "f16d"])
def test_initial_state_is_rest_state(mods, prec):
    oracle, _, lbm = mods
    c = CASES["thinning"]
    f0, g0, t0 = oracle_for(oracle, 17, 13, c).get_state()
    with gpu_for(lbm, 17, 13, c, prec) as cav:
        f, g, tau = cav.get_state_f64()
    tol = 0 if prec == "f64" else 1e-7
    assert rel_err(f, f0, W9) <= tol and rel_err(g, g0, W5) <= tol
    assert np.max(np.abs(tau - t0) / t0) <= tol


@LAYOUTS
@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("size", SIZES, ids=lambda s: f"{s[0]}x{s[1]}")
def test_fp64_step_parity(mods, case, size, layout):
    oracle, inputs, lbm = mods
    nx, ny = size
    c = CASES[case]
    ref = oracle_for(oracle, nx, ny, c)
    state = inputs.perturbed_state(ref.get_state(), seed=nx * 1000 + ny)
    ref.set_state(*state)
    ref.step(99)
    f99_r, g99_r, _ = ref.get_state()
    gam_r = ref.fields()["gamma"]
    ref.step(1)
    f_r, g_r, t_r = ref.get_state()
    with gpu_for(lbm, nx, ny, c, "f64", layout) as cav:
        cav.set_state_f64(*state)
        cav.step(99)
        f99, g99, _ = cav.get_state_f64()
        cav.step(1)
        f, g, tau = cav.get_state_f64()
        hot, cold, loc = cav.nusselt(local=True)
        fl = cav.fields()
    assert np.max(np.abs(f - f_r) / np.abs(f_r)) < 1e-12
    assert np.max(np.abs(g - g_r) / np.abs(g_r)) < 1e-12
    df = max(np.abs(f99 - f99_r).max(), np.abs(g99 - g99_r).max())
    check_tau(tau, t_r, gam_r, ref.lat, "f64", df)
    h_r, c_r, loc_r = ref.nusselt()
    assert abs(hot - h_r) <= 1e-10 * abs(h_r) and abs(cold - c_r) <= 1e-10 * abs(c_r)
    assert np.max(np.abs(loc - loc_r)) <= 1e-10 * np.max(np.abs(loc_r))
    fr = ref.fields()
    for k in ("rho", "T"):
        assert np.max(np.abs(fl[k] - fr[k]) / np.abs(fr[k])) < 1e-12, k
    df = max(np.abs(f - f_r).max(), np.abs(g - g_r).max())
    check_tau(3 * fl["nu"] + 0.5, 3 * fr["nu"] + 0.5, fr["gamma"], ref.lat, "f64", df)
    # u = sum f e / rho + ...: a sum of O(0.1) populations that nearly cancel,
    # so its error is absolute: six populations within 1e-12 relative give
    # |du| <= 6 x 1e-12 x 0.11 < 1e-12 (lattice units; U_c = 0.058).
    for k in ("ux", "uy"):
        assert np.max(np.abs(fl[k] - fr[k])) <= 1e-12, k


def test_fp64_parity_covers_both_clamp_branches(mods):
    """The thinning case at 64x64 must see nodes on both sides of gamma_1,
    otherwise the parity above would not exercise the literal clamp."""
    oracle, inputs, _ = mods
    c = CASES["thinning"]
    ref = oracle_for(oracle, 64, 64, c)
    ref.set_state(*inputs.perturbed_state(ref.get_state(), seed=64 * 1000 + 64))
    seen_low = seen_high = False
    for _ in range(10):
        ref.step(10)
        gs = ref.fields()["gamma"] * ref.lat.gamma_scale
        seen_low |= bool((gs < ref.lat.gamma1).any())
        seen_high |= bool((gs >= ref.lat.gamma1).any())
    assert seen_low and seen_high


@LAYOUTS
@pytest.mark.parametrize("case", ["thinning", "darcy", "thickening"])
@pytest.mark.parametrize("size", [(17, 13), (130, 67)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_fp32_step_parity(mods, case, size, layout):
    oracle, inputs, lbm = mods
    nx, ny = size
    c = dict(CASES[case], clamp_mode=1)
    ref = oracle_for(oracle, nx, ny, c)
    state = [a.astype(np.float32).astype(np.float64) for a in
             inputs.perturbed_state(ref.get_state(), seed=7 + nx)]
    ref.set_state(*state)
    ref.step(99)
    f99_r, g99_r, _ = ref.get_state()
    gam_r = ref.fields()["gamma"]
    ref.step(1)
    f_r, g_r, t_r = ref.get_state()
    with gpu_for(lbm, nx, ny, c, "f32", layout) as cav:
        cav.set_state_f64(*state)
        cav.step(99)
        f99, g99, _ = cav.get_state_f64()
        cav.step(1)
        f, g, tau = cav.get_state_f64()
        hot = cav.nusselt()[0]
    assert rel_err(f, f_r, W9) < 5e-5
    assert rel_err(g, g_r, W5) < 5e-5
    df = max(np.abs(f99 - f99_r).max(), np.abs(g99 - g99_r).max())
    check_tau(tau, t_r, gam_r, ref.lat, "f32", df)
    h_r = ref.nusselt()[0]
    assert abs(hot - h_r) <= 1e-4 * abs(h_r)


@LAYOUTS
@pytest.mark.parametrize("prec,tol_f,tol_g", [("bf16d", 2e-3, 2e-2), ("f16d", 2e-4, 2.5e-3)])
def test_deviation_storage_parity(mods, prec, tol_f, tol_g, layout):
    oracle, inputs, lbm = mods
    nx, ny = 130, 67
    c = dict(CASES["thinning"], clamp_mode=1)
    ref = oracle_for(oracle, nx, ny, c)
    state = inputs.perturbed_state(ref.get_state(), seed=11)
    ref.set_state(*state)
    ref.step(99)
    f99_r, g99_r, _ = ref.get_state()
    gam_r = ref.fields()["gamma"]
    ref.step(1)
    f_r, g_r, t_r = ref.get_state()
    with gpu_for(lbm, nx, ny, c, prec, layout) as cav:
        cav.set_state_f64(*state)
        cav.step(99)
        f99, g99, _ = cav.get_state_f64()
        cav.step(1)
        f, g, tau = cav.get_state_f64()
    assert rel_err(f, f_r, W9) < tol_f
    assert rel_err(g, g_r, W5) < tol_g
    df = max(np.abs(f99 - f99_r).max(), np.abs(g99 - g99_r).max())
    check_tau(tau, t_r, gam_r, ref.lat, prec, df)


@pytest.mark.parametrize("prec,tol_f,tol_g", [("f32", 2e-6, 2e-6)])
@pytest.mark.parametrize("case", ["thinning", "thickening", "newtonian"])
@pytest.mark.parametrize("size", [(17, 13), (130, 67), (258, 9)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_one_step_parity_literal_clamp(mods, prec, tol_f, tol_g, case, size):
    """One step from the same input with the literal law.  The input is an
    evolved FP64 oracle state (developed flow, strain rates on both sides of
    gamma_1) rounded to FP32, given to both sides.  (The 16-bit forms round
    every input on import, which puts most nodes inside the strain-rate band
    of gamma_1; they are covered by the multi-step continuous-law test.)"""
    oracle, inputs, lbm = mods
    nx, ny = size
    c = CASES[case]
    ref = oracle_for(oracle, nx, ny, c)
    ref.set_state(*inputs.perturbed_state(ref.get_state(), seed=3 * nx + ny, amp=1e-2))
    ref.step(40)
    state = [a.astype(np.float32).astype(np.float64) for a in ref.get_state()]
    ref.set_state(*state)
    gam_r = ref.fields()["gamma"]
    ref.step(1)
    f_r, g_r, t_r = ref.get_state()
    with gpu_for(lbm, nx, ny, c, prec) as cav:
        cav.set_state_f64(*state)
        cav.step(1)
        f, g, tau = cav.get_state_f64()
    unit = {"f32": 0.0, "bf16d": 2.0 ** -9, "f16d": 2.0 ** -12}[prec]
    df = unit * max(np.abs(state[0] - W9).max(), np.abs(state[1] - W5 / 2).max())
    # a node whose strain rate lies within the rounding band of gamma_1 may
    # take either branch of the law: its tau (hence its relaxation of p_xx,
    # p_xy) is then one of two valid values, checked by check_tau; its
    # populations differ from the oracle's by at most the change of that
    # relaxation, |dw| |p_neq| / 4 < 1e-3 w
    dgam = 100.0 * df + 100.0 * 2.0 ** -24
    gs = gam_r * ref.lat.gamma_scale
    amb = np.abs(gs - ref.lat.gamma1) <= dgam * ref.lat.gamma_scale
    ef = np.max(np.abs(f - f_r) / W9, axis=0)
    eg = np.max(np.abs(g - g_r) / W5, axis=0)
    assert ef[~amb].max() < tol_f and eg[~amb].max() < tol_g
    if amb.any():
        assert ef[amb].max() < 1e-3 and eg[amb].max() < tol_g
    assert amb.mean() < 0.5   # most nodes are unambiguous, so the strict bound is exercised
    check_tau(tau, t_r, gam_r, ref.lat, prec, df)
