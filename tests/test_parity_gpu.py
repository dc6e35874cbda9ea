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
  to 2^-9 or 2^-12 of the deviation (stochastic rounding, F16S / BF16S: up to
  one whole spacing per store, so twice the bounds below).  Deviations reach 2e-2 w for the flow
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


@pytest.mark.parametrize("prec", ["f64", "f32", "f32d", "bf16d", "f16d", "f16s", "bf16s"])
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
@pytest.mark.parametrize("prec", ["f32", "f32d"])
@pytest.mark.parametrize("case", ["thinning", "darcy", "thickening"])
@pytest.mark.parametrize("size", [(17, 13), (130, 67)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_fp32_step_parity(mods, case, size, layout, prec):
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
    with gpu_for(lbm, nx, ny, c, prec, layout) as cav:
        cav.set_state_f64(*state)
        cav.step(99)
        f99, g99, _ = cav.get_state_f64()
        cav.step(1)
        f, g, tau = cav.get_state_f64()
        hot = cav.nusselt()[0]
    assert rel_err(f, f_r, W9) < 5e-5
    assert rel_err(g, g_r, W5) < 5e-5
    df = max(np.abs(f99 - f99_r).max(), np.abs(g99 - g99_r).max())
    check_tau(tau, t_r, gam_r, ref.lat, prec, df)
    h_r = ref.nusselt()[0]
    assert abs(hot - h_r) <= 1e-4 * abs(h_r)


@LAYOUTS
@pytest.mark.parametrize("prec,tol_f,tol_g", [("bf16d", 2e-3, 2e-2), ("f16d", 2e-4, 2.5e-3),
                                              ("bf16s", 4e-3, 4e-2), ("f16s", 4e-4, 5e-3)])
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


@pytest.mark.parametrize("prec,tol_f,tol_g", [("bf16s", 4e-3, 4e-2), ("f16s", 4e-4, 5e-3)])
def test_rounding_stream_seed(mods, prec, tol_f, tol_g):
    """lbm_opts.seed selects another stochastic-rounding stream: the states
    differ from the default stream's, and both stay within the stochastic
    bounds of the oracle after 100 steps."""
    oracle, inputs, lbm = mods
    nx, ny = 130, 67
    c = dict(CASES["thinning"], clamp_mode=1)
    ref = oracle_for(oracle, nx, ny, c)
    state = inputs.perturbed_state(ref.get_state(), seed=11)
    ref.set_state(*state)
    ref.step(100)
    f_r, g_r, _ = ref.get_state()
    out = {}
    for seed in (0, 7):
        with lbm.Cavity(nx, ny, c["n"], c["Da"], c["Ra"], c["Pr"], c["porosity"], prec=prec,
                        porous_model=c["porous_model"], clamp_mode=1, seed=seed) as cav:
            cav.set_state_f64(*state)
            cav.step(100)
            out[seed] = cav.get_state_f64()[:2]
    for f, g in out.values():
        assert rel_err(f, f_r, W9) < tol_f
        assert rel_err(g, g_r, W5) < tol_g
    assert not np.array_equal(out[0][0], out[7][0])


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


@LAYOUTS
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_darcy_field_parity(mods, prec, layout):
    """A per-node Darcy field, log-uniform in [1e-3, 1e-1], against the oracle
    with the same field (FP32 with the continuous law, as above)."""
    oracle, inputs, lbm = mods
    nx, ny = 130, 67
    c = dict(CASES["thinning"], clamp_mode=1 if prec == "f32" else 0)
    Da = inputs.darcy_field(2011, nx, ny)
    ref = oracle_for(oracle, nx, ny, c)
    ref.set_darcy_field(Da)
    state = inputs.perturbed_state(ref.get_state(), seed=77)
    if prec == "f32":
        state = [a.astype(np.float32).astype(np.float64) for a in state]
    ref.set_state(*state)
    ref.step(59)
    f59_r, g59_r, _ = ref.get_state()
    gam_r = ref.fields()["gamma"]
    ref.step(1)
    f_r, g_r, t_r = ref.get_state()
    with gpu_for(lbm, nx, ny, c, prec, layout) as cav:
        cav.set_darcy_field(Da)
        cav.set_state_f64(*state)
        cav.step(59)
        f59, g59, _ = cav.get_state_f64()
        cav.step(1)
        f, g, tau = cav.get_state_f64()
    tol = 1e-12 if prec == "f64" else 5e-5
    assert rel_err(f, f_r, W9) < tol and rel_err(g, g_r, W5) < tol
    df = max(np.abs(f59 - f59_r).max(), np.abs(g59 - g59_r).max())
    check_tau(tau, t_r, gam_r, ref.lat, prec, df)


def test_zero_steps_and_repeat_calls(mods):
    oracle, inputs, lbm = mods
    c = CASES["thinning"]
    ref = oracle_for(oracle, 17, 13, c)
    state = inputs.perturbed_state(ref.get_state(), seed=5)
    with gpu_for(lbm, 17, 13, c, "f64") as cav:
        cav.set_state_f64(*state)
        cav.step(0)
        f, g, tau = cav.get_state_f64()
        assert np.array_equal(f, state[0]) and np.array_equal(g, state[1])
        cav.step(3)
        cav.step(4)
        a = cav.get_state_f64()
    ref.set_state(*state)
    ref.step(7)
    b = ref.get_state()
    for x, y in zip(a[:2], b[:2]):
        assert np.max(np.abs(x - y) / np.abs(y)) < 1e-13
    assert np.max(np.abs(a[2] - b[2]) / b[2]) < 1e-10   # tau: see check_tau


@LAYOUTS
@pytest.mark.parametrize("nx", [33, 128], ids=["padded", "unpadded"])
def test_native_state_roundtrip(mods, layout, nx):
    """Native state out and back in: padded rows (strided copies) and rows
    of a multiple of 64 nodes (one linear copy), both layouts."""
    _, inputs, lbm = mods
    c = CASES["thinning"]
    for prec in ("f64", "f32", "f32d", "bf16d", "f16d"):
        with gpu_for(lbm, nx, 21, c, prec, layout) as cav:
            cav.step(5)
            buf = np.empty(cav.state_bytes(), dtype=np.uint8)
            cav.get_state(buf)
            cav.step(5)
            after = np.empty_like(buf)
            cav.get_state(after)
            cav.set_state(buf)
            cav.step(5)
            again = np.empty_like(buf)
            cav.get_state(again)
            assert np.array_equal(after, again), prec
            if prec == "f64":   # native layout: f0..f8, g0..g4, tau planes of ny x nx values
                f, g, tau = cav.get_state_f64()
                planes = again.view(np.float64).reshape(15, 21, nx)
                assert np.array_equal(planes[:9], f) and np.array_equal(planes[9:14], g)
                assert np.array_equal(planes[14], tau)


def test_residual_matches_definition(mods):
    oracle, inputs, lbm = mods
    c = CASES["thinning"]
    nx, ny = 40, 30
    ref = oracle_for(oracle, nx, ny, c)
    state = inputs.perturbed_state(ref.get_state(), seed=9)
    ref.set_state(*state)
    with gpu_for(lbm, nx, ny, c, "f64") as cav:
        cav.set_state_f64(*state)
        assert math.isinf(cav.residual())
        cav.step(50)
        r = cav.residual()
    a = ref.fields()
    ref.step(50)
    b = ref.fields()
    expect = max(np.linalg.norm(b[k] - a[k]) / np.linalg.norm(b[k]) for k in ("ux", "uy", "T"))
    assert r == pytest.approx(expect, rel=1e-9)


def test_nonfinite_state_is_reported(mods):
    oracle, inputs, lbm = mods
    c = CASES["thinning"]
    ref = oracle_for(oracle, 16, 16, c)
    f, g, tau = ref.get_state()
    f = f.copy()
    f[3, 7, 9] = np.nan
    with gpu_for(lbm, 16, 16, c, "f32") as cav:
        cav.set_state_f64(f, g, tau)
        with pytest.raises(lbm.LBMError) as e:
            cav.residual()
        assert e.value.code == -3


@pytest.mark.parametrize("prec,layout", [("f32", 0), ("f64", 0), ("f32", 1), ("f32d", 0), ("f16s", 0)])
def test_full_size_sampled_parity(mods, prec, layout):
    """4096 x 4096, the benchmark's launch configuration: the state after k
    steps at a node depends only on the (2k+1)^2 nodes around it, so the
    oracle recomputes sampled nodes one window at a time.  A window that
    touches a real wall keeps it; its artificial edges stay more than k nodes
    away from the sampled node.  The state goes in and out in the native
    storage (values, FP32 deviations from rest, or FP16 deviations x 2^15)."""
    oracle, inputs, lbm = mods
    N, k, h = 4096, 3, 5
    c = CASES["thinning"]
    lat_full = oracle.map_params(N, N, c["n"], c["Da"], c["Ra"], c["Pr"], porosity=c["porosity"])
    rest = oracle.Cavity(oracle.map_params(4, 4, 1.0, 1e-2, 1e5, 6.2))
    f0, g0, t0 = rest.get_state()
    wf, wg = f0[:, :1, :1], g0[:, :1, :1]          # rest values w_i and w_i T_m
    rng = np.random.default_rng(4096)
    df_in = wf * rng.uniform(-1e-3, 1e-3, (9, N, N))
    dg_in = wg * rng.uniform(-1e-3, 1e-3, (5, N, N))
    if prec == "f16s":   # stored: FP16 of the deviation x 2^15 (exactly representable inputs)
        sf, sg = (df_in * 32768).astype(np.float16), (dg_in * 32768).astype(np.float16)
        f = wf + sf.astype(np.float64) / 32768
        g = wg + sg.astype(np.float64) / 32768
        host_fg = [sf.reshape(-1).view(np.uint8), sg.reshape(-1).view(np.uint8)]
    else:
        dt = np.float64 if prec == "f64" else np.float32
        if prec == "f32d":
            sf, sg = df_in.astype(dt), dg_in.astype(dt)
            f, g = wf + sf.astype(np.float64), wg + sg.astype(np.float64)
        else:
            sf, sg = (wf + df_in).astype(dt), (wg + dg_in).astype(dt)
            f, g = sf.astype(np.float64), sg.astype(np.float64)
        host_fg = [sf.reshape(-1).view(np.uint8), sg.reshape(-1).view(np.uint8)]
    tdt = np.float64 if prec == "f64" else np.float32
    tau_s = np.full((N, N), lat_full.tau0, dtype=tdt)
    tau = tau_s.astype(np.float64)
    with gpu_for(lbm, N, N, c, prec, layout) as cav:
        host = np.concatenate(host_fg + [tau_s.reshape(-1).view(np.uint8)])
        cav.set_state(host)
        cav.step(k)
        out = np.empty_like(host)
        cav.get_state(out)
    nn = N * N
    nf, ng = len(host_fg[0]), len(host_fg[1])
    if prec == "f16s":
        fo = wf + out[:nf].view(np.float16).astype(np.float64).reshape(9, N, N) / 32768
        go = wg + out[nf:nf + ng].view(np.float16).astype(np.float64).reshape(5, N, N) / 32768
    else:
        fo = out[:nf].view(tdt).astype(np.float64).reshape(9, N, N)
        go = out[nf:nf + ng].view(tdt).astype(np.float64).reshape(5, N, N)
        if prec == "f32d":
            fo, go = wf + fo, wg + go
    to = out[nf + ng:].view(tdt).astype(np.float64).reshape(N, N)
    assert nf == 9 * nn * (2 if prec == "f16s" else tdt().itemsize)
    samples = [(0, 0), (N - 1, 0), (0, N - 1), (N - 1, N - 1), (N // 2, 0), (0, N // 2),
               (N - 1, N // 2), (N // 2, N - 1)] + [tuple(rng.integers(0, N, 2)) for _ in range(24)]
    tol = 1e-12 if prec == "f64" else 2e-6
    for (x, y) in samples:
        x0 = 0 if x < h + k else (N - (2 * h + 1) if x > N - 1 - h - k else x - h)
        y0 = 0 if y < h + k else (N - (2 * h + 1) if y > N - 1 - h - k else y - h)
        w = 2 * h + 1
        lat = lat_full.copy()
        lat.nx = lat.ny = w
        win = oracle.Cavity(lat)
        win.set_state(f[:, y0:y0 + w, x0:x0 + w].astype(np.float64),
                      g[:, y0:y0 + w, x0:x0 + w].astype(np.float64),
                      tau[y0:y0 + w, x0:x0 + w].astype(np.float64))
        win.step(k - 1)
        gam_w = win.fields()["gamma"]
        win.step(1)
        fw, gw, tw = win.get_state()
        lx, ly = x - x0, y - y0
        if prec == "f16s":
            # each store rounds a deviation to one of its two FP16 neighbours
            # (spacing at most 2^-10 of its size); after k steps the error stays
            # within k spacings of the largest deviation in the window (at the
            # isothermal walls the thermal ones reach 2w (T_w - T_m))
            for a, b, w in ((fo, fw, wf), (go, gw, wg)):
                dev = np.abs(b - w).max()
                assert np.all(np.abs(a[:, y, x] - b[:, ly, lx]) <= k * 2.0 ** -10 * dev + 1e-9), (x, y)
        else:
            assert np.max(np.abs(fo[:, y, x] - fw[:, ly, lx]) / W9[:, 0, 0]) < tol, (x, y)
            assert np.max(np.abs(go[:, y, x] - gw[:, ly, lx]) / W5[:, 0, 0]) < tol, (x, y)
        df = max(np.max(np.abs(fo[:, y, x] - fw[:, ly, lx])), np.max(np.abs(go[:, y, x] - gw[:, ly, lx])))
        check_tau(np.array([to[y, x]], float), tw[ly, lx:lx + 1], gam_w[ly, lx:lx + 1], lat, prec, df)
