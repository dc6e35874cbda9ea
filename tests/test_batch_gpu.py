"""The batched sweep (lbm_batch_*) against single contexts and the oracle.

A batch steps many cavities of different sizes over one list of row tiles
(per-step launches or one persistent launch per chunk); each case must
evolve exactly as it would alone:
* FP32: bit-for-bit equal to the same case stepped as a single context
  (the batched kernel runs the same tile code on the same numbers), with
  the lagged and with the node-local implicit tau;
* FP64: within the parity bounds of test_parity_gpu against the oracle;
* run-to-steady (host-looped graph and single device-looped graph): the same
  per-case stopping step and Nusselt numbers as lbm_run_to_steady alone;
* the stochastic-rounding storages: bit for bit the single contexts too (each
  step's seed is computed on the device from the case's step count).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [
    dict(nx=17, ny=13, n=0.6, Da=1e-2, Ra=1e5, Pr=6.2, porosity=0.6),
    dict(nx=130, ny=67, n=1.0, Da=1e-1, Ra=1e3, Pr=10.0, porosity=0.6),
    dict(nx=64, ny=64, n=0.8, Da=1e-3, Ra=1e4, Pr=6.2, porosity=0.6),
    dict(nx=258, ny=9, n=1.4, Da=1e-3, Ra=1e5, Pr=6.2, porosity=0.6),
]


@pytest.fixture(scope="module")
def mods():
    import oracle
    from paper_2011_15073_gb300 import inputs, lbm
    oracle.build()
    lbm.lib()
    return oracle, inputs, lbm


def start_states(oracle, inputs, cases):
    out = []
    for i, c in enumerate(cases):
        ref = oracle.Cavity.from_params(c["nx"], c["ny"], c["n"], c["Da"], c["Ra"], c["Pr"],
                                        porosity=c["porosity"], clamp_mode=1)
        out.append((ref, inputs.perturbed_state(ref.get_state(), seed=100 + i)))
    return out


@pytest.mark.parametrize("tuned", [False, True])
def test_batch_fp32_equals_single_contexts(mods, tuned):
    oracle, inputs, lbm = mods
    st = start_states(oracle, inputs, CASES)
    with lbm.Batch(CASES, prec="f32", clamp_mode=1) as b:
        for i, (_, s) in enumerate(st):
            lbm.set_state_f64(b.case_ctx(i), *s)
        if tuned:
            b.tune(20)   # whatever block size it picks, the results may not change
        b.step(37)
        got = [lbm.get_state_f64(b.case_ctx(i), c["nx"], c["ny"]) for i, c in enumerate(CASES)]
    for i, c in enumerate(CASES):
        with lbm.Cavity(c["nx"], c["ny"], c["n"], c["Da"], c["Ra"], c["Pr"], c["porosity"], prec="f32",
                        clamp_mode=1) as cav:
            cav.set_state_f64(*st[i][1])
            cav.step(37)
            want = cav.get_state_f64()
        for a, w in zip(got[i], want):
            assert np.array_equal(a, w), i


@pytest.mark.parametrize("prec", ["f32", "f32d", "f64", "bf16d"])
def test_batch_implicit_tau_equals_single_contexts(mods, prec):
    """With the node-local implicit tau the batched kernel runs the same tile
    (and, in FP64, node) code as a single context: bit for bit."""
    oracle, inputs, lbm = mods
    st = start_states(oracle, inputs, CASES)
    with lbm.Batch(CASES, prec=prec, clamp_mode=1, tau_iters=2) as b:
        for i, (_, s) in enumerate(st):
            lbm.set_state_f64(b.case_ctx(i), *s)
        b.step(37)
        got = [lbm.get_state_f64(b.case_ctx(i), c["nx"], c["ny"]) for i, c in enumerate(CASES)]
    for i, c in enumerate(CASES):
        with lbm.Cavity(c["nx"], c["ny"], c["n"], c["Da"], c["Ra"], c["Pr"], c["porosity"], prec=prec,
                        clamp_mode=1, tau_iters=2) as cav:
            cav.set_state_f64(*st[i][1])
            cav.step(37)
            want = cav.get_state_f64()
        for a, w in zip(got[i], want):
            assert np.array_equal(a, w), i


def test_batch_implicit_tau_fp64_parity_with_oracle(mods):
    oracle, inputs, lbm = mods
    cases = CASES[:3]
    st = []
    for i, c in enumerate(cases):
        ref = oracle.Cavity.from_params(c["nx"], c["ny"], c["n"], c["Da"], c["Ra"], c["Pr"],
                                        porosity=c["porosity"], clamp_mode=1, tau_iters=4)
        st.append((ref, inputs.perturbed_state(ref.get_state(), seed=200 + i)))
    with lbm.Batch(cases, prec="f64", clamp_mode=1, tau_iters=4) as b:
        for i, (_, s) in enumerate(st):
            lbm.set_state_f64(b.case_ctx(i), *s)
        b.step(60)
        got = [lbm.get_state_f64(b.case_ctx(i), c["nx"], c["ny"]) for i, c in enumerate(cases)]
    for i, (ref, s) in enumerate(st):
        ref.set_state(*s)
        ref.step(60)
        f_r, g_r, _ = ref.get_state()
        f, g, _ = got[i]
        assert np.max(np.abs(f - f_r) / np.abs(f_r)) < 1e-12
        assert np.max(np.abs(g - g_r) / np.abs(g_r)) < 1e-12


def test_batch_fp64_parity_with_oracle(mods):
    oracle, inputs, lbm = mods
    st = start_states(oracle, inputs, CASES)
    with lbm.Batch(CASES, prec="f64", clamp_mode=1) as b:
        for i, (_, s) in enumerate(st):
            lbm.set_state_f64(b.case_ctx(i), *s)
        b.step(60)
        got = [lbm.get_state_f64(b.case_ctx(i), c["nx"], c["ny"]) for i, c in enumerate(CASES)]
    for i, (ref, s) in enumerate(st):
        ref.set_state(*s)
        ref.step(60)
        f_r, g_r, t_r = ref.get_state()
        f, g, tau = got[i]
        assert np.max(np.abs(f - f_r) / np.abs(f_r)) < 1e-12
        assert np.max(np.abs(g - g_r) / np.abs(g_r)) < 1e-12
        assert np.max(np.abs(tau - t_r) / t_r) < 1e-10


@pytest.mark.parametrize("graph_mode", [0, 1])
def test_batch_run_to_steady_matches_single_runs(mods, graph_mode):
    _, _, lbm = mods
    cases = [dict(nx=24, ny=24, n=0.8, Da=1e-2, Ra=1e3, Pr=6.2, porosity=0.6),
             dict(nx=32, ny=20, n=1.0, Da=1e-1, Ra=1e4, Pr=6.2, porosity=0.6),
             dict(nx=20, ny=28, n=0.6, Da=1e-3, Ra=1e4, Pr=6.2, porosity=1.0)]
    with lbm.Batch(cases, prec="f64", clamp_mode=1, resid_interval=200) as b:
        steps, res, why = b.run_to_steady(1e-8, 400_000, graph_mode=graph_mode)
        hot, cold = b.nusselt()
    assert all(w == 0 for w in why), (steps, res, why)
    for i, c in enumerate(cases):
        with lbm.Cavity(c["nx"], c["ny"], c["n"], c["Da"], c["Ra"], c["Pr"], c["porosity"], prec="f64",
                        clamp_mode=1, resid_interval=200) as cav:
            s1, r1, w1 = cav.run_to_steady(1e-8, 400_000)
            h1, c1, _ = cav.nusselt()
        assert (steps[i], why[i]) == (s1, w1)
        assert res[i] == pytest.approx(r1, rel=1e-12)
        assert hot[i] == h1 and cold[i] == c1


def test_batch_run_stops_at_max_steps(mods):
    _, _, lbm = mods
    cases = [dict(nx=16, ny=16, n=0.6, Da=1e-2, Ra=1e5, Pr=6.2, porosity=0.6)] * 2
    with lbm.Batch(cases, prec="f32", resid_interval=100) as b:
        steps, res, why = b.run_to_steady(0.0, 1000, graph_mode=1)
    assert steps == [1000, 1000] and why == [2, 2]


PLANS = [("per_step", 64, 2), ("per_step", 256, 32), ("persistent", 128, 4), ("persistent", 64, 1)]


@pytest.mark.parametrize("plan", PLANS, ids=lambda p: f"{p[0]}-{p[1]}x{p[2]}")
@pytest.mark.parametrize("prec,tau_iters", [("f32d", 0), ("f64", 0), ("f32", 2)])
def test_batch_plans_equal_single_contexts(mods, plan, prec, tau_iters):
    """Every execution plan (per-step or persistent launches, block size,
    blocks per SM) runs the same tile code: bit for bit the single contexts,
    over an odd number of steps and after a case drops out of the tile list."""
    oracle, inputs, lbm = mods
    st = start_states(oracle, inputs, CASES)
    with lbm.Batch(CASES, prec=prec, clamp_mode=1, tau_iters=tau_iters) as b:
        b.set_plan(*plan)
        assert b.plan()["mode"] == plan[0]
        for i, (_, s) in enumerate(st):
            lbm.set_state_f64(b.case_ctx(i), *s)
        b.step(37)
        got = [lbm.get_state_f64(b.case_ctx(i), c["nx"], c["ny"]) for i, c in enumerate(CASES)]
    for i, c in enumerate(CASES):
        with lbm.Cavity(c["nx"], c["ny"], c["n"], c["Da"], c["Ra"], c["Pr"], c["porosity"], prec=prec,
                        clamp_mode=1, tau_iters=tau_iters) as cav:
            cav.set_state_f64(*st[i][1])
            cav.step(37)
            want = cav.get_state_f64()
        for a, w in zip(got[i], want):
            assert np.array_equal(a, w), i


@pytest.mark.parametrize("plan", [("per_step", 128, 8), ("persistent", 128, 4)])
def test_batch_run_to_steady_plans_agree(mods, plan):
    """Run-to-steady with cases that retire at different chunks (the tile
    list shrinks on the device): per case the same steps, residual and Nu
    as the case run alone."""
    _, _, lbm = mods
    cases = [dict(nx=24, ny=24, n=0.8, Da=1e-2, Ra=1e3, Pr=6.2, porosity=0.6),
             dict(nx=40, ny=36, n=1.0, Da=1e-1, Ra=1e4, Pr=6.2, porosity=0.6),
             dict(nx=20, ny=28, n=0.6, Da=1e-3, Ra=1e4, Pr=6.2, porosity=1.0)]
    with lbm.Batch(cases, prec="f64", clamp_mode=1, resid_interval=200) as b:
        b.set_plan(*plan)
        steps, res, why = b.run_to_steady(1e-8, 400_000, graph_mode=1)
        hot, _ = b.nusselt()
    assert all(w == 0 for w in why) and len(set(steps)) > 1, (steps, why)
    for i, c in enumerate(cases):
        with lbm.Cavity(c["nx"], c["ny"], c["n"], c["Da"], c["Ra"], c["Pr"], c["porosity"], prec="f64",
                        clamp_mode=1, resid_interval=200) as cav:
            s1, r1, w1 = cav.run_to_steady(1e-8, 400_000)
            h1 = cav.nusselt()[0]
        assert (steps[i], why[i]) == (s1, w1)
        assert res[i] == pytest.approx(r1, rel=1e-12)
        assert hot[i] == h1


def test_persistent_barrier_gives_up_within_its_budget(mods):
    """A wait budget of a few cycles makes the persistent kernel's blocks
    give up the barrier between steps: every block leaves (no wait is
    unbounded) and the batch reports LBM_ERR_TIMEOUT, then keeps reporting
    it (the states are no longer valid)."""
    _, _, lbm = mods
    cases = [dict(nx=256, ny=256, n=0.8, Da=1e-2, Ra=1e4, Pr=6.2, porosity=0.6)] * 3
    with lbm.Batch(cases, prec="f32", resid_interval=100) as b:
        b.set_plan("persistent", 128, 4)
        b.set_wait_budget(4)
        with pytest.raises(lbm.LBMError) as e:
            b.step(20)
        assert e.value.code == -6
        with pytest.raises(lbm.LBMError) as e:
            b.run_to_steady(1e-8, 1000)
        assert e.value.code == -6


def test_batch_tune_keeps_states(mods):
    oracle, inputs, lbm = mods
    st = start_states(oracle, inputs, CASES)
    with lbm.Batch(CASES, prec="f32", clamp_mode=1) as b:
        for i, (_, s) in enumerate(st):
            lbm.set_state_f64(b.case_ctx(i), *s)
        before = [lbm.get_state_f64(b.case_ctx(i), c["nx"], c["ny"]) for i, c in enumerate(CASES)]
        t = b.tune(20)
        plan = b.plan()
        after = [lbm.get_state_f64(b.case_ctx(i), c["nx"], c["ny"]) for i, c in enumerate(CASES)]
    assert t in (64, 128, 256) and plan["threads"] == t
    assert plan["mode"] in ("per_step", "persistent") and plan["blocks_per_sm"] >= 1
    for x, y in zip(before, after):
        for a, w in zip(x, y):
            assert np.array_equal(a, w)


@pytest.mark.parametrize("plan", [("per_step", 128, 8), ("persistent", 128, 4)], ids=lambda p: p[0])
@pytest.mark.parametrize("prec,seed", [("f16s", 0), ("bf16s", 0), ("f16s", 5)])
def test_batch_stochastic_rounding_equals_single_contexts(mods, plan, prec, seed):
    """The stochastic-rounding storages in a batch: each step's seed comes
    from the case's step count on the device, so a batch stepped in two calls
    (20 + 17 steps) holds bit for bit the states of the cases stepped alone
    (the same start states, copied in natively)."""
    oracle, inputs, lbm = mods
    st = start_states(oracle, inputs, CASES)
    start, want = [], []
    for i, c in enumerate(CASES):
        with lbm.Cavity(c["nx"], c["ny"], c["n"], c["Da"], c["Ra"], c["Pr"], c["porosity"], prec=prec,
                        clamp_mode=1, seed=seed) as cav:
            cav.set_state_f64(*st[i][1])
            s0 = np.empty(cav.state_bytes(), np.uint8)
            cav.get_state(s0)
            cav.step(37)
            s1 = np.empty_like(s0)
            cav.get_state(s1)
        start.append(s0)
        want.append(s1)
    with lbm.Batch(CASES, prec=prec, clamp_mode=1, seed=seed) as b:
        b.set_plan(*plan)
        for i in range(len(CASES)):
            lbm.set_state(b.case_ctx(i), start[i])
        b.step(20)
        b.step(17)
        for i in range(len(CASES)):
            got = np.empty_like(want[i])
            lbm.get_state(b.case_ctx(i), got)
            assert np.array_equal(got, want[i]), i
            assert not np.array_equal(got, start[i])


@pytest.mark.parametrize("prec", ["f16s", "bf16s"])
def test_batch_stochastic_run_to_steady_matches_single_runs(mods, prec):
    """Run to steady state with the stochastic storages (the chunks replay one
    graph, the seeds advance on the device): per case the same stopping step,
    reason, residual and Nusselt numbers as the case run alone."""
    _, _, lbm = mods
    cases = [dict(nx=24, ny=24, n=0.8, Da=1e-2, Ra=1e3, Pr=6.2, porosity=0.6),
             dict(nx=40, ny=36, n=1.0, Da=1e-1, Ra=1e4, Pr=6.2, porosity=0.6)]
    with lbm.Batch(cases, prec=prec, clamp_mode=1, resid_interval=200) as b:
        steps, res, why = b.run_to_steady(1e-8, 40_000, graph_mode=1)
        hot, cold = b.nusselt()
    for i, c in enumerate(cases):
        with lbm.Cavity(c["nx"], c["ny"], c["n"], c["Da"], c["Ra"], c["Pr"], c["porosity"], prec=prec,
                        clamp_mode=1, resid_interval=200) as cav:
            s1, r1, w1 = cav.run_to_steady(1e-8, 40_000)
            h1, c1, _ = cav.nusselt()
        assert (steps[i], why[i]) == (s1, w1), (i, steps, why, s1, w1)
        assert res[i] == r1 and hot[i] == h1 and cold[i] == c1
