"""GPU parity of the node-local implicit relaxation time (lbm_opts.tau_iters).

The oracle runs the same number of Newton steps on ln tau from tau0 per
collision (``oracle.c``, pinned on the CPU by ``test_oracle_implicit.py``).
Tolerances follow ``test_parity_gpu.py``: the implicit solve only changes
where the collision's tau comes from, and each Newton step is a smooth
function of the node's populations (away from the literal law's jump at
gamma_1), so FP64 stays within the stated 1e-12 relative on f and g and FP32
within 5e-5 of the population scale after 100 steps; the viscosity of the
next collision is checked node by node with ``check_tau``.
"""
import numpy as np
import pytest

from parity_util import check_tau
from test_parity_gpu import CASES, W5, W9, oracle_for, rel_err

pytestmark = pytest.mark.gpu

LAYOUTS = pytest.mark.parametrize("layout", [0, 1], ids=["ab", "aa"])
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


@pytest.fixture(scope="module")
def mods():
    import oracle
    from paper_2011_15073_gb300 import inputs, lbm
    oracle.build()
    lbm.lib()
    return oracle, inputs, lbm


def implicit_oracle(oracle, nx, ny, c, K):
    return oracle.Cavity.from_params(nx, ny, c["n"], c["Da"], c["Ra"], c["Pr"], porosity=c["porosity"],
                                     porous_model=c["porous_model"], clamp_mode=c["clamp_mode"], tau_iters=K)


def implicit_gpu(lbm, nx, ny, c, prec, K, layout=0):
    return lbm.Cavity(nx, ny, c["n"], c["Da"], c["Ra"], c["Pr"], c["porosity"], prec=prec,
                      porous_model=c["porous_model"], clamp_mode=c["clamp_mode"], layout=layout, tau_iters=K)


@LAYOUTS
@pytest.mark.parametrize("K", [1, 4])
@pytest.mark.parametrize("case", ["thinning", "darcy", "thickening"])
@pytest.mark.parametrize("size", [(17, 13), (64, 64), (130, 67), (3, 70)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_fp64_implicit_step_parity(mods, case, size, K, layout):
    oracle, inputs, lbm = mods
    nx, ny = size
    c = CASES[case]
    ref = implicit_oracle(oracle, nx, ny, c, K)
    state = inputs.perturbed_state(ref.get_state(), seed=nx * 100 + ny + K)
    ref.set_state(*state)
    ref.step(100)
    f_r, g_r, _ = ref.get_state()
    fr = ref.fields()
    h_r, c_r, _ = ref.nusselt()
    with implicit_gpu(lbm, nx, ny, c, "f64", K, layout) as cav:
        cav.set_state_f64(*state)
        cav.step(100)
        f, g, _ = cav.get_state_f64()
        fl = cav.fields()
        hot, cold = cav.nusselt()[:2]
    assert np.max(np.abs(f - f_r) / np.abs(f_r)) < 1e-12
    assert np.max(np.abs(g - g_r) / np.abs(g_r)) < 1e-12
    assert abs(hot - h_r) <= 1e-10 * abs(h_r) and abs(cold - c_r) <= 1e-10 * abs(c_r)
    df = max(np.abs(f - f_r).max(), np.abs(g - g_r).max())
    check_tau(3 * fl["nu"] + 0.5, 3 * fr["nu"] + 0.5, fr["gamma"], ref.lat, "f64", df)
    for k in ("ux", "uy"):
        assert np.max(np.abs(fl[k] - fr[k])) <= 1e-12, k


@LAYOUTS
@pytest.mark.parametrize("prec", ["f32", "f32d"])
@pytest.mark.parametrize("case", ["thinning", "darcy", "thickening"])
@pytest.mark.parametrize("size", [(17, 13), (130, 67)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_fp32_implicit_step_parity(mods, case, size, layout, prec):
    oracle, inputs, lbm = mods
    nx, ny = size
    c = dict(CASES[case], clamp_mode=1)
    ref = implicit_oracle(oracle, nx, ny, c, 2)
    state = [a.astype(np.float32).astype(np.float64) for a in
             inputs.perturbed_state(ref.get_state(), seed=17 + nx)]
    ref.set_state(*state)
    ref.step(100)
    f_r, g_r, _ = ref.get_state()
    fr = ref.fields()
    with implicit_gpu(lbm, nx, ny, c, prec, 2, layout) as cav:
        cav.set_state_f64(*state)
        cav.step(100)
        f, g, _ = cav.get_state_f64()
        fl = cav.fields()
        hot = cav.nusselt()[0]
    assert rel_err(f, f_r, W9) < 5e-5
    assert rel_err(g, g_r, W5) < 5e-5
    df = max(np.abs(f - f_r).max(), np.abs(g - g_r).max())
    check_tau(3 * fl["nu"] + 0.5, 3 * fr["nu"] + 0.5, fr["gamma"], ref.lat, prec, df)
    h_r = ref.nusselt()[0]
    assert abs(hot - h_r) <= 1e-4 * abs(h_r)


@LAYOUTS
def test_exported_tau_is_the_next_implicit_tau(mods, layout):
    """In implicit mode the state's tau is the tau each node's next collision
    starts from: at interior nodes, the oracle's Newton solve on the pulled
    populations."""
    oracle, inputs, lbm = mods
    nx, ny, K = 40, 30, 3
    c = CASES["thinning"]
    ref = implicit_oracle(oracle, nx, ny, c, K)
    state = inputs.perturbed_state(ref.get_state(), seed=9)
    ref.set_state(*state)
    ref.step(30)
    f_r, g_r, _ = ref.get_state()
    with implicit_gpu(lbm, nx, ny, c, "f64", K, layout) as cav:
        cav.set_state_f64(*state)
        cav.step(30)
        _, _, tau = cav.get_state_f64()
    lat = ref.lat.copy()
    worst = 0.0
    for j in range(1, ny - 1):
        for i in range(1, nx - 1):
            fn = f_r[np.arange(9), j - EY, i - EX]
            gn = g_r[np.arange(5), j - EY[:5], i - EX[:5]]
            t = oracle.implicit_tau(lat, fn, gn)
            worst = max(worst, abs(tau[j, i] - t) / t)
    assert worst < 1e-10


def test_newtonian_implicit_equals_lagged(mods):
    """n = 1: D is 1 at every strain rate, so both ways of finding tau give
    tau0 and the same run."""
    _, inputs, lbm = mods
    c = dict(CASES["newtonian"])
    runs = []
    for K in (0, 3):
        with implicit_gpu(lbm, 64, 48, c, "f64", K) as cav:
            f, g, tau = cav.get_state_f64()
            cav.set_state_f64(*inputs.perturbed_state((f, g, tau), seed=4))
            cav.step(200)
            runs.append(cav.get_state_f64()[:2])
    for a, b in zip(*runs):
        assert np.max(np.abs(a - b) / np.abs(b)) < 1e-13


def test_implicit_mode_is_refused_where_not_built(mods):
    _, _, lbm = mods
    with implicit_gpu(lbm, 16, 16, CASES["darcy"], "f64", 2) as cav:
        with pytest.raises(lbm.LBMError) as e:
            cav.adjoint_nu(10, ckpt_every=5)
        assert e.value.code == -7   # LBM_ERR_UNSUPPORTED
