"""The step kernel with its inputs staged in shared memory by bulk
asynchronous copies (lbm_opts.staging = 2) against the register path
(staging = 1) and the oracle.

Both kernels run the same per-node arithmetic on the same values (only the
route of the loads differs), so their states must agree bit for bit after
many steps, for every storage, tau scheme and Darcy-field mode, on grids
whose rows end inside a tile, span several tiles, or have no interior rows.
The staged kernel also meets the FP32 oracle tolerance of
test_parity_gpu.py on its own."""
import numpy as np
import pytest

from test_parity_gpu import CASES, W5, W9, oracle_for, rel_err

pytestmark = pytest.mark.gpu

SIZES = [(17, 13), (130, 67), (300, 20), (520, 9), (1000, 5), (64, 2), (2, 40), (320, 37)]


@pytest.fixture(scope="module")
def mods():
    import oracle
    from paper_2011_15073_gb300 import inputs, lbm
    oracle.build()
    lbm.lib()
    return oracle, inputs, lbm


def run(lbm, state, nx, ny, c, prec, staging, tau_iters, Da, steps):
    with lbm.Cavity(nx, ny, c["n"], c["Da"], c["Ra"], c["Pr"], c["porosity"], prec=prec, clamp_mode=c["clamp_mode"],
                    porous_model=c["porous_model"], staging=staging, tau_iters=tau_iters) as cav:
        if Da is not None:
            cav.set_darcy_field(Da)
        cav.set_state_f64(*state)
        cav.step(steps)
        cav.synchronize()
        return cav.get_state_f64()


@pytest.mark.parametrize("prec", ["f32", "f32d", "bf16d", "f16d", "f16s", "bf16s"])
@pytest.mark.parametrize("tau_iters", [0, 2])
@pytest.mark.parametrize("field", [False, True], ids=["uniform", "field"])
@pytest.mark.parametrize("size", SIZES, ids=lambda s: f"{s[0]}x{s[1]}")
def test_staged_equals_register_path(mods, prec, tau_iters, field, size):
    oracle, inputs, lbm = mods
    nx, ny = size
    c = dict(CASES["thinning"], clamp_mode=1)
    ref = oracle_for(oracle, nx, ny, c)
    state = inputs.perturbed_state(ref.get_state(), seed=nx + 7 * ny, amp=1e-2)
    Da = inputs.darcy_field(5, nx, ny) if field else None
    a = run(lbm, state, nx, ny, c, prec, 1, tau_iters, Da, 40)
    for staging in [2]:   # bulk copies to shared memory
        b = run(lbm, state, nx, ny, c, prec, staging, tau_iters, Da, 40)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), staging
        if tau_iters == 0:
            assert np.array_equal(a[2], b[2]), staging
    assert not np.array_equal(a[0], state[0])


@pytest.mark.parametrize("tau_iters", [0, 2])
@pytest.mark.parametrize("case", ["thinning", "thickening"])
def test_staged_fp32_oracle_parity(mods, case, tau_iters):
    oracle, inputs, lbm = mods
    nx, ny = 300, 67
    c = dict(CASES[case], clamp_mode=1)
    ref = oracle.Cavity.from_params(nx, ny, c["n"], c["Da"], c["Ra"], c["Pr"], porosity=c["porosity"],
                                    porous_model=c["porous_model"], clamp_mode=1, tau_iters=tau_iters)
    state = [a.astype(np.float32).astype(np.float64) for a in inputs.perturbed_state(ref.get_state(), seed=23)]
    ref.set_state(*state)
    ref.step(100)
    f_r, g_r, _ = ref.get_state()
    f, g, _ = run(lbm, state, nx, ny, c, "f32", 2, tau_iters, None, 100)
    assert rel_err(f, f_r, W9) < 5e-5
    assert rel_err(g, g_r, W5) < 5e-5
