"""The four-nodes-per-thread step kernel of the 16-bit storages
(lbm_opts.staging = 3) against the two-node kernel (staging = 1) and the
oracle.

Wherever both kernels take their fast path (a warp whose nodes and their
neighbours are all interior: 64 nodes for the two-node kernel, 128 for the
four-node one) they run the same arithmetic on the same values and draw the
same random bits; elsewhere a kernel updates its nodes one at a time with the
wall rules, which computes the same FP32 values but draws other random bits.
So:

* round-to-nearest storages (BF16D, F16D): the states agree bit for bit after
  many steps, for both Darcy-field modes;
* stochastic rounding (F16S, BF16S), one step from the same stored state: the
  stored 16-bit codes agree at every node where both kernels take the same
  path; at the other nodes both round the same FP32 value to one of its two
  neighbours, so the codes differ by at most one; the relaxation times (not
  rounded) agree everywhere.

The four-node kernel also meets the deviation-storage tolerances of
test_parity_gpu.py against the oracle on its own.
"""
import numpy as np
import pytest

from parity_util import check_tau
from test_parity_gpu import CASES, W5, W9, oracle_for, rel_err

pytestmark = pytest.mark.gpu

SIZES = [(17, 13), (300, 20), (520, 9), (1000, 5), (700, 33), (1030, 17), (64, 2), (2, 40), (260, 3)]


@pytest.fixture(scope="module")
def mods():
    import oracle
    from paper_2011_15073_gb300 import inputs, lbm
    oracle.build()
    lbm.lib()
    return oracle, inputs, lbm


def cavity(lbm, nx, ny, c, prec, staging):
    return lbm.Cavity(nx, ny, c["n"], c["Da"], c["Ra"], c["Pr"], c["porosity"], prec=prec,
                      clamp_mode=c["clamp_mode"], porous_model=c["porous_model"], staging=staging)


def fast_path(nx, ny, span):
    """Nodes that a kernel with warps of `span` nodes updates on its fast
    path (warps start at multiples of span along each row)."""
    x = np.arange(nx)
    wx = x - x % span
    fx = (wx > 0) & (wx + span < nx)
    y = np.arange(ny)
    fy = (y > 0) & (y < ny - 1)
    return fy[:, None] & fx[None, :]


@pytest.mark.parametrize("prec", ["bf16d", "f16d"])
@pytest.mark.parametrize("field", [False, True], ids=["uniform", "field"])
@pytest.mark.parametrize("size", SIZES, ids=lambda s: f"{s[0]}x{s[1]}")
def test_four_node_equals_two_node_round_to_nearest(mods, prec, field, size):
    oracle, inputs, lbm = mods
    nx, ny = size
    c = dict(CASES["thinning"], clamp_mode=1)
    state = inputs.perturbed_state(oracle_for(oracle, nx, ny, c).get_state(), seed=nx + 5 * ny, amp=1e-2)
    Da = inputs.darcy_field(3, nx, ny) if field else None
    out = []
    for staging in (1, 3):
        with cavity(lbm, nx, ny, c, prec, staging) as cav:
            if Da is not None:
                cav.set_darcy_field(Da)
            cav.set_state_f64(*state)
            cav.step(40)
            out.append(cav.get_state_f64())
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    assert not np.array_equal(out[0][0], state[0])


def native_planes(cav, nx, ny, code_dtype):
    buf = np.empty(cav.state_bytes(), dtype=np.uint8)
    cav.get_state(buf)
    n = nx * ny
    codes = buf[:14 * n * 2].view(code_dtype).reshape(14, ny, nx)
    tau = buf[14 * n * 2:].view(np.float32).reshape(ny, nx)
    return buf, codes, tau


@pytest.mark.parametrize("prec", ["f16s", "bf16s"])
@pytest.mark.parametrize("size", SIZES, ids=lambda s: f"{s[0]}x{s[1]}")
def test_four_node_one_step_stochastic_rounding(mods, prec, size):
    oracle, inputs, lbm = mods
    nx, ny = size
    c = dict(CASES["thinning"], clamp_mode=1)
    state = inputs.perturbed_state(oracle_for(oracle, nx, ny, c).get_state(), seed=nx + 3 * ny, amp=1e-2)
    with cavity(lbm, nx, ny, c, prec, 1) as a, cavity(lbm, nx, ny, c, prec, 3) as b:
        a.set_state_f64(*state)          # rounded once (address-seeded), then copied byte for byte
        raw, _, _ = native_planes(a, nx, ny, np.uint16)
        b.set_state(raw)
        a.step(1)
        b.step(1)
        _, ca, ta = native_planes(a, nx, ny, np.uint16)
        _, cb, tb = native_planes(b, nx, ny, np.uint16)
    assert np.array_equal(ta, tb)
    same = fast_path(nx, ny, 64) == fast_path(nx, ny, 128)
    assert np.array_equal(ca[:, same], cb[:, same])
    d = np.abs(ca.astype(np.int32) - cb.astype(np.int32))
    assert d.max() <= 1, d.max()
    if not same.all():   # the other random bits do round some values the other way
        assert d[:, ~same].any()


@pytest.mark.parametrize("prec,tol_f,tol_g", [("bf16d", 2e-3, 2e-2), ("f16d", 2e-4, 2.5e-3),
                                              ("bf16s", 4e-3, 4e-2), ("f16s", 4e-4, 5e-3)])
def test_four_node_oracle_parity(mods, prec, tol_f, tol_g):
    oracle, inputs, lbm = mods
    nx, ny = 520, 67
    c = dict(CASES["thinning"], clamp_mode=1)
    ref = oracle_for(oracle, nx, ny, c)
    state = inputs.perturbed_state(ref.get_state(), seed=12)
    ref.set_state(*state)
    ref.step(99)
    f99_r, g99_r, _ = ref.get_state()
    gam_r = ref.fields()["gamma"]
    ref.step(1)
    f_r, g_r, t_r = ref.get_state()
    with cavity(lbm, nx, ny, c, prec, 3) as cav:
        cav.set_state_f64(*state)
        cav.step(99)
        f99, g99, _ = cav.get_state_f64()
        cav.step(1)
        f, g, tau = cav.get_state_f64()
    assert rel_err(f, f_r, W9) < tol_f
    assert rel_err(g, g_r, W5) < tol_g
    df = max(np.abs(f99 - f99_r).max(), np.abs(g99 - g99_r).max())
    check_tau(tau, t_r, gam_r, ref.lat, prec, df)


def test_four_node_mode_is_refused_where_not_built(mods):
    _, _, lbm = mods
    c = dict(CASES["thinning"], clamp_mode=1)
    for prec, kw in [("f32d", {}), ("f32", {}), ("f16s", {"tau_iters": 2})]:
        with pytest.raises(lbm.LBMError) as e:
            lbm.Cavity(64, 64, c["n"], c["Da"], c["Ra"], c["Pr"], c["porosity"], prec=prec, staging=3, **kw)
        assert e.value.code == -7   # LBM_ERR_UNSUPPORTED
