"""The four-nodes-per-thread step kernel of the 16-bit storages
(lbm_opts.staging = 3) against the two-node kernel (staging = 1) and the
oracle.

Wherever both kernels take their packed path (two-node kernel: a warp of 64
nodes whose nodes and neighbours are all interior; four-node kernel: a warp
of 128 nodes inside an interior row, the side-wall node itself excepted,
which it updates again with the wall rules) they run the same packed
arithmetic on the same values and draw the same random bits.  Elsewhere a kernel updates its nodes one at a
time with the wall rules: scalar arithmetic, which the compiler may contract
into other fused multiply-adds (the relaxation time can differ in its last
bits), and other random bits for the stochastic-rounding storages.  So, one
step from the same stored state:

* at every node where both kernels take the same path, the stored 16-bit
  codes and the relaxation times agree bit for bit;
* at the other nodes both kernels round nearly the same FP32 value (RN) or
  the same value with other random bits (SR), so the codes differ by at most
  one, and the relaxation times by a few FP32 units in the last place.

The four-node kernel also meets the deviation-storage tolerances of
test_parity_gpu.py against the oracle on its own over 100 steps.
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


def cavity(lbm, nx, ny, c, prec, staging, tau_iters=0):
    return lbm.Cavity(nx, ny, c["n"], c["Da"], c["Ra"], c["Pr"], c["porosity"], prec=prec,
                      clamp_mode=c["clamp_mode"], porous_model=c["porous_model"], staging=staging,
                      tau_iters=tau_iters)


def fast_path(nx, ny, span):
    """Nodes that a kernel with warps of `span` nodes updates on its packed
    path (warps start at multiples of span along each row).  Two-node
    kernel (span 64): warps whose nodes and neighbours are all interior.
    Four-node kernel (span 128): every warp that lies inside an interior
    row, except the side-wall nodes themselves."""
    x = np.arange(nx)
    wx = x - x % span
    if span == 64:
        fx = (wx > 0) & (wx + span < nx)
    else:
        fx = (wx + span <= nx) & (x > 0) & (x < nx - 1)
    y = np.arange(ny)
    fy = (y > 0) & (y < ny - 1)
    return fy[:, None] & fx[None, :]


def native_planes(cav, nx, ny):
    buf = np.empty(cav.state_bytes(), dtype=np.uint8)
    cav.get_state(buf)
    n = nx * ny
    codes = buf[:14 * n * 2].view(np.uint16).reshape(14, ny, nx)
    tau = buf[14 * n * 2:].view(np.float32).reshape(ny, nx)
    return buf, codes, tau


def ordinal(codes):
    """Sign-magnitude 16-bit codes (FP16, BF16) -> integers in the order of
    the values they encode, +0 and -0 both 0: adjacent values differ by 1."""
    c = codes.astype(np.int32)
    return np.where(c < 0x8000, c, 0x8000 - c)


@pytest.mark.parametrize("prec", ["bf16d", "f16d", "f16s", "bf16s"])
@pytest.mark.parametrize("tau_iters", [0, 2])
@pytest.mark.parametrize("field", [False, True], ids=["uniform", "field"])
@pytest.mark.parametrize("size", SIZES, ids=lambda s: f"{s[0]}x{s[1]}")
def test_four_node_one_step_equals_two_node(mods, prec, tau_iters, field, size):
    oracle, inputs, lbm = mods
    nx, ny = size
    c = dict(CASES["thinning"], clamp_mode=1)
    state = inputs.perturbed_state(oracle_for(oracle, nx, ny, c).get_state(), seed=nx + 3 * ny, amp=1e-2)
    Da = inputs.darcy_field(3, nx, ny) if field else None
    with cavity(lbm, nx, ny, c, prec, 1, tau_iters) as a, cavity(lbm, nx, ny, c, prec, 3, tau_iters) as b:
        if Da is not None:
            a.set_darcy_field(Da)
            b.set_darcy_field(Da)
        a.set_state_f64(*state)          # rounded once, then copied byte for byte
        raw, c0, _ = native_planes(a, nx, ny)
        b.set_state(raw)
        a.step(1)
        b.step(1)
        _, ca, ta = native_planes(a, nx, ny)
        _, cb, tb = native_planes(b, nx, ny)
    same = fast_path(nx, ny, 64) == fast_path(nx, ny, 128)
    assert np.array_equal(ca[:, same], cb[:, same])
    assert np.array_equal(ta[same], tb[same])
    d = np.abs(ordinal(ca) - ordinal(cb))
    assert d.max() <= 1, d.max()
    assert np.all(np.abs(ta - tb) <= 1e-6 * np.abs(ta))
    assert not np.array_equal(ca, c0)
    if prec in ("f16s", "bf16s") and not same.all():   # other random bits round some values the other way
        assert d[:, ~same].any()


@pytest.mark.parametrize("tau_iters", [0, 2])
@pytest.mark.parametrize("prec,tol_f,tol_g", [("bf16d", 2e-3, 2e-2), ("f16d", 2e-4, 2.5e-3),
                                              ("bf16s", 4e-3, 4e-2), ("f16s", 4e-4, 5e-3)])
def test_four_node_oracle_parity(mods, prec, tol_f, tol_g, tau_iters):
    oracle, inputs, lbm = mods
    nx, ny = 520, 67
    c = dict(CASES["thinning"], clamp_mode=1)
    ref = oracle.Cavity.from_params(nx, ny, c["n"], c["Da"], c["Ra"], c["Pr"], porosity=c["porosity"],
                                    porous_model=c["porous_model"], clamp_mode=1, tau_iters=tau_iters)
    state = inputs.perturbed_state(ref.get_state(), seed=12)
    ref.set_state(*state)
    ref.step(99)
    f99_r, g99_r, _ = ref.get_state()
    gam_r = ref.fields()["gamma"]
    ref.step(1)
    f_r, g_r, t_r = ref.get_state()
    with cavity(lbm, nx, ny, c, prec, 3, tau_iters) as cav:
        cav.set_state_f64(*state)
        cav.step(99)
        f99, g99, _ = cav.get_state_f64()
        cav.step(1)
        f, g, tau = cav.get_state_f64()
        nu = cav.fields()["nu"]
    assert rel_err(f, f_r, W9) < tol_f
    assert rel_err(g, g_r, W5) < tol_g
    df = max(np.abs(f99 - f99_r).max(), np.abs(g99 - g99_r).max())
    if tau_iters == 0:
        check_tau(tau, t_r, gam_r, ref.lat, prec, df)
    else:   # no stored tau: the viscosity of the last collision, node by node
        fr = ref.fields()
        check_tau(3 * nu + 0.5, 3 * fr["nu"] + 0.5, fr["gamma"], ref.lat, prec,
                  max(np.abs(f - f_r).max(), np.abs(g - g_r).max()))


def test_four_node_mode_is_refused_where_not_built(mods):
    _, _, lbm = mods
    c = dict(CASES["thinning"], clamp_mode=1)
    for prec, kw in [("f32d", {}), ("f32", {}), ("f64", {}), ("f32d", {"tau_iters": 2})]:
        with pytest.raises(lbm.LBMError) as e:
            lbm.Cavity(64, 64, c["n"], c["Da"], c["Ra"], c["Pr"], c["porosity"], prec=prec, staging=3, **kw)
        assert e.value.code == -7   # LBM_ERR_UNSUPPORTED
