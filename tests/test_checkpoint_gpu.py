"""Checkpoint / resume (lbm_checkpoint_save / lbm_checkpoint_load).

A run saved after k steps and resumed in a new context must continue exactly
as the saved run does after its save: the native state bytes agree bit for
bit after further steps, for FP64, FP32-deviation and both stochastic
16-bit storages (whose random bits depend on the restored step count), in
both layouts.  A blob of another run, a truncated one or one with a broken
header is refused.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASE = dict(n=0.6, Da=1e-2, Ra=1e5, Pr=6.2, porosity=0.6)


@pytest.fixture(scope="module")
def mods():
    import oracle
    from paper_2011_15073_gb300 import inputs, lbm
    oracle.build()
    lbm.lib()
    return oracle, inputs, lbm


def _native(cav):
    buf = np.empty(cav.state_bytes(), dtype=np.uint8)
    cav.get_state(buf)
    return buf


@pytest.mark.parametrize("layout", [0, 1], ids=["ab", "aa"])
@pytest.mark.parametrize("prec", ["f64", "f32d", "f16s", "bf16s"])
def test_resumed_run_continues_bit_for_bit(mods, prec, layout):
    oracle, inputs, lbm = mods
    nx, ny = 70, 45
    rest = oracle.Cavity.from_params(nx, ny, CASE["n"], CASE["Da"], CASE["Ra"], CASE["Pr"],
                                     porosity=CASE["porosity"], clamp_mode=1)
    state = inputs.perturbed_state(rest.get_state(), seed=17, amp=1e-2)
    opts = dict(prec=prec, layout=layout, clamp_mode=1, seed=3)
    with lbm.Cavity(nx, ny, **CASE, **opts) as a:
        a.set_state_f64(*state)
        a.step(37)                       # odd: the in-place layout is in its odd-step form here
        blob = a.checkpoint()
        a.step(41)
        want = _native(a)
    with lbm.Cavity(nx, ny, **CASE, **opts) as b:
        b.restore(blob)
        b.step(41)
        got = _native(b)
    assert np.array_equal(got, want)


def test_foreign_or_damaged_checkpoints_are_refused(mods):
    _, _, lbm = mods
    with lbm.Cavity(40, 30, prec="f32d", **CASE) as a:
        a.step(5)
        blob = a.checkpoint()
    with lbm.Cavity(40, 30, prec="f32d", **dict(CASE, Ra=1e4)) as other:   # another Rayleigh number
        with pytest.raises(lbm.LBMError) as e:
            other.restore(blob)
        assert e.value.code == -1
    with lbm.Cavity(40, 30, prec="f32d", **CASE) as same:
        with pytest.raises(lbm.LBMError):
            same.restore(blob[:-8])            # truncated
        bad = bytearray(blob)
        bad[0] ^= 0xFF                         # broken magic
        with pytest.raises(lbm.LBMError):
            same.restore(bytes(bad))
        same.restore(blob)                     # the intact one loads
