"""No kernel writes outside the rows of a state plane.

Every plane row is padded to a multiple of 64 elements and the buffers are
zero-filled at creation; after stepping (every storage, both layouts, both
tau schemes, the per-node Darcy field, the two-node and four-node kernels),
the reductions, the state export and the in-place normalisation, the
batched sweep and the row-slab exchange, the padding must still read zero
(lbm_debug_padding_canary).  A substitute for an out-of-bounds checker:
the widths below leave padding (130 -> pitch 192, 260 -> 320, 75 -> 128).
"""
import pytest

pytestmark = pytest.mark.gpu

CASE = dict(n=0.6, Da=1e-2, Ra=1e5, Pr=6.2, porosity=0.6, clamp_mode=1)

VARIANTS = [
    dict(prec="f64"), dict(prec="f64", layout=1), dict(prec="f64", tau_iters=4),
    dict(prec="f32"), dict(prec="f32d"), dict(prec="f32d", layout=1), dict(prec="f32d", tau_iters=2),
    dict(prec="bf16d", staging=1), dict(prec="bf16d", staging=3), dict(prec="f16d", staging=3),
    dict(prec="f16s", staging=1), dict(prec="f16s", staging=3), dict(prec="f16s", staging=3, tau_iters=2),
    dict(prec="bf16s", staging=3), dict(prec="f16s", layout=1),
]


@pytest.fixture(scope="module")
def mods():
    from paper_2011_15073_gb300 import inputs, lbm
    lbm.lib()
    return inputs, lbm


@pytest.mark.parametrize("field", [False, True], ids=["uniform", "field"])
@pytest.mark.parametrize("opts", VARIANTS, ids=lambda o: "-".join(f"{k}{v}" for k, v in o.items()))
@pytest.mark.parametrize("size", [(130, 67), (260, 9), (75, 40)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_padding_stays_untouched(mods, size, opts, field):
    inputs, lbm = mods
    nx, ny = size
    with lbm.Cavity(nx, ny, **CASE, **opts) as cav:
        if field:
            cav.set_darcy_field(inputs.darcy_field(7, nx, ny))
        cav.step(25)
        cav.fields()
        cav.nusselt(local=True)
        cav.residual()
        cav.step(3)
        cav.get_state_f64()
        cav.residual()
        assert lbm.debug_padding_canary(cav.ctx) == 0


@pytest.mark.parametrize("plan", [("per_step", 64, 4), ("persistent", 128, 2)])
def test_padding_untouched_by_the_batch(mods, plan):
    _, lbm = mods
    cases = [dict(nx=130, ny=30, n=0.8, Da=1e-2, Ra=1e4, Pr=6.2, porosity=0.6),
             dict(nx=75, ny=40, n=1.0, Da=1e-1, Ra=1e3, Pr=6.2, porosity=0.6)]
    with lbm.Batch(cases, prec="f32d", clamp_mode=1, resid_interval=100) as b:
        b.set_plan(*plan)
        b.step(21)
        b.run_to_steady(1e-12, 400, graph_mode=1)
        for i in range(len(cases)):
            assert lbm.debug_padding_canary(b.case_ctx(i)) == 0


def test_padding_untouched_by_the_slab_exchange(mods):
    _, lbm = mods
    from paper_2011_15073_gb300 import slabs
    with slabs.SlabRun(130, 50, 3, prec="f32d", **CASE) as run:
        run.step(20)
        run.nusselt()
        run.residual()
        for s in run.slabs:
            assert lbm.debug_padding_canary(s.ctx) == 0
