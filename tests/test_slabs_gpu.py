"""Row-slab decomposition on one GPU: several slab contexts exchanging their
cut populations by device buffers after every step must compute exactly
what the undivided cavity computes.

The pull scheme makes every interior node's update a function of the
previous state of its neighbours only; a slab gets the neighbours across a
cut through its ghost row, so with the same tile code (FP64 one node per
thread, FP32 two nodes per thread; the fast-path decision is made on the
same rows) the states are bit-identical.  The Nusselt number and the
residual are sums over rows, added up in another order: equal to rounding.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASE = dict(n=0.6, Da=1e-2, Ra=1e5, Pr=6.2, porosity=0.6)


@pytest.fixture(scope="module")
def mods():
    import oracle
    from paper_2011_15073_gb300 import inputs, lbm, slabs
    oracle.build()
    lbm.lib()
    return oracle, inputs, lbm, slabs


@pytest.mark.parametrize("prec", ["f64", "f32d", "f32"])
@pytest.mark.parametrize("nx,ny,parts", [(64, 50, 2), (130, 67, 3), (40, 9, 4), (33, 20, 1)])
def test_slabs_equal_the_undivided_cavity(mods, prec, nx, ny, parts):
    oracle, inputs, lbm, slabs = mods
    import torch
    rest = oracle.Cavity.from_params(nx, ny, CASE["n"], CASE["Da"], CASE["Ra"], CASE["Pr"],
                                     porosity=CASE["porosity"], clamp_mode=1)
    state = inputs.perturbed_state(rest.get_state(), seed=nx + ny, amp=1e-2)
    with lbm.Cavity(nx, ny, prec=prec, clamp_mode=1, graph_steps=-1, **CASE) as cav:
        cav.set_state_f64(*state)
        cav.residual()
        cav.step(100)
        want = cav.get_state_f64()
        nu_w = cav.nusselt()
        r_w = cav.residual()
    with slabs.SlabRun(nx, ny, parts, prec=prec, clamp_mode=1, stream=torch.cuda.Stream(), **CASE) as run:
        run.set_state_f64(*state)
        run.residual()
        run.step(100)
        got = run.get_state_f64()
        nu_g = run.nusselt()
        r_g = run.residual()
    for a, w in zip(got, want):
        assert np.array_equal(a, w)
    assert nu_g[0] == pytest.approx(nu_w[0], rel=1e-13) and nu_g[1] == pytest.approx(nu_w[1], rel=1e-13)
    assert r_g == pytest.approx(r_w, rel=1e-10)


def test_slab_calls_refused_where_they_cannot_apply(mods):
    _, _, lbm, _ = mods
    import torch
    buf = torch.empty(1 << 16, dtype=torch.uint8, device="cuda:0")
    bottom = lbm.init_slab(32, 40, 0, 20, **CASE)
    middle = lbm.init_slab(32, 40, 10, 30, **CASE)
    try:
        assert lbm.slab_rows(bottom) == (0, 0, 20, 21)
        assert lbm.slab_rows(middle) == (10, 1, 21, 22)
        assert lbm.halo_bytes(bottom) == 4 * 32 * 8
        with pytest.raises(lbm.LBMError) as e:      # no neighbour below the bottom slab
            lbm.halo_pack(bottom, buf.data_ptr(), None)
        assert e.value.code == -1
        with pytest.raises(lbm.LBMError) as e:      # ghost rows need an exchange every step
            lbm.run_to_steady(middle, 1e-8, 1000)
        assert e.value.code == -7
        with pytest.raises(lbm.LBMError):
            lbm.init_slab(32, 40, 30, 20, **CASE)
    finally:
        lbm.destroy(bottom)
        lbm.destroy(middle)
