"""Replayed step graphs (lbm_opts.graph_steps): lbm_step on small grids
replays a captured CUDA graph of an even number of step launches.  The
graph holds the same kernels with the same arguments, so a run must be bit
for bit the run of one launch per step, whatever the layout, storage, step
count (remainders, odd starts) and after the Darcy field changes (which
drops and recaptures the graphs)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASE = dict(n=0.7, Da=1e-2, Ra=1e5, Pr=6.2, porosity=0.6, clamp_mode=1)


@pytest.fixture(scope="module")
def mods():
    from paper_2011_15073_gb300 import inputs, lbm
    lbm.lib()
    return inputs, lbm


def run(lbm, inputs, nx, ny, prec, layout, graph_steps, chunks, Da=None, Da2=None):
    with lbm.Cavity(nx, ny, CASE["n"], CASE["Da"], CASE["Ra"], CASE["Pr"], CASE["porosity"], prec=prec,
                    layout=layout, clamp_mode=CASE["clamp_mode"], graph_steps=graph_steps) as cav:
        cav.set_state_f64(*inputs.perturbed_state(cav.get_state_f64(), seed=nx + ny, amp=1e-2))
        if Da is not None:
            cav.set_darcy_field(Da)
        for i, k in enumerate(chunks):
            if Da2 is not None and i == len(chunks) // 2:
                cav.set_darcy_field(Da2)
            cav.step(k)
        return cav.get_state_f64()


@pytest.mark.parametrize("layout", [0, 1], ids=["ab", "aa"])
@pytest.mark.parametrize("prec", ["f64", "f32d", "f16d"])
@pytest.mark.parametrize("graph_steps", [0, 16, 7])
def test_graph_replay_equals_plain_launches(mods, layout, prec, graph_steps):
    inputs, lbm = mods
    nx, ny = 130, 67
    chunks = [1, 200, 63, 3, 128]   # odd starts, remainders, several replays
    a = run(lbm, inputs, nx, ny, prec, layout, -1, chunks)
    b = run(lbm, inputs, nx, ny, prec, layout, graph_steps, chunks)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_graph_recaptured_after_darcy_field_change(mods):
    inputs, lbm = mods
    nx, ny = 96, 40
    Da = inputs.darcy_field(3, nx, ny)
    Da2 = inputs.darcy_field(4, nx, ny)
    chunks = [128, 128, 128, 128]
    a = run(lbm, inputs, nx, ny, "f32d", 0, -1, chunks, Da, Da2)
    b = run(lbm, inputs, nx, ny, "f32d", 0, 32, chunks, Da, Da2)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("prec,staging", [("f16s", 0), ("bf16s", 0), ("f16s", 3), ("bf16s", 3)])
@pytest.mark.parametrize("graph_steps", [0, 16])
def test_graph_replay_with_stochastic_rounding(mods, prec, staging, graph_steps):
    """The stochastic-rounding storages in replayed step graphs: each
    captured launch computes its seed on the device from the step count the
    replay starts at, so the states equal one launch per step bit for bit
    (two- and four-node kernels; the start state is copied in natively,
    since an import rounds with address-dependent bits)."""
    inputs, lbm = mods
    nx, ny = 130, 67
    chunks = [1, 200, 63, 3, 128]
    kw = dict(prec=prec, clamp_mode=CASE["clamp_mode"], staging=staging)
    with lbm.Cavity(nx, ny, CASE["n"], CASE["Da"], CASE["Ra"], CASE["Pr"], CASE["porosity"], graph_steps=-1,
                    **kw) as a:
        a.set_state_f64(*inputs.perturbed_state(a.get_state_f64(), seed=nx + ny, amp=1e-2))
        start = np.empty(a.state_bytes(), np.uint8)
        a.get_state(start)
        for k in chunks:
            a.step(k)
        want = np.empty_like(start)
        a.get_state(want)
    with lbm.Cavity(nx, ny, CASE["n"], CASE["Da"], CASE["Ra"], CASE["Pr"], CASE["porosity"],
                    graph_steps=graph_steps, **kw) as b:
        b.set_state(start)
        for k in chunks:
            b.step(k)
        got = np.empty_like(start)
        b.get_state(got)
    assert np.array_equal(got, want)
    assert not np.array_equal(got, start)
