"""Discrete adjoint of the hot-wall Nusselt number (lbm_adjoint_nu).

* FP64 GPU adjoint against the reverse-mode gradient of the FP64 PyTorch
  restatement of the oracle (oracle/torch_step.py, pinned to the C oracle on
  the CPU): dJ/dDa(x) at every node, dJ/dn and dJ/dRa, from a fixed perturbed
  state and from the rest state (whose tau_0 depends on n and Ra).
* FP64 GPU adjoint against central differences of the FP64 GPU forward run
  (h = 1e-4 relative in log Da; truncation O(h^2) ~ 1e-8, rounding
  1e-14 / 1e-4 = 1e-10, so 1e-5 relative is a safe bound).
* FP32 adjoint against the FP64 one (the FP32 run's gradient carries the
  FP32 trajectory's rounding: 1e-2 relative on the aggregate gradients).
* The same gradients, bit for bit, whatever the checkpoint segmentation.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASE = dict(n=0.8, Ra=1e4, Pr=6.2, porosity=0.6)


@pytest.fixture(scope="module")
def mods():
    from paper_2011_15073_gb300 import inputs, lbm
    lbm.lib()
    return inputs, lbm


def torch_grad(nx, ny, Da, steps, state, clamp_mode):
    from oracle import torch_step as ts
    Dt = torch.tensor(Da, requires_grad=True)
    n = torch.tensor(CASE["n"], dtype=torch.float64, requires_grad=True)
    Ra = torch.tensor(CASE["Ra"], dtype=torch.float64, requires_grad=True)
    p = ts.Params(nx, ny, n, Ra, Dt, CASE["Pr"], porosity=CASE["porosity"], clamp_mode=clamp_mode)
    if state is None:
        f, g, tau = ts.rest_state(p)
    else:
        f, g, tau = [torch.tensor(a) for a in state]
    f, g, tau = ts.step(f, g, tau, p, steps)
    J = ts.nusselt_hot(g, p)
    J.backward()
    return float(J.detach()), Dt.grad.numpy(), float(n.grad), float(Ra.grad)


@pytest.mark.parametrize("clamp_mode", [1, 0])
@pytest.mark.parametrize("from_rest", [False, True])
def test_fp64_adjoint_equals_torch_oracle_gradient(mods, clamp_mode, from_rest):
    inputs, lbm = mods
    import oracle
    nx, ny, steps = 24, 20, 160
    Da = inputs.darcy_field(7, nx, ny)
    state = None
    if not from_rest:
        ref = oracle.Cavity.from_params(nx, ny, CASE["n"], 1e-2, CASE["Ra"], CASE["Pr"], porosity=CASE["porosity"],
                                        clamp_mode=clamp_mode)
        state = inputs.perturbed_state(ref.get_state(), seed=5, amp=1e-2)
    J_t, dDa_t, dn_t, dRa_t = torch_grad(nx, ny, Da, steps, state, clamp_mode)
    with lbm.Cavity(nx, ny, CASE["n"], 1e-2, CASE["Ra"], CASE["Pr"], CASE["porosity"], prec="f64",
                    clamp_mode=clamp_mode) as cav:
        cav.set_darcy_field(Da)
        if state is not None:
            cav.set_state_f64(*state)
        J, dDa, dn, dRa, peak = cav.adjoint_nu(steps, ckpt_every=50, from_rest=from_rest)
    assert J == pytest.approx(J_t, rel=1e-12)
    scale = np.abs(dDa_t).max()
    assert scale > 0
    assert np.max(np.abs(dDa - dDa_t)) <= 1e-8 * scale
    assert dn == pytest.approx(dn_t, rel=1e-8, abs=1e-12)
    assert dRa == pytest.approx(dRa_t, rel=1e-8, abs=1e-16)
    assert peak > 0


def test_fp64_adjoint_equals_central_differences(mods):
    inputs, lbm = mods
    nx, ny, steps = 40, 32, 600
    Da = inputs.darcy_field(11, nx, ny)

    def J_of(D, n=CASE["n"], Ra=CASE["Ra"]):
        with lbm.Cavity(nx, ny, n, 1e-2, Ra, CASE["Pr"], CASE["porosity"], prec="f64", clamp_mode=1) as c:
            c.set_darcy_field(D)
            c.step(steps)
            return c.nusselt()[0]

    with lbm.Cavity(nx, ny, CASE["n"], 1e-2, CASE["Ra"], CASE["Pr"], CASE["porosity"], prec="f64",
                    clamp_mode=1) as cav:
        cav.set_darcy_field(Da)
        J, dDa, dn, dRa, _ = cav.adjoint_nu(steps, ckpt_every=100, from_rest=True)
    assert J == pytest.approx(J_of(Da), rel=1e-13)
    h = 1e-4
    rng = np.random.default_rng(3)
    for _ in range(6):
        j, i = int(rng.integers(0, ny)), int(rng.integers(0, nx))
        Dp, Dm = Da.copy(), Da.copy()
        Dp[j, i] *= np.exp(h)
        Dm[j, i] *= np.exp(-h)
        fd = (J_of(Dp) - J_of(Dm)) / (2 * h)          # dJ/dlog Da
        ad = dDa[j, i] * Da[j, i]
        assert ad == pytest.approx(fd, rel=1e-5, abs=1e-9 * max(1.0, abs(J))), (j, i)
    fdn = (J_of(Da, n=CASE["n"] * (1 + h)) - J_of(Da, n=CASE["n"] * (1 - h))) / (2 * h * CASE["n"])
    assert dn == pytest.approx(fdn, rel=1e-5)
    fdR = (J_of(Da, Ra=CASE["Ra"] * (1 + h)) - J_of(Da, Ra=CASE["Ra"] * (1 - h))) / (2 * h * CASE["Ra"])
    assert dRa == pytest.approx(fdR, rel=1e-5)


def test_fp32_adjoint_close_to_fp64(mods):
    inputs, lbm = mods
    nx, ny, steps = 64, 64, 500
    Da = inputs.darcy_field(13, nx, ny)
    out = {}
    for prec in ("f64", "f32"):
        with lbm.Cavity(nx, ny, CASE["n"], 1e-2, CASE["Ra"], CASE["Pr"], CASE["porosity"], prec=prec,
                        clamp_mode=1) as cav:
            cav.set_darcy_field(Da)
            out[prec] = cav.adjoint_nu(steps, ckpt_every=100, from_rest=True)
    J64, d64, n64, R64, _ = out["f64"]
    J32, d32, n32, R32, _ = out["f32"]
    assert J32 == pytest.approx(J64, rel=1e-4)
    assert np.linalg.norm(d32 - d64) <= 1e-2 * np.linalg.norm(d64)
    assert n32 == pytest.approx(n64, rel=1e-2)
    assert R32 == pytest.approx(R64, rel=1e-2)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_adjoint_is_independent_of_the_segmentation(mods, prec):
    """The reverse sweep recomputes each checkpoint segment on a second
    stream while the reverse steps of the following segment run.  The
    kernels and their inputs do not depend on how the run is cut, so every
    segmentation must give the same J and gradients bit for bit: one segment
    (nothing recomputed beside the reverse steps), even segments (replayed
    stage graphs), odd ones (both adjoint-buffer parities) with a shorter
    last segment, and segments of two steps."""
    inputs, lbm = mods
    nx, ny, steps = 48, 40, 230
    Da = inputs.darcy_field(19, nx, ny)
    out = []
    for ckpt in (230, 50, 7, 2):
        with lbm.Cavity(nx, ny, CASE["n"], 1e-2, CASE["Ra"], CASE["Pr"], CASE["porosity"], prec=prec,
                        clamp_mode=1) as cav:
            cav.set_darcy_field(Da)
            out.append(cav.adjoint_nu(steps, ckpt_every=ckpt, from_rest=True))
    J0, d0, n0, R0, peak0 = out[0]
    assert np.abs(d0).max() > 0
    for J, dDa, dn, dRa, peak in out[1:]:
        assert J == J0 and dn == n0 and dRa == R0
        assert np.array_equal(dDa, d0)
        assert peak > 0


def test_autograd_function_carries_the_adjoint(mods):
    """hot_wall_nusselt's gradients through torch.autograd equal the C call's,
    and a directional central difference of its value (FP64)."""
    inputs, lbm = mods
    from paper_2011_15073_gb300.autograd import hot_wall_nusselt
    nx, ny, steps = 40, 32, 400
    Da = torch.tensor(inputs.darcy_field(17, nx, ny), dtype=torch.float64, requires_grad=True)
    n = torch.tensor(CASE["n"], dtype=torch.float64, requires_grad=True)
    Ra = torch.tensor(CASE["Ra"], dtype=torch.float64, requires_grad=True)
    kw = dict(Pr=CASE["Pr"], porosity=CASE["porosity"], steps=steps, ckpt_every=100, prec="f64", clamp_mode=1)
    J = hot_wall_nusselt(Da, n, Ra, **kw)
    (2.0 * J).backward()
    with lbm.Cavity(nx, ny, CASE["n"], 1e-2, CASE["Ra"], CASE["Pr"], CASE["porosity"], prec="f64",
                    clamp_mode=1) as cav:
        cav.set_darcy_field(Da.detach().numpy())
        J0, dDa, dn, dRa, _ = cav.adjoint_nu(steps, ckpt_every=100, from_rest=True)
    assert float(J.detach()) == J0
    assert np.array_equal(Da.grad.numpy(), 2.0 * dDa)
    assert float(n.grad) == 2.0 * dn and float(Ra.grad) == 2.0 * dRa
    # direction in log Da
    rng = np.random.default_rng(5)
    v = torch.tensor(rng.standard_normal((ny, nx)), dtype=torch.float64)
    h = 1e-4
    with torch.no_grad():
        Jp = hot_wall_nusselt(Da * torch.exp(h * v), n, Ra, **kw)
        Jm = hot_wall_nusselt(Da * torch.exp(-h * v), n, Ra, **kw)
    fd = float(Jp - Jm) / (2 * h)
    ad = float((Da.grad / 2.0 * Da.detach() * v).sum())
    assert ad == pytest.approx(fd, rel=1e-5)
