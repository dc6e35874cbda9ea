"""CPU pins of the PyTorch restatement of the oracle (oracle/torch_step.py).

* Its forward step equals the C oracle's (same states to round-off), with a
  uniform and with a per-node Darcy field, for the literal and the
  continuous power law.
* Its reverse-mode gradients of the hot-wall Nusselt number with respect to
  the per-node Darcy field, n and Ra equal central differences of the C
  oracle (FP64).
* The same for the node-local implicit tau: node-by-node solve, whole runs
  and gradients against the C oracle with the same Newton steps.  (Checked
  once by planted mistakes, not committed: the Newton factor without
  (Phi - 1/2)/Phi, the exponent J for 1/J and R without the s8 row each fail;
  dropping the upper threshold gamma2 from the slope test changes nothing,
  since no lattice strain rate reaches gamma* = 1e6.)
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def c_run(orc, nx, ny, n, Ra, Da_field, steps, seed, clamp_mode, Pr=6.2):
    from paper_2011_15073_gb300 import inputs
    c = orc.Cavity.from_params(nx, ny, n, 1e-2, Ra, Pr, clamp_mode=clamp_mode)
    if Da_field is not None:
        c.set_darcy_field(Da_field)
    c.set_state(*inputs.perturbed_state(c.get_state(), seed=seed, amp=1e-2))
    c.step(steps)
    return c


def t_run(nx, ny, n, Ra, Da_field, steps, seed, clamp_mode, Pr=6.2):
    from oracle import torch_step as ts
    from paper_2011_15073_gb300 import inputs
    Da = torch.tensor(Da_field) if Da_field is not None else 1e-2
    p = ts.Params(nx, ny, n, Ra, Da, Pr, clamp_mode=clamp_mode)
    f0, g0, t0 = ts.rest_state(p)
    dF, dG = inputs.perturbation(seed, nx, ny, 1e-2)
    f, g, tau = ts.step(f0 * (1 + torch.tensor(dF)), g0 * (1 + torch.tensor(dG)), t0, p, steps)
    return p, f, g, tau


@pytest.mark.parametrize("clamp_mode", [0, 1])
@pytest.mark.parametrize("field", [False, True])
def test_torch_step_equals_c_oracle(orc, clamp_mode, field):
    nx, ny = 13, 11
    Da = np.exp(np.random.default_rng(1).uniform(np.log(1e-3), np.log(1e-1), (ny, nx))) if field else None
    c = c_run(orc, nx, ny, 0.7, 1e5, Da, 25, 4, clamp_mode)
    p, f, g, tau = t_run(nx, ny, 0.7, 1e5, Da, 25, 4, clamp_mode)
    fc, gc, tc = c.get_state()
    np.testing.assert_allclose(f.numpy(), fc, rtol=1e-12, atol=0)
    np.testing.assert_allclose(g.numpy(), gc, rtol=1e-12, atol=0)
    np.testing.assert_allclose(tau.numpy(), tc, rtol=1e-10, atol=0)
    from oracle import torch_step as ts
    assert float(ts.nusselt_hot(g, p)) == pytest.approx(c.nusselt()[0], rel=1e-12)


def test_torch_gradients_equal_c_oracle_differences(orc):
    from oracle import torch_step as ts
    from paper_2011_15073_gb300 import inputs
    nx, ny, steps, seed = 12, 10, 30, 9
    Da0 = np.exp(np.random.default_rng(2).uniform(np.log(1e-3), np.log(1e-1), (ny, nx)))
    n0, Ra0 = 0.8, 1e4
    Da = torch.tensor(Da0, requires_grad=True)
    n = torch.tensor(n0, dtype=torch.float64, requires_grad=True)
    Ra = torch.tensor(Ra0, dtype=torch.float64, requires_grad=True)
    p = ts.Params(nx, ny, n, Ra, Da, 6.2, clamp_mode=1)
    f0, g0, t0 = ts.rest_state(p)
    dF, dG = inputs.perturbation(seed, nx, ny, 1e-2)
    f, g, tau = ts.step(f0 * (1 + torch.tensor(dF)), g0 * (1 + torch.tensor(dG)), t0, p, steps)
    J = ts.nusselt_hot(g, p)
    J.backward()

    def J_c(n_, Ra_, Da_):
        c = orc.Cavity.from_params(nx, ny, n_, 1e-2, Ra_, 6.2, clamp_mode=1)
        c.set_darcy_field(Da_)
        c.set_state(*inputs.perturbed_state(c.get_state(), seed=seed, amp=1e-2))
        c.step(steps)
        return c.nusselt()[0]

    # central differences, relative steps
    h = 1e-5
    dn = (J_c(n0 * (1 + h), Ra0, Da0) - J_c(n0 * (1 - h), Ra0, Da0)) / (2 * h * n0)
    dRa = (J_c(n0, Ra0 * (1 + h), Da0) - J_c(n0, Ra0 * (1 - h), Da0)) / (2 * h * Ra0)
    assert float(n.grad) == pytest.approx(dn, rel=1e-5, abs=1e-9)
    assert float(Ra.grad) == pytest.approx(dRa, rel=1e-5, abs=1e-12)
    for (j, i) in [(0, 0), (3, 1), (5, 6), (9, 11), (4, 4)]:
        Dp, Dm = Da0.copy(), Da0.copy()
        Dp[j, i] *= 1 + h
        Dm[j, i] *= 1 - h
        d = (J_c(n0, Ra0, Dp) - J_c(n0, Ra0, Dm)) / (2 * h * Da0[j, i])
        g_ad = float(Da.grad[j, i])
        assert g_ad == pytest.approx(d, rel=1e-4, abs=1e-6 * max(1.0, abs(d))), (j, i)


def c_run_implicit(orc, nx, ny, n, Ra, Da_field, steps, seed, clamp_mode, tau_iters, Pr=6.2):
    from paper_2011_15073_gb300 import inputs
    c = orc.Cavity.from_params(nx, ny, n, 1e-2, Ra, Pr, clamp_mode=clamp_mode, tau_iters=tau_iters)
    if Da_field is not None:
        c.set_darcy_field(Da_field)
    c.set_state(*inputs.perturbed_state(c.get_state(), seed=seed, amp=1e-2))
    c.step(steps)
    return c


@pytest.mark.parametrize("n,clamp_mode,field", [(0.6, 1, True), (0.6, 0, False), (1.4, 1, False), (1.0, 0, True)])
def test_torch_implicit_tau_step_equals_c_oracle(orc, n, clamp_mode, field):
    """The node-local implicit tau (three Newton steps on ln tau per
    collision) restated with whole-grid operations gives the C oracle's
    states."""
    from oracle import torch_step as ts
    from paper_2011_15073_gb300 import inputs
    nx, ny, steps, seed, iters = 13, 11, 25, 6, 3
    Da = np.exp(np.random.default_rng(3).uniform(np.log(1e-3), np.log(1e-1), (ny, nx))) if field else None
    c = c_run_implicit(orc, nx, ny, n, 1e5, Da, steps, seed, clamp_mode, iters)
    p = ts.Params(nx, ny, n, 1e5, torch.tensor(Da) if field else 1e-2, 6.2, clamp_mode=clamp_mode,
                  tau_iters=iters)
    f0, g0, t0 = ts.rest_state(p)
    dF, dG = inputs.perturbation(seed, nx, ny, 1e-2)
    f, g, _ = ts.step(f0 * (1 + torch.tensor(dF)), g0 * (1 + torch.tensor(dG)), t0, p, steps)
    fc, gc, _ = c.get_state()
    np.testing.assert_allclose(f.numpy(), fc, rtol=1e-12, atol=0)
    np.testing.assert_allclose(g.numpy(), gc, rtol=1e-12, atol=0)
    assert float(ts.nusselt_hot(g, p)) == pytest.approx(c.nusselt()[0], rel=1e-12)


def test_torch_implicit_tau_equals_c_node_solve(orc):
    """Node by node, the whole-grid implicit solve equals the C oracle's
    orc_implicit_tau on the streamed populations of a developed state."""
    from oracle import torch_step as ts
    from paper_2011_15073_gb300 import inputs
    nx, ny, iters = 12, 9, 4
    lat = orc.map_params(nx, ny, 0.6, 1e-2, 1e5, 6.2, clamp_mode=1, tau_iters=iters)
    c = orc.Cavity(lat)
    c.set_state(*inputs.perturbed_state(c.get_state(), seed=8, amp=3e-2))
    c.step(40)
    f, g, _ = c.get_state()
    p = ts.Params(nx, ny, 0.6, 1e5, 1e-2, 6.2, clamp_mode=1, tau_iters=iters)
    fs, gs = ts.stream(torch.tensor(f), torch.tensor(g), p)
    tau_t = ts.implicit_tau(fs, gs, p, iters).numpy()
    fsn, gsn = fs.numpy(), gs.numpy()
    for j in range(ny):
        for i in range(nx):
            tc = orc.implicit_tau(lat, fsn[:, j, i].copy(), gsn[:, j, i].copy())
            assert tau_t[j, i] == pytest.approx(tc, rel=1e-13), (j, i)


def test_torch_implicit_tau_gradients_equal_c_oracle_differences(orc):
    """Reverse-mode gradients through the implicit tau (autograd through the
    Newton steps as computed) equal central differences of the C oracle run
    with the same number of Newton steps."""
    from oracle import torch_step as ts
    from paper_2011_15073_gb300 import inputs
    nx, ny, steps, seed, iters = 12, 10, 30, 9, 2
    Da0 = np.exp(np.random.default_rng(2).uniform(np.log(1e-3), np.log(1e-1), (ny, nx)))
    n0, Ra0 = 0.8, 1e4
    Da = torch.tensor(Da0, requires_grad=True)
    n = torch.tensor(n0, dtype=torch.float64, requires_grad=True)
    Ra = torch.tensor(Ra0, dtype=torch.float64, requires_grad=True)
    p = ts.Params(nx, ny, n, Ra, Da, 6.2, clamp_mode=1, tau_iters=iters)
    f0, g0, t0 = ts.rest_state(p)
    dF, dG = inputs.perturbation(seed, nx, ny, 1e-2)
    f, g, _ = ts.step(f0 * (1 + torch.tensor(dF)), g0 * (1 + torch.tensor(dG)), t0, p, steps)
    J = ts.nusselt_hot(g, p)
    J.backward()

    def J_c(n_, Ra_, Da_):
        c = orc.Cavity.from_params(nx, ny, n_, 1e-2, Ra_, 6.2, clamp_mode=1, tau_iters=iters)
        c.set_darcy_field(Da_)
        c.set_state(*inputs.perturbed_state(c.get_state(), seed=seed, amp=1e-2))
        c.step(steps)
        return c.nusselt()[0]

    h = 1e-5
    dn = (J_c(n0 * (1 + h), Ra0, Da0) - J_c(n0 * (1 - h), Ra0, Da0)) / (2 * h * n0)
    dRa = (J_c(n0, Ra0 * (1 + h), Da0) - J_c(n0, Ra0 * (1 - h), Da0)) / (2 * h * Ra0)
    assert float(n.grad) == pytest.approx(dn, rel=1e-5, abs=1e-9)
    assert float(Ra.grad) == pytest.approx(dRa, rel=1e-5, abs=1e-12)
    for (j, i) in [(0, 0), (3, 1), (5, 6), (9, 11)]:
        Dp, Dm = Da0.copy(), Da0.copy()
        Dp[j, i] *= 1 + h
        Dm[j, i] *= 1 - h
        d = (J_c(n0, Ra0, Dp) - J_c(n0, Ra0, Dm)) / (2 * h * Da0[j, i])
        assert float(Da.grad[j, i]) == pytest.approx(d, rel=1e-4, abs=1e-6 * max(1.0, abs(d))), (j, i)
