"""CPU pins of the PyTorch restatement of the oracle (oracle/torch_step.py).

* Its forward step equals the C oracle's (same states to round-off), with a
  uniform and with a per-node Darcy field, for the literal and the
  continuous power law.
* Its reverse-mode gradients of the hot-wall Nusselt number with respect to
  the per-node Darcy field, n and Ra equal central differences of the C
  oracle (FP64).
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
