"""CPU pins of the oracle's node-local implicit relaxation time.

The implicit tau of a node is the root of tau = Phi(tau), where Phi(tau) is
the modified power law (Eq. MPL) evaluated at the strain rate that the
collision computes when it starts from tau (velocity solve and s7 = s8 =
1/tau).  The oracle finds it by a fixed number of Newton steps on ln tau.
These tests fix it independently of that iteration:

* n = 1: D is identically 1, so the implicit update is the lagged one, bit
  for bit, over many steps.
* the Newton result equals the root found by bisection on
  h(y) = y - ln Phi(e^y) over a wide bracket, at nodes of a developed flow,
  and converges fast (a wrong Newton factor converges linearly at best);
* a power-law channel run with the implicit tau reaches the closed-form
  profile (the steady state does not depend on how tau is found);
* a lagged steady state of the cavity is a fixed point of the implicit step.
"""
import math

import numpy as np
import pytest

from test_oracle_pins import channel_lattice, powerlaw_profile, run_to_steady, start_from_profile

EX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
EY = [0, 0, 1, 0, -1, 1, 1, -1, -1]


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.lib()
    return oracle


def pulled(f, g, j, i):
    """Pre-collision populations of interior node (j, i): each one comes from
    the neighbour it streams from."""
    fn = np.array([f[q, j - EY[q], i - EX[q]] for q in range(9)])
    gn = np.array([g[q, j - EY[q], i - EX[q]] for q in range(5)])
    return fn, gn


def test_newtonian_implicit_equals_lagged_bitwise(orc):
    from paper_2011_15073_gb300 import inputs
    a = orc.Cavity.from_params(24, 20, 1.0, 1e-2, 1e5, 6.2, porosity=0.6)
    f, g, tau = inputs.perturbed_state(a.get_state(), seed=3, amp=1e-2)
    tau[:] = a.lat.tau0
    a.set_state(f, g, tau)
    b = orc.Cavity.from_params(24, 20, 1.0, 1e-2, 1e5, 6.2, porosity=0.6, tau_iters=3)
    b.set_state(f, g, tau)
    a.step(40)
    b.step(40)
    fa, ga, _ = a.get_state()
    fb, gb, _ = b.get_state()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    assert not np.array_equal(fa, f)


def bisect_root(orc, lat, fn, gn):
    """Root of y - ln Phi(e^y) by bisection on a bracket of ln tau."""
    lo, hi = math.log(0.5 + 1e-9), math.log(1e4)

    def h(y):
        return y - math.log(orc.phi(lat, fn, gn, math.exp(y))[0])

    assert h(lo) < 0 < h(hi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if h(mid) < 0:
            lo = mid
        else:
            hi = mid
    return math.exp(0.5 * (lo + hi))


@pytest.mark.parametrize("n,Da,Ra", [(0.6, 1e-2, 1e5), (1.4, 1e-3, 1e5), (0.6, 1e-4, 1e4)])
def test_newton_tau_is_the_bisection_root(orc, n, Da, Ra):
    N = 32
    c = orc.Cavity.from_params(N, N, n, Da, Ra, 6.2, porosity=0.6, clamp_mode=1)
    c.step(1500)
    f, g, _ = c.get_state()
    lat = c.lat.copy()
    rng = np.random.default_rng(1)
    checked = 0
    for _ in range(25):
        j, i = (int(v) for v in rng.integers(1, N - 1, 2))
        fn, gn = pulled(f, g, j, i)
        root = bisect_root(orc, lat, fn, gn)
        phi_root = orc.phi(lat, fn, gn, root)[0]
        assert abs(phi_root - root) <= 1e-12 * root
        lat.tau_iters = 0
        assert orc.implicit_tau(lat, fn, gn) == lat.tau0   # the start: rest-state tau0
        errs = []
        for K in (1, 3, 6):
            lat.tau_iters = K
            errs.append(abs(orc.implicit_tau(lat, fn, gn) - root) / root)
        assert errs[1] < 1e-8 and errs[2] < 1e-11, (j, i, errs)
        checked += 1
    assert checked == 25


@pytest.mark.parametrize("n", [0.6, 1.3])
def test_implicit_powerlaw_channel_matches_closed_form(orc, n):
    errs = []
    for ny in (32, 64):
        gam_w = 2e-3 * (32 / ny) ** 2
        lat = channel_lattice(orc, ny, n, nu_w=0.1, gam_w=gam_w)
        lat.tau_iters = 4
        y = np.arange(ny) + 0.5
        ua = powerlaw_profile(y, ny / 2, n, lat.Gx, lat.nu_ref)
        c = start_from_profile(orc, lat, ua)
        run_to_steady(c, 2000, 1e-11, 400000)
        u = c.fields()["ux"][:, 0]
        errs.append(np.linalg.norm(u - ua) / np.linalg.norm(ua))
    assert errs[1] < 1e-3, errs
    assert errs[0] / errs[1] > 3.0, errs


def test_lagged_steady_state_is_an_implicit_fixed_point(orc):
    """At a steady state of the lagged scheme each node's stored tau equals
    Phi(tau), i.e. the implicit root: one implicit step leaves the state."""
    kw = dict(porosity=0.6, clamp_mode=1)
    lag = orc.Cavity.from_params(16, 16, 0.8, 1e-2, 1e4, 6.2, **kw)
    run_to_steady(lag, 2000, 1e-13, 200000)
    f, g, tau = lag.get_state()
    imp = orc.Cavity.from_params(16, 16, 0.8, 1e-2, 1e4, 6.2, tau_iters=6, **kw)
    imp.set_state(f, g, tau)
    lag.step(1)
    imp.step(1)
    f1, g1, tau1 = lag.get_state()
    f2, g2, _ = imp.get_state()
    assert np.abs(tau1 - tau).max() <= 1e-10 * tau.max()
    assert np.abs(f2 - f1).max() <= 1e-12 and np.abs(g2 - g1).max() <= 1e-12
    nu_imp = imp.fields()["nu"]
    nu_lag = lag.fields()["nu"]
    assert np.abs(nu_imp - nu_lag).max() <= 1e-9 * nu_lag.max()
