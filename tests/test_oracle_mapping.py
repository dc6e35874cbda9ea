"""CPU pins of the oracle's lattice-unit mapping and of its per-node Darcy field.

``orc_map_params`` turns the paper's groups (n, Da, Ra, Pr, porosity) into
lattice parameters.  These tests do not re-type its formulas.  They measure
what the oracle's collision and streaming actually do -- the viscosity a node
takes at a known strain rate, the momentum one collision adds through the
buoyancy and the drag, the rate at which heat diffuses -- and check the
measured values against the paper's own definitions:

* the dimensional groups of Eq. (non_dim_var):
  Ra = g beta L^(2n+1) dT / (nu_c alpha^n),
  Pr = nu_c / (alpha^(2-n) L^(2(n-1))),  Da = K / L^2,
  with nu_c the power-law consistency (apparent viscosity nu_c |gamma|^(n-1));
* the non-dimensional equations (par_sim_*): velocity scale alpha sqrt(Ra)/L,
  viscous coefficient Pr / sqrt(Ra)^(2-n) times D of Eq. (D) on the
  non-dimensional strain rate, buoyancy Pr theta, diffusivity 1/sqrt(Ra);
* the modified power law of Eq. (MPL) for D, with gamma_1 = 0.01 and
  gamma_2 = 1e6 on the non-dimensional strain rate;
* the Ergun form of the Forchheimer factor and the porosity of the generalized
  porous model (reading R4);
* the transient conduction between the isothermal walls, a Fourier series.

The thermal diffusivity of the D2Q5 lattice is alpha = (tauT - 1/2) / 3 (its
sound speed squared is 1/3); the transient-conduction test pins that the
streaming and collision really diffuse heat at that rate.
"""
import math

import numpy as np
import pytest

E9 = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], float)
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
W5 = np.array([1 / 3] + [1 / 6] * 4)

CASES = [  # (nx, ny, n, Da, Ra, Pr, porosity, Ma)
    (64, 64, 1.0, 1e-2, 1e4, 6.2, 0.6, 0.1),
    (64, 48, 0.6, 1e-3, 1e5, 6.2, 0.6, 0.1),
    (160, 160, 0.6, 1e-2, 1e5, 100.0, 1.0, 0.1),
    (96, 96, 1.4, 1e-1, 1e3, 10.0, 0.4, 0.05),
    (128, 40, 0.8, 3e-2, 2e4, 1.0, 0.9, 0.2),
]


def textbook_M():
    ex, ey = E9[:, 0], E9[:, 1]
    e2 = ex * ex + ey * ey
    return np.array([
        np.ones(9), 3 * e2 - 4, 4.5 * e2 * e2 - 10.5 * e2 + 4, ex, (3 * e2 - 5) * ex,
        ey, (3 * e2 - 5) * ey, ex * ex - ey * ey, ex * ey])


def rest_feq(rho, u):
    """Textbook D2Q9 equilibrium at porosity 1."""
    eu = E9 @ u
    return W9 * rho * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * (u @ u))


def alpha_of(lat):
    """D2Q5 thermal diffusivity with c_s^2 = 1/3."""
    return (lat.tauT - 0.5) / 3.0


def D_mpl(gs, n, g1=0.01, g2=1e6):
    """Eq. (MPL) as printed, as a factor on nu_0."""
    if gs < g1:
        return 1.0
    if gs <= g2:
        return gs ** (n - 1)
    return g2 ** (n - 1)


def sheared_node(rho, Sab, tau_prev):
    """Populations at rest velocity whose non-equilibrium part carries the
    strain-rate tensor Sab to first Chapman-Enskog order, for the MRT rates
    of the collision (s7 = s8 = 1/tau_prev).  Mass and momentum are those of
    the rest state, so no force acts."""
    s = np.array([1.0, 1.4, 1.4, 1.0, 1.2, 1.0, 1.2, 1 / tau_prev, 1 / tau_prev])
    Q = np.einsum("ia,ib->iab", E9, E9) - np.eye(2) / 3
    src = 3 * rho * W9 * np.einsum("iab,ab->i", Q, Sab)
    Mt = textbook_M()
    fneq = -np.linalg.solve(Mt, (Mt @ src) / s)
    return rest_feq(rho, np.zeros(2)) + fneq


def measured_viscosity(orc, lat, gamma_lat, tau_prev=1.0, seed=0):
    """(apparent lattice viscosity, lattice |gamma|) of one collision of a
    node sheared at |gamma| = gamma_lat, at the mean temperature."""
    rng = np.random.default_rng(seed)
    a, b = rng.normal(size=2)
    Sab = np.array([[a, b], [b, -a]])
    Sab *= gamma_lat / math.sqrt(2 * np.sum(Sab * Sab))
    f = sheared_node(1.0, Sab, tau_prev)
    g = W5 * lat.Tm
    _, _, tau_new, gam = orc.collide_node(lat, f, g, tau_prev)
    return (tau_new - 0.5) / 3.0, gam


def momentum_gain(orc, lat, u0, T, tau_prev=1.0):
    """Momentum one collision adds to a node holding the equilibrium of
    velocity u0 at temperature T, and the node's density and momentum."""
    f = rest_feq(1.0, np.asarray(u0, float))
    g = W5 * T
    fo, _, _, _ = orc.collide_node(lat, f, g, tau_prev)
    return E9.T @ (fo - f), f.sum(), E9.T @ f


def paper_viscosity(lat_alpha, L, n, Ra, Pr, gamma_lat, clamp="literal", g1=0.01, g2=1e6):
    """Apparent lattice viscosity the non-dimensional momentum equations ask
    for at lattice strain rate gamma_lat: velocity scale U = alpha sqrt(Ra)/L,
    so the non-dimensional strain rate is gamma_lat L / U and the viscous
    coefficient Pr / sqrt(Ra)^(2-n) D multiplies U L."""
    U = lat_alpha * math.sqrt(Ra) / L
    gs = gamma_lat * L / U
    if clamp == "literal":
        D = D_mpl(gs, n, g1, g2)
    else:
        D = min(max(gs, g1), g2) ** (n - 1)
    return Pr / math.sqrt(Ra) ** (2 - n) * D * U * L, gs


# ------------------------------------------------------ viscosity and Pr, Ra
@pytest.mark.parametrize("case", CASES)
def test_mapping_gives_the_papers_groups(orc, case):
    """Measured consistency, diffusivity and buoyancy reproduce Ra and Pr of
    Eq. (non_dim_var) with the paper's power-law definitions, and the drag
    reproduces Da = K / L^2."""
    nx, ny, n, Da, Ra, Pr, eps, Ma = case
    lat = orc.map_params(nx, ny, n, Da, Ra, Pr, porosity=eps, Ma=Ma, porous_model=0)
    L = float(nx)
    alpha = alpha_of(lat)
    # consistency from a node sheared in the power-law branch (gamma* ~ 0.5)
    Uref = alpha * math.sqrt(Ra) / L
    nu_app, gam = measured_viscosity(orc, lat, 0.5 * Uref / L)
    nu_c = nu_app / gam ** (n - 1)
    # buoyancy per unit temperature difference from one collision at rest
    lat_nodrag = lat.copy()
    lat_nodrag.K = math.inf
    dj, rho, _ = momentum_gain(orc, lat_nodrag, (0.0, 0.0), 1.0)
    dj0, _, _ = momentum_gain(orc, lat_nodrag, (0.0, 0.0), 0.0)
    assert abs(dj[0]) < 1e-18 and abs(dj0[0]) < 1e-18
    gbeta_dT = (dj[1] - dj0[1]) / rho          # T from 0 to 1 = T_h - T_c
    Tm = -dj0[1] / (dj[1] - dj0[1])
    assert abs(Tm - 0.5) < 1e-12               # T_m = (T_h + T_c) / 2
    Ra_def = gbeta_dT * L ** (2 * n + 1) / (nu_c * alpha ** n)
    Pr_def = nu_c / (alpha ** (2 - n) * L ** (2 * (n - 1)))
    assert abs(Ra_def / Ra - 1) < 1e-11, (Ra_def, Ra)
    assert abs(Pr_def / Pr - 1) < 1e-11, (Pr_def, Pr)
    # buoyancy of the non-dimensional v-equation: Pr theta in units U^2 / L
    assert abs(gbeta_dT / (Pr * Uref ** 2 / L) - 1) < 1e-12
    # Darcy drag (porosity 1, no Forchheimer term): F = -nu u / K
    tau_prev = 0.9
    nu_prev = (tau_prev - 0.5) / 3
    dj, rho, j = momentum_gain(orc, lat, (0.02, -0.01), lat.Tm, tau_prev)
    F = dj / rho
    u = j / rho + F / 2
    K = -nu_prev * u / F
    assert np.allclose(K / L ** 2, Da, rtol=1e-11, atol=0), (K / L ** 2, Da)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("clamp_mode", [0, 1])
def test_apparent_viscosity_follows_the_modified_power_law(orc, case, clamp_mode):
    """Eq. (MPL) on the non-dimensional strain rate of the paper's scaling,
    across all three branches (the upper threshold is lowered so that a
    lattice population can reach it)."""
    nx, ny, n, Da, Ra, Pr, eps, Ma = case
    lat = orc.map_params(nx, ny, n, Da, Ra, Pr, porosity=eps, Ma=Ma, clamp_mode=clamp_mode)
    L = float(nx)
    alpha = alpha_of(lat)
    Uref = alpha * math.sqrt(Ra) / L
    lat.gamma2 = 3.0
    mode = "literal" if clamp_mode == 0 else "continuous"
    for k, gs_target in enumerate((1e-3, 0.009, 0.0101, 0.3, 2.9, 3.1, 7.0)):
        gamma_lat = gs_target * Uref / L
        nu_app, gam = measured_viscosity(orc, lat, gamma_lat, tau_prev=0.8, seed=k)
        assert abs(gam / gamma_lat - 1) < 1e-9
        expect, gs = paper_viscosity(alpha, L, n, Ra, Pr, gam, mode, g2=3.0)
        assert abs(gs / gs_target - 1) < 1e-9
        assert abs(nu_app / expect - 1) < 1e-11, (gs_target, nu_app, expect)


@pytest.mark.parametrize("clamp_mode", [0, 1])
@pytest.mark.parametrize("n", [0.6, 1.0, 1.4])
def test_rest_state_relaxation_time(orc, clamp_mode, n):
    """The rest state has zero strain rate: D = 1 under the printed law and
    gamma_1^(n-1) under the continuous clamp."""
    Ra, Pr, L = 1e5, 6.2, 64
    c = orc.Cavity.from_params(L, 32, n, 1e-2, Ra, Pr, clamp_mode=clamp_mode)
    tau = c.get_state()[2]
    alpha = alpha_of(c.lat)
    D0 = 1.0 if clamp_mode == 0 else 0.01 ** (n - 1)
    expect = 3 * Pr / math.sqrt(Ra) ** (2 - n) * D0 * alpha * math.sqrt(Ra) + 0.5
    assert np.all(np.abs(tau / expect - 1) < 1e-13)


# ------------------------------------------------------------ porous model
@pytest.mark.parametrize("eps", [0.3, 0.6, 0.95])
def test_generalized_porous_drag_is_darcy_plus_ergun(orc, eps):
    """porous_model 1: F = -eps nu u / K - eps F_eps |u| u / sqrt(K), with
    K = Da L^2 and the Ergun factor F_eps = 1.75 / sqrt(150 eps^3); the two
    coefficients are read off the drag at two speeds."""
    nx, Da = 48, 2e-3
    lat = orc.map_params(nx, nx, 1.0, Da, 1e4, 6.2, porosity=eps, porous_model=1)
    tau_prev = 1.1
    nu_prev = (tau_prev - 0.5) / 3
    d = np.array([0.6, 0.8])
    ratios, speeds = [], []
    for s in (0.01, 0.03):
        dj, rho, j = momentum_gain(orc, lat, s * d, lat.Tm, tau_prev)
        F = dj / rho
        u = j / rho + F / 2
        # the force is antiparallel to u
        assert abs(F[0] * u[1] - F[1] * u[0]) < 1e-15
        speeds.append(math.hypot(*u))
        ratios.append(-(F @ u) / (u @ u))
    slope = (ratios[1] - ratios[0]) / (speeds[1] - speeds[0])
    icpt = ratios[0] - slope * speeds[0]
    K = Da * nx ** 2
    assert abs(icpt / (eps * nu_prev / K) - 1) < 1e-9
    Feps = slope * math.sqrt(K) / eps
    assert abs(Feps / (1.75 / math.sqrt(150 * eps ** 3)) - 1) < 1e-9


# ------------------------------------------------------ thermal diffusivity
def conduction_series(X, t_nd, Ra, kmax=4000):
    """theta(X, t) between theta(0) = 1 and theta(1) = 0 from theta = 1/2,
    under d theta/dt = (1/sqrt(Ra)) theta_XX (non-dimensional energy
    equation without flow): 1 - X minus the even sine modes of X - 1/2."""
    kappa = 1 / math.sqrt(Ra)
    th = 1 - X
    for k in range(2, kmax, 2):
        th = th - 2 / (k * math.pi) * np.sin(k * math.pi * X) * math.exp(-(k * math.pi) ** 2 * kappa * t_nd)
    return th


@pytest.mark.parametrize("Ra,Ma", [(1e3, 0.1), (1e4, 0.2)])
def test_transient_conduction_runs_on_the_papers_clock(orc, Ra, Ma):
    """With buoyancy off the temperature obeys the non-dimensional energy
    equation; its time unit is L / U_c (U_c = Ma c_s, the lattice velocity of
    the scale alpha sqrt(Ra)/L).  Compared at two times with the series."""
    L = 48
    lat = orc.map_params(L, 2, 1.0, 1e-1, Ra, 6.2, Ma=Ma)
    lat.gbeta = 0.0
    c = orc.Cavity(lat)
    Uc = Ma / math.sqrt(3)
    X = (np.arange(L) + 0.5) / L
    done = 0
    for kt in (0.01, 0.04):  # diffusion lengths of 0.1 and 0.2 cavity widths
        t_nd = kt * math.sqrt(Ra)
        steps = int(round(t_nd * L / Uc))
        c.step(steps - done)
        done = steps
        T = c.fields()["T"][0]
        th = conduction_series(X, steps * Uc / L, Ra)
        assert np.abs(T - th).max() < 2e-3, np.abs(T - th).max()


# ------------------------------------------------------------ Darcy field
def test_uniform_darcy_field_equals_uniform_permeability(orc):
    from paper_2011_15073_gb300 import inputs
    nx, ny, Da = 20, 14, 3e-3
    a = orc.Cavity.from_params(nx, ny, 0.6, Da, 1e5, 6.2)
    b = orc.Cavity.from_params(nx, ny, 0.6, Da, 1e5, 6.2)
    st = inputs.perturbed_state(a.get_state(), seed=11, amp=1e-2)
    a.set_state(*st)
    b.set_state(*st)
    b.set_darcy_field(np.full((ny, nx), Da))
    a.step(40)
    b.step(40)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)


def test_darcy_field_acts_at_its_own_node(orc):
    """One step with Da(x) = Da everywhere but Da_q at node q: node q's
    collision is the one of a uniform-Da_q run, every other node's the one of
    the uniform-Da run (the drag is node-local: K(x) = Da(x) L^2)."""
    from paper_2011_15073_gb300 import inputs
    nx, ny, Da, Da_q = 16, 12, 1e-3, 5e-2
    q = (5, 7)  # (y, x)
    runs = [orc.Cavity.from_params(nx, ny, 0.8, d, 1e5, 6.2) for d in (Da, Da_q, Da)]
    st = inputs.perturbed_state(runs[0].get_state(), seed=5, amp=2e-2)
    # develop some flow first so that the drag matters
    runs[0].set_state(*st)
    runs[0].step(30)
    st = runs[0].get_state()
    for r in runs:
        r.set_state(*st)
    field = np.full((ny, nx), Da)
    field[q] = Da_q
    runs[2].set_darcy_field(field)
    for r in runs:
        r.step(1)
    s_uni, s_q, s_fld = (r.get_state() for r in runs)
    mask = np.zeros((ny, nx), bool)
    mask[q] = True
    for a, b, c in zip(s_uni, s_q, s_fld):
        assert np.array_equal(c[..., mask], b[..., mask])
        assert np.array_equal(c[..., ~mask], a[..., ~mask])
    assert not np.array_equal(s_uni[0][..., mask], s_q[0][..., mask])
