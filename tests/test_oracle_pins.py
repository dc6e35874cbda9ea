"""CPU pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks one part of ``oracle/oracle.c`` against an independent
statement of it: the textbook polynomial definition of the MRT basis, the
defining moments of the equilibrium and of the body-force term, the single
relaxation-time (BGK) special case, the Chapman-Enskog strain rate, exact
conservation laws, and closed-form or independently integrated steady flows.
None of them re-types the oracle's own formula.
"""
import math

import numpy as np
import pytest

E9 = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], float)
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
E5 = E9[:5]
W5 = np.array([1 / 3] + [1 / 6] * 4)


def textbook_M():
    """Lallemand & Luo (2000) D2Q9 basis as polynomials of the velocities,
    rows (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy)."""
    ex, ey = E9[:, 0], E9[:, 1]
    e2 = ex * ex + ey * ey
    return np.array([
        np.ones(9), 3 * e2 - 4, 4.5 * e2 * e2 - 10.5 * e2 + 4, ex, (3 * e2 - 5) * ex,
        ey, (3 * e2 - 5) * ey, ex * ex - ey * ey, ex * ey])


def textbook_N():
    ex, ey = E5[:, 0], E5[:, 1]
    e2 = ex * ex + ey * ey
    return np.array([np.ones(5), ex, ey, 5 * e2 - 4, ex * ex - ey * ey])


def gz_feq(rho, u, eps):
    """Generalized (porous) equilibrium, Guo & Zhao, Phys. Rev. E 66, 036304 (2002)."""
    eu = E9 @ u
    return W9 * rho * (1 + 3 * eu + 4.5 * eu ** 2 / eps - 1.5 * (u @ u) / eps)


def gz_force(rho, u, F, eps, tau):
    """Guo-Zhao body-force term including its (1 - 1/(2 tau)) factor."""
    eu = E9 @ u
    eF = E9 @ F
    return W9 * rho * (1 - 0.5 / tau) * (3 * eF + 9 * eu * eF / eps - 3 * (u @ F) / eps)


# ------------------------------------------------------------------ matrices
def test_M_rows_are_the_lallemand_luo_polynomials(orc):
    M, Mi, N, Ni = orc.matrices()
    np.testing.assert_array_equal(M, textbook_M())
    np.testing.assert_array_equal(N, textbook_N())


def test_transform_orthogonality_and_inverse(orc):
    M, Mi, N, Ni = orc.matrices()
    np.testing.assert_array_equal(M @ M.T, np.diag([9, 36, 36, 6, 12, 6, 12, 4, 4]))
    np.testing.assert_array_equal(N @ N.T, np.diag([5, 2, 2, 20, 4]))
    assert np.abs(M @ Mi - np.eye(9)).max() < 1e-15
    assert np.abs(Mi @ M - np.eye(9)).max() < 1e-15
    assert np.abs(N @ Ni - np.eye(5)).max() < 1e-15
    # independent inverse from LAPACK
    assert np.abs(Mi - np.linalg.inv(textbook_M())).max() < 1e-15


# -------------------------------------------------------------- equilibrium
@pytest.mark.parametrize("seed", range(5))
def test_feq_defining_moments(orc, seed):
    rng = np.random.default_rng(seed)
    rho, eps = rng.uniform(0.8, 1.2), rng.uniform(0.3, 1.0)
    u = rng.uniform(-0.1, 0.1, 2)
    f = orc.feq(rho, u[0], u[1], eps)
    assert abs(f.sum() - rho) < 1e-15
    np.testing.assert_allclose(E9.T @ f, rho * u, atol=1e-16)
    Pi = np.einsum("i,ia,ib->ab", f, E9, E9)
    np.testing.assert_allclose(Pi, rho * (np.eye(2) / 3 + np.outer(u, u) / eps), atol=2e-16)


@pytest.mark.parametrize("seed", range(5))
def test_meq_is_projection_of_velocity_space_feq(orc, seed):
    rng = np.random.default_rng(100 + seed)
    rho, eps = rng.uniform(0.8, 1.2), rng.uniform(0.3, 1.0)
    u = rng.uniform(-0.1, 0.1, 2)
    np.testing.assert_allclose(orc.meq(rho, u[0], u[1], eps), textbook_M() @ gz_feq(rho, u, eps),
                               atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_forcing_defining_moments(orc, seed):
    rng = np.random.default_rng(200 + seed)
    rho, eps = rng.uniform(0.8, 1.2), rng.uniform(0.3, 1.0)
    u = rng.uniform(-0.1, 0.1, 2)
    F = rng.uniform(-1e-3, 1e-3, 2)
    Fi = orc.forcing_vel(rho, u[0], u[1], F[0], F[1], eps)
    assert abs(Fi.sum()) < 1e-18
    np.testing.assert_allclose(E9.T @ Fi, rho * F, atol=1e-18)
    Pi = np.einsum("i,ia,ib->ab", Fi, E9, E9)
    np.testing.assert_allclose(Pi, rho * (np.outer(u, F) + np.outer(F, u)) / eps, atol=1e-18)


# ------------------------------------------------------------ collision pins
def base_lattice(orc, **over):
    lat = orc.map_params(8, 8, 1.0, 1e-2, 1e4, 6.2)
    for k, v in over.items():
        if k == "s":
            for i, sv in enumerate(v):
                lat.s[i] = sv
        else:
            setattr(lat, k, v)
    return lat


def solve_velocity(j, rho, G, nu, eps, K, Feps):
    """u from rho u = sum f e + rho F(u) / 2 with the porous force
    F(u) = -eps nu u / K - eps Feps |u| u / sqrt K + eps G (Newton iteration)."""
    u = j / rho
    for _ in range(60):
        um = math.hypot(*u)
        F = -eps * nu * u / K - eps * Feps * um * u / math.sqrt(K) + eps * G
        r = u - j / rho - 0.5 * F
        # Jacobian of r
        J = np.eye(2) * (1 + 0.5 * eps * nu / K + 0.5 * eps * Feps * um / math.sqrt(K))
        if um > 0:
            J += 0.5 * eps * Feps / math.sqrt(K) * np.outer(u, u) / um
        u = u - np.linalg.solve(J, r)
    return u


@pytest.mark.parametrize("seed", range(6))
def test_mrt_reduces_to_bgk_with_porous_forcing(orc, seed):
    """With every flow rate equal to 1/tau and both free thermal rates equal
    to 1/tauT, the MRT collisions must be the BGK collisions with the
    Guo-Zhao force and the D2Q5 BGK with g^eq = w T (1 + 3 e.u)."""
    rng = np.random.default_rng(300 + seed)
    eps = rng.uniform(0.4, 1.0)
    Kl = rng.uniform(5.0, 50.0)
    lat0 = base_lattice(orc, n=1.0, eps=eps, K=Kl, Feps=1.75 / math.sqrt(150 * eps ** 3),
                        gbeta=rng.uniform(1e-4, 1e-3), Gx=rng.uniform(-1e-4, 1e-4))
    tau = 3 * lat0.nu_ref + 0.5
    tauT = lat0.tauT
    lat = base_lattice(orc, n=1.0, eps=lat0.eps, K=lat0.K, Feps=lat0.Feps, gbeta=lat0.gbeta,
                       Gx=lat0.Gx, s=[1 / tau] * 7 + [0, 0], s_e=1 / tauT, s_p=1 / tauT)
    rho = rng.uniform(0.95, 1.05)
    u0 = rng.uniform(-0.05, 0.05, 2)
    f = gz_feq(rho, u0, eps) * (1 + rng.uniform(-0.02, 0.02, 9))
    T0 = rng.uniform(0.2, 0.8)
    g = W5 * T0 * (1 + rng.uniform(-0.05, 0.05, 5))
    fo, go, tn, _ = orc.collide_node(lat, f, g, tau)
    assert abs(tn - tau) < 1e-15
    rho = f.sum()
    j = E9.T @ f
    T = g.sum()
    G = np.array([lat.Gx, lat.gbeta * (T - lat.Tm)])
    nu = (tau - 0.5) / 3
    u = solve_velocity(j, rho, G, nu, eps, lat.K, lat.Feps)
    um = math.hypot(*u)
    F = -eps * nu * u / lat.K - eps * lat.Feps * um * u / math.sqrt(lat.K) + eps * G
    f_bgk = f - (f - gz_feq(rho, u, eps)) / tau + gz_force(rho, u, F, eps, tau)
    geq = W5 * T * (1 + 3 * (E5 @ u))
    g_bgk = g - (g - geq) / tauT
    np.testing.assert_allclose(fo, f_bgk, rtol=0, atol=2e-15)
    np.testing.assert_allclose(go, g_bgk, rtol=0, atol=2e-15)


@pytest.mark.parametrize("seed", range(4))
def test_conserved_moment_rates_do_not_matter(orc, seed):
    """s0, s3, s5 act on conserved moments; with the half-force velocity the
    result cannot depend on them."""
    rng = np.random.default_rng(400 + seed)
    lat_a = orc.map_params(32, 32, 0.6, 1e-2, 1e5, 6.2)
    lat_b = lat_a.copy()
    lat_b.s[0], lat_b.s[3], lat_b.s[5] = 0.7, 1.6, 1.9
    f = W9 * (1 + rng.uniform(-0.05, 0.05, 9))
    g = W5 * 0.5 * (1 + rng.uniform(-0.05, 0.05, 5))
    tau_prev = lat_a.tau0 * rng.uniform(0.9, 1.1)
    ra = orc.collide_node(lat_a, f, g, tau_prev)
    rb = orc.collide_node(lat_b, f, g, tau_prev)
    np.testing.assert_allclose(ra[0], rb[0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(ra[1], rb[1], rtol=0, atol=1e-15)
    assert abs(ra[2] - rb[2]) < 1e-13 and abs(ra[3] - rb[3]) < 1e-15


@pytest.mark.parametrize("seed", range(6))
def test_strain_rate_recovers_chapman_enskog_shear(orc, seed):
    """First-order Chapman-Enskog: f^neq = -M^-1 S^-1 M (3 rho w_i Q_i : S_ab)
    gives back gamma_ab = S_ab, so |gamma| = sqrt(2 S:S)."""
    rng = np.random.default_rng(500 + seed)
    rho = rng.uniform(0.9, 1.1)
    u = rng.uniform(-0.05, 0.05, 2)
    a, b, c = rng.uniform(-1e-3, 1e-3, 3)
    if seed < 3:
        c = 0.0  # traceless shear
    Sab = np.array([[a + c, b], [b, -a + c]])
    lat = base_lattice(orc, n=1.0, K=math.inf, Feps=0.0, gbeta=0.0, Gx=0.0, eps=1.0)
    tau_prev = rng.uniform(0.6, 2.0)
    Mt = textbook_M()
    s = np.array([1.0, 1.4, 1.4, 1.0, 1.2, 1.0, 1.2, 1 / tau_prev, 1 / tau_prev])
    Q = np.einsum("ia,ib->iab", E9, E9) - np.eye(2) / 3
    src = 3 * rho * W9 * np.einsum("iab,ab->i", Q, Sab)
    fneq = -np.linalg.solve(Mt, (Mt @ src) / s)
    f = gz_feq(rho, u, 1.0) + fneq
    _, _, _, gamma = orc.collide_node(lat, f, W5 * 0.5, tau_prev)
    expect = math.sqrt(2 * np.sum(Sab * Sab))
    assert abs(gamma - expect) < 1e-12 * expect


def test_newtonian_limit_keeps_reference_viscosity(orc):
    from paper_2011_15073_gb300 import inputs
    c = orc.Cavity.from_params(12, 10, 1.0, 1e-2, 1e5, 6.2)
    c.set_state(*inputs.perturbed_state(c.get_state(), seed=7, amp=1e-2))
    c.step(20)
    fl = c.fields()
    assert np.all(fl["nu"] == c.lat.nu_ref)
    assert np.all(c.get_state()[2] == 3 * c.lat.nu_ref + 0.5)


@pytest.mark.parametrize("n,porous", [(0.6, 1), (1.0, 0)])
def test_mass_is_conserved(orc, n, porous):
    from paper_2011_15073_gb300 import inputs
    c = orc.Cavity.from_params(24, 20, n, 1e-2, 1e5, 6.2, porous_model=porous)
    c.set_state(*inputs.perturbed_state(c.get_state(), seed=3))
    m0 = c.get_state()[0].sum()
    for _ in range(4):
        c.step(50)
        assert abs(c.get_state()[0].sum() - m0) < 1e-13 * m0


# ------------------------------------------------------------ steady states
def run_to_steady(c, chunk, tol, max_steps, key="ux"):
    prev = None
    done = 0
    while done < max_steps:
        c.step(chunk)
        done += chunk
        cur = c.fields()[key]
        if prev is not None and np.abs(cur - prev).max() <= tol * max(np.abs(cur).max(), 1e-300):
            return done
        prev = cur
    raise AssertionError("no steady state")


def test_conduction_limit_gives_unit_nusselt(orc):
    """No buoyancy: the steady temperature is linear between the isothermal
    walls and the halfway-wall difference is exact for it, so Nu = 1."""
    lat = orc.map_params(16, 16, 1.0, 1e-1, 10.0, 6.2)
    lat.gbeta = 0.0
    c = orc.Cavity(lat)
    steps = run_to_steady(c, 500, 1e-15, 40000, key="T")
    hot, cold, loc = c.nusselt()
    assert abs(hot - 1.0) < 1e-10 and abs(cold - 1.0) < 1e-10, (hot, cold, steps)
    T = c.fields()["T"]
    x = (np.arange(16) + 0.5) / 16
    np.testing.assert_allclose(T, np.broadcast_to(1 - x, T.shape), atol=1e-11)


def test_low_rayleigh_is_nearly_conductive(orc):
    c = orc.Cavity.from_params(16, 16, 1.0, 1e-1, 10.0, 6.2)
    run_to_steady(c, 500, 1e-12, 60000, key="T")
    hot, cold, _ = c.nusselt()
    assert abs(hot - 1.0) < 1e-3 and abs(cold - 1.0) < 1e-3


def channel_lattice(orc, ny, n, nu_w, gam_w, eps=1.0, K=math.inf, Feps=0.0, G=None):
    lat = base_lattice(orc)
    lat.nx, lat.ny = 2, ny
    lat.periodic_x = 1
    lat.n = n
    lat.clamp_mode = 1
    lat.gamma_scale = 1.0
    lat.gamma1 = 1e-3 * gam_w
    lat.gamma2 = 1e12
    lat.nu_ref = nu_w / gam_w ** (n - 1)      # consistency K_c
    lat.K, lat.eps, lat.Feps = K, eps, Feps
    lat.gbeta = 0.0
    h = ny / 2
    lat.Gx = lat.nu_ref * gam_w ** n / h if G is None else G
    lat.tau0 = 3 * nu_w + 0.5
    return lat


def start_from_profile(orc, lat, uprof):
    c = orc.Cavity(lat)
    f, g, tau = c.get_state()
    for j in range(lat.ny):
        f[:, j, :] = gz_feq(1.0, np.array([uprof[j], 0.0]), lat.eps)[:, None]
    c.set_state(f, g, tau)
    return c


def powerlaw_profile(y, h, n, G, Kc):
    r = np.abs(y - h)
    return n / (n + 1) * (G / Kc) ** (1 / n) * (h ** ((n + 1) / n) - r ** ((n + 1) / n))


@pytest.mark.parametrize("n", [0.6, 0.8, 1.0])
def test_powerlaw_channel_matches_closed_form(orc, n):
    errs = []
    for ny in (32, 64):
        gam_w = 2e-3 * (32 / ny) ** 2   # diffusive scaling: same tau field
        lat = channel_lattice(orc, ny, n, nu_w=0.1, gam_w=gam_w)
        y = np.arange(ny) + 0.5
        ua = powerlaw_profile(y, ny / 2, n, lat.Gx, lat.nu_ref)
        c = start_from_profile(orc, lat, ua)
        run_to_steady(c, 2000, 1e-11, 400000)
        u = c.fields()["ux"][:, 0]
        errs.append(np.linalg.norm(u - ua) / np.linalg.norm(ua))
    assert errs[1] < 1e-3, errs
    assert errs[0] / errs[1] > 3.0, errs   # second order in the grid spacing


def test_powerlaw_channel_shear_rate(orc):
    """The locally computed |gamma| follows the analytic |du/dy| across the
    channel (away from the clamped centreline)."""
    n, ny = 0.7, 64
    lat = channel_lattice(orc, ny, n, nu_w=0.1, gam_w=5e-4)
    y = np.arange(ny) + 0.5
    h = ny / 2
    ua = powerlaw_profile(y, h, n, lat.Gx, lat.nu_ref)
    c = start_from_profile(orc, lat, ua)
    run_to_steady(c, 2000, 1e-11, 400000)
    gam = c.fields()["gamma"][:, 0]
    ga = (lat.Gx * np.abs(y - h) / lat.nu_ref) ** (1 / n)
    sel = np.abs(y - h) > 4
    assert np.max(np.abs(gam[sel] - ga[sel]) / ga[sel]) < 2e-2


def test_brinkman_channel_matches_closed_form(orc):
    ny, eps = 64, 0.6
    nu = 0.1
    K = (ny / 8) ** 2
    G = 1e-6
    lat = channel_lattice(orc, ny, 1.0, nu_w=nu, gam_w=1.0, eps=eps, K=K, Feps=0.0, G=G)
    lat.nu_ref = nu
    y = np.arange(ny) + 0.5
    h = ny / 2
    r = math.sqrt(eps / K)
    ua = G * K / nu * (1 - np.cosh(r * (y - h)) / math.cosh(r * h))
    c = start_from_profile(orc, lat, 0.9 * ua)
    run_to_steady(c, 2000, 1e-12, 400000)
    u = c.fields()["ux"][:, 0]
    assert np.linalg.norm(u - ua) / np.linalg.norm(ua) < 1e-3


def test_brinkman_forchheimer_channel_matches_bvp(orc):
    """With the Forchheimer term the steady channel solves
    nu u'' - eps nu u / K - eps Feps u^2 / sqrt K + eps G = 0, u(0)=u(H)=0,
    integrated here independently with scipy's collocation solver."""
    from scipy.integrate import solve_bvp
    ny, eps = 64, 0.5
    nu, K = 0.1, (ny / 8) ** 2
    Feps = 1.75 / math.sqrt(150 * eps ** 3)
    G = 4e-5
    lat = channel_lattice(orc, ny, 1.0, nu_w=nu, gam_w=1.0, eps=eps, K=K, Feps=Feps, G=G)
    lat.nu_ref = nu

    def rhs(yy, s):
        u, du = s
        return np.vstack([du, (eps * nu * u / K + eps * Feps * np.abs(u) * u / math.sqrt(K) - eps * G) / nu])

    yy = np.linspace(0, ny, 2001)
    sol = solve_bvp(rhs, lambda a, b: np.array([a[0], b[0]]), yy, np.zeros((2, yy.size)), tol=1e-10,
                    max_nodes=200000)
    assert sol.success
    y = np.arange(ny) + 0.5
    ua = sol.sol(y)[0]
    assert np.abs(ua).max() * math.sqrt(3) < 0.1   # low Mach
    c = start_from_profile(orc, lat, ua)
    run_to_steady(c, 2000, 1e-12, 400000)
    u = c.fields()["ux"][:, 0]
    assert np.linalg.norm(u - ua) / np.linalg.norm(ua) < 1e-3
    # the Forchheimer term matters at this forcing: without it the flow is faster
    uD = G * K / nu * (1 - np.cosh(math.sqrt(eps / K) * (y - ny / 2)) / math.cosh(math.sqrt(eps / K) * ny / 2))
    assert np.linalg.norm(uD - ua) / np.linalg.norm(ua) > 0.05


@pytest.mark.parametrize("tau_iters", [0, 4])
def test_powerlaw_porous_channel_matches_bvp(orc, tau_iters):
    """A power-law fluid driven through a porous channel: the apparent
    viscosity enters both the shear stress and the Darcy drag, so the steady
    profile solves (nu(|u'|) u')' - eps nu(|u'|) u / K - eps Feps u^2 / sqrt K
    + eps G = 0, u(0) = u(H) = 0, with nu(s) = K_c max(s, gamma_1)^(n-1).
    Integrated independently with scipy's collocation solver in the
    variables (u, q = nu u'); both the lagged and the implicit tau must land
    on it (it fixes the viscosity the velocity solve uses)."""
    from scipy.integrate import solve_bvp
    n, ny, eps = 0.7, 64, 0.6
    K = (ny / 8) ** 2
    Feps = 1.75 / math.sqrt(150 * eps ** 3)
    G = 1e-5
    lat = channel_lattice(orc, ny, n, nu_w=0.1, gam_w=1e-3, eps=eps, K=K, Feps=Feps, G=G)
    lat.tau_iters = tau_iters
    Kc, g1 = lat.nu_ref, lat.gamma1
    q1 = Kc * g1 ** n

    def dudy(q):
        a = np.abs(q)
        return np.sign(q) * np.where(a >= q1, (a / Kc) ** (1 / n), a / (Kc * g1 ** (n - 1)))

    def rhs(yy, s):
        u, q = s
        nu = Kc * np.maximum(np.abs(dudy(q)), g1) ** (n - 1)
        return np.vstack([dudy(q), eps * nu * u / K + eps * Feps * np.abs(u) * u / math.sqrt(K) - eps * G])

    yy = np.linspace(0, ny, 4001)
    guess = np.vstack([1e-3 * np.sin(np.pi * yy / ny), np.zeros_like(yy)])
    sol = solve_bvp(rhs, lambda a, b: np.array([a[0], b[0]]), yy, guess, tol=1e-10, max_nodes=400000)
    assert sol.success
    y = np.arange(ny) + 0.5
    ua = sol.sol(y)[0]
    c = start_from_profile(orc, lat, ua)
    run_to_steady(c, 2000, 1e-12, 400000)
    u = c.fields()["ux"][:, 0]
    assert np.linalg.norm(u - ua) / np.linalg.norm(ua) < 2e-3
    # the viscosity varies across the channel by a factor of ~5, so a drag
    # taken with one viscosity would give a visibly different profile
    nu = c.fields()["nu"][:, 0]
    assert nu.max() / nu.min() > 3
