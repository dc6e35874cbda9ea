"""FP64 PyTorch restatement of the oracle's step, for reverse-mode gradients.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``).  It follows
the same algorithm as ``oracle.c`` -- literal moment-space MRT with explicit
M, N and their inverses, the literal strain-rate double sum, the modified
power law, the generalized porous forcing, push streaming with per-link wall
rules, and the wall Nusselt number -- written with whole-grid tensor
operations so that ``torch.autograd`` yields the gradient of a result with
respect to the parameters (per-node Darcy field, power-law index n, Rayleigh
number Ra) through a whole run.  It is pinned to ``oracle.c`` by a CPU test
(same states to round-off) and its gradients to central differences of the C
oracle.  Branches of the literal power law are taken by the forward values
(the derivative is the one of the branch taken).  The node-local implicit
tau (tau_iters > 0: Newton steps on ln tau toward tau = Phi(tau), the
alternative to the lagged tau for the implicit tau-strain coupling of the
collision-matrix and strain-rate equations) is restated too, and autograd
differentiates through its Newton steps as computed; it is pinned to the C
oracle's implicit solve node by node and over whole runs, and its gradients
to central differences of the C oracle run with the same Newton steps.
"""
from __future__ import annotations

import math

import torch

DT = torch.float64
E9 = torch.tensor([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], dtype=DT)
W9 = torch.tensor([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=DT)
OPP9 = [0, 3, 4, 1, 2, 7, 8, 5, 6]
E5 = E9[:5]
W5 = torch.tensor([1 / 3] + [1 / 6] * 4, dtype=DT)
OPP5 = [0, 3, 4, 1, 2]


def _matrices():
    ex, ey = E9[:, 0], E9[:, 1]
    e2 = ex * ex + ey * ey
    M = torch.stack([torch.ones(9, dtype=DT), 3 * e2 - 4, 4.5 * e2 * e2 - 10.5 * e2 + 4, ex, (3 * e2 - 5) * ex,
                     ey, (3 * e2 - 5) * ey, ex * ex - ey * ey, ex * ey])
    ex5, ey5 = E5[:, 0], E5[:, 1]
    e25 = ex5 * ex5 + ey5 * ey5
    N = torch.stack([torch.ones(5, dtype=DT), ex5, ey5, 5 * e25 - 4, ex5 * ex5 - ey5 * ey5])
    return M, torch.linalg.inv(M), N, torch.linalg.inv(N)


M, MINV, N, NINV = _matrices()


class Params:
    """Lattice parameters as differentiable functions of (n, Ra, Da field),
    following the same mapping as the C oracle's orc_map_params."""

    def __init__(self, nx, ny, n, Ra, Da, Pr, porosity=0.6, Ma=0.1, porous_model=1, clamp_mode=0,
                 s_e=1.5, s_p=1.5, tau_iters=0):
        self.nx, self.ny = nx, ny
        self.tau_iters = int(tau_iters)
        self.n = n if torch.is_tensor(n) else torch.tensor(float(n), dtype=DT)
        self.Ra = Ra if torch.is_tensor(Ra) else torch.tensor(float(Ra), dtype=DT)
        Da = Da if torch.is_tensor(Da) else torch.tensor(Da, dtype=DT)
        Uc = Ma / math.sqrt(3.0)
        L = float(nx)
        self.L = L
        nu0 = Pr / torch.pow(torch.sqrt(self.Ra), 2.0 - self.n)
        self.nu_ref = nu0 * Uc * L
        self.gamma_scale = L / Uc
        self.gamma1, self.gamma2 = 0.01, 1.0e6
        self.clamp_mode = clamp_mode
        self.K = Da * L * L            # scalar or [ny][nx]
        if porous_model == 1:
            self.eps = porosity
            self.Feps = 1.75 / math.sqrt(150.0 * porosity ** 3)
        else:
            self.eps, self.Feps = 1.0, 0.0
        self.T_hot, self.T_cold = 1.0, 0.0
        self.Tm = 0.5
        self.gbeta = Pr * Uc * Uc / L
        self.tauT = 3.0 * Uc * L / torch.sqrt(self.Ra) + 0.5
        self.s = torch.tensor([1.0, 1.4, 1.4, 1.0, 1.2, 1.0, 1.2, 0.0, 0.0], dtype=DT)
        self.s_e, self.s_p = s_e, s_p
        D0 = 1.0 if clamp_mode == 0 else torch.pow(torch.tensor(self.gamma1, dtype=DT), self.n - 1.0)
        self.tau0 = 3.0 * self.nu_ref * D0 + 0.5


def rest_state(p: Params):
    f = (W9 * 1.0)[:, None, None].expand(9, p.ny, p.nx).clone()
    g = (W5 * 0.5)[:, None, None].expand(5, p.ny, p.nx).clone()
    tau = p.tau0 * torch.ones(p.ny, p.nx, dtype=DT)
    return f, g, tau


def _shift(a, ex, ey):
    """out[y, x] = a[y - ey, x - ex] where the source exists, else 0."""
    ny, nx = a.shape
    out = torch.zeros_like(a)
    ys, yd = (slice(0, ny - ey), slice(ey, ny)) if ey >= 0 else (slice(-ey, ny), slice(0, ny + ey))
    xs, xd = (slice(0, nx - ex), slice(ex, nx)) if ex >= 0 else (slice(-ex, nx), slice(0, nx + ex))
    out[yd, xd] = a[ys, xs]
    return out


def _arrives(nx, ny, ex, ey):
    """Mask of nodes that receive a population along (ex, ey) from a node."""
    m = torch.ones(ny, nx, dtype=torch.bool)
    return _shift(m.to(DT), ex, ey) > 0.5


def stream(f, g, p: Params):
    """Push every population one link; a link leaving the cavity returns to
    its node reversed (bounce-back; anti-bounce-back on the isothermal walls)."""
    nx, ny = p.nx, p.ny
    fs = []
    for i in range(9):
        ex, ey = int(E9[i, 0]), int(E9[i, 1])
        inside = _arrives(nx, ny, ex, ey)
        # the population arriving along e_i at x came from x - e_i, or, if
        # that node does not exist, is the node's own opposite population
        fs.append(torch.where(inside, _shift(f[i], ex, ey), f[OPP9[i]]))
    gs = []
    for i in range(5):
        ex, ey = int(E5[i, 0]), int(E5[i, 1])
        inside = _arrives(nx, ny, ex, ey)
        if ex == 1:      # source x - 1 missing at x = 0: hot wall
            wall = -g[OPP5[i]] + 2.0 * W5[OPP5[i]] * p.T_hot
        elif ex == -1:   # source x + 1 missing at x = nx - 1: cold wall
            wall = -g[OPP5[i]] + 2.0 * W5[OPP5[i]] * p.T_cold
        else:            # adiabatic top / bottom
            wall = g[OPP5[i]]
        gs.append(torch.where(inside, _shift(g[i], ex, ey), wall))
    return torch.stack(fs), torch.stack(gs)


def _apparent(p: Params, gs):
    nm1 = p.n - 1.0
    if p.clamp_mode == 0:
        safe = torch.clamp(gs, min=1e-300)
        mid = torch.pow(safe, nm1)
        hi = torch.pow(torch.tensor(p.gamma2, dtype=DT), nm1)
        return torch.where(gs < p.gamma1, torch.ones_like(gs), torch.where(gs <= p.gamma2, mid, hi))
    return torch.pow(torch.clamp(gs, p.gamma1, p.gamma2), nm1)


def _strain(fs, gs, tau_in, p: Params, want_R=False):
    """Steps 1-6 of oracle.c's node update (its strain_state) for every node,
    started from the relaxation time tau_in: the porous velocity, the force,
    and |gamma| from the literal strain-rate sum; with want_R also
    R = d ln|gamma| / d ln(1/tau_in) at fixed velocity (omega gamma:gamma_p /
    gamma:gamma, gamma_p the same sum with S replaced by diag(0, ..., 0, 1, 1)),
    0 where gamma = 0."""
    ex, ey = E9[:, 0][:, None, None], E9[:, 1][:, None, None]
    rho = fs.sum(0)
    jx = (fs * ex).sum(0)
    jy = (fs * ey).sum(0)
    T = gs.sum(0)
    Gx = torch.zeros_like(T)
    Gy = p.gbeta * (T - p.Tm)
    vx = jx / rho + 0.5 * p.eps * Gx
    vy = jy / rho + 0.5 * p.eps * Gy
    nu_in = (tau_in - 0.5) / 3.0
    K = p.K
    c0 = 0.5 * (1.0 + p.eps * nu_in / (2.0 * K))
    c1 = p.eps * p.Feps / (2.0 * torch.sqrt(torch.as_tensor(K, dtype=DT)))
    vmag = torch.sqrt(vx * vx + vy * vy)
    den = c0 + torch.sqrt(c0 * c0 + c1 * vmag)
    ux, uy = vx / den, vy / den
    umag = torch.sqrt(ux * ux + uy * uy)
    sK = torch.sqrt(torch.as_tensor(K, dtype=DT))
    Fx = -p.eps * nu_in * ux / K - p.eps * p.Feps * umag * ux / sK + p.eps * Gx
    Fy = -p.eps * nu_in * uy / K - p.eps * p.Feps * umag * uy / sK + p.eps * Gy
    # velocity-space equilibrium and the literal strain-rate sum
    eu = ex * ux + ey * uy
    u2 = ux * ux + uy * uy
    W = W9[:, None, None]
    feq = W * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu / p.eps - 1.5 * u2 / p.eps)
    fneq = fs - feq
    Sp = p.s[:, None, None].expand(9, *rho.shape).clone()
    Sp[7] = 1.0 / tau_in
    Sp[8] = 1.0 / tau_in
    mfneq = torch.einsum("ij,jyx->iyx", M, fneq)
    h = torch.einsum("ij,jyx->iyx", MINV, mfneq * Sp)
    gxx = -3.0 / (2.0 * rho) * (h * ex * ex).sum(0)
    gyy = -3.0 / (2.0 * rho) * (h * ey * ey).sum(0)
    gxy = -3.0 / (2.0 * rho) * (h * ex * ey).sum(0)
    gg = gxx * gxx + gyy * gyy + 2.0 * gxy * gxy
    gamma = torch.sqrt(2.0 * gg)
    R = None
    if want_R:
        Pm = torch.zeros(9, dtype=DT)
        Pm[7] = Pm[8] = 1.0
        hp = torch.einsum("ij,jyx->iyx", MINV, mfneq * Pm[:, None, None])
        pxx = -3.0 / (2.0 * rho) * (hp * ex * ex).sum(0)
        pyy = -3.0 / (2.0 * rho) * (hp * ey * ey).sum(0)
        pxy = -3.0 / (2.0 * rho) * (hp * ex * ey).sum(0)
        ggp = gxx * pxx + gyy * pyy + 2.0 * gxy * pxy
        safe = torch.where(gg > 0, gg, torch.ones_like(gg))
        R = torch.where(gg > 0, (1.0 / tau_in) * ggp / safe, torch.zeros_like(gg))
    return rho, T, ux, uy, Fx, Fy, gamma, R


def implicit_tau(fs, gs, p: Params, iters):
    """oracle.c's node-local implicit tau for every node: `iters` Newton steps
    on ln tau toward tau = Phi(tau) = 3 nu_ref D(gamma*(tau)) + 1/2 from the
    rest-state tau0, tau <- tau (Phi / tau)^(1/J) with
    J = 1 - (1 - n) R (Phi - 1/2) / Phi where the power law has slope
    (gamma1 < gamma* < gamma2), else J = 1 and tau <- Phi."""
    tau = p.tau0 * torch.ones(fs.shape[1:], dtype=DT)
    for _ in range(iters):
        *_, gamma, R = _strain(fs, gs, tau, p, want_R=True)
        gsn = gamma * p.gamma_scale
        phi = 3.0 * p.nu_ref * _apparent(p, gsn) + 0.5
        slope = (gsn > p.gamma1) & (gsn < p.gamma2)
        J = torch.where(slope, 1.0 - (1.0 - p.n) * R * (phi - 0.5) / phi, torch.ones_like(phi))
        newton = tau * torch.pow(phi / tau, 1.0 / J)
        tau = torch.where(J == 1.0, phi, newton)
    return tau


def collide(fs, gs, tau_prev, p: Params):
    """Node update of every node, steps 1-9 of oracle.c's node_update, started
    from tau_prev (the lagged tau, or the implicit one)."""
    ex, ey = E9[:, 0][:, None, None], E9[:, 1][:, None, None]
    rho, T, ux, uy, Fx, Fy, gamma, _ = _strain(fs, gs, tau_prev, p)
    eu = ex * ux + ey * uy
    u2 = ux * ux + uy * uy
    W = W9[:, None, None]
    nu = p.nu_ref * _apparent(p, gamma * p.gamma_scale)
    tau = 3.0 * nu + 0.5
    # forced MRT collision
    m = torch.einsum("ij,jyx->iyx", M, fs)
    meq = torch.stack([rho, rho * (-2.0 + 3.0 * u2 / p.eps), rho * (1.0 - 3.0 * u2 / p.eps), rho * ux, -rho * ux,
                       rho * uy, -rho * uy, rho * (ux * ux - uy * uy) / p.eps, rho * ux * uy / p.eps])
    eF = ex * Fx + ey * Fy
    uF = ux * Fx + uy * Fy
    Fv = W * rho * (3.0 * eF + 9.0 * eu * eF / p.eps - 3.0 * uF / p.eps)
    Fh = torch.einsum("ij,jyx->iyx", M, Fv)
    S = p.s[:, None, None].expand(9, *tau_prev.shape).clone()
    S[7] = 1.0 / tau
    S[8] = 1.0 / tau
    ms = m - S * (m - meq) + (1.0 - 0.5 * S) * Fh
    fo = torch.einsum("ij,jyx->iyx", MINV, ms)
    # thermal MRT collision
    n_ = torch.einsum("ij,jyx->iyx", N, gs)
    neq = torch.stack([T, T * ux, T * uy, -2.0 * T / 3.0, torch.zeros_like(T)])
    ST = torch.stack([torch.ones((), dtype=DT), 1.0 / p.tauT, 1.0 / p.tauT,
                      torch.tensor(p.s_e, dtype=DT), torch.tensor(p.s_p, dtype=DT)])[:, None, None]
    ns = n_ - ST * (n_ - neq)
    go = torch.einsum("ij,jyx->iyx", NINV, ns)
    return fo, go, tau


def step(f, g, tau, p: Params, k=1):
    """k steps.  With p.tau_iters > 0 each collision starts from the implicit
    tau and the tau passed in is not used (the returned tau is then the one
    the last collision produced, which the C oracle does not keep)."""
    for _ in range(k):
        fs, gs = stream(f, g, p)
        t_in = implicit_tau(fs, gs, p, p.tau_iters) if p.tau_iters > 0 else tau
        f, g, tau = collide(fs, gs, t_in, p)
    return f, g, tau


def nusselt_hot(g, p: Params):
    """Hot-wall average Nu from the streamed temperature (same formula as the
    C oracle: -L (9 theta_0 - theta_1 - 8) / 3 per row, averaged)."""
    _, gs = stream(torch.zeros(9, p.ny, p.nx, dtype=DT), g, p)
    T = gs.sum(0)
    th = (T - p.T_cold) / (p.T_hot - p.T_cold)
    return (-p.L * (9.0 * th[:, 0] - th[:, 1] - 8.0) / 3.0).mean()
