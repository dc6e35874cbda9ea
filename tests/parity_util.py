"""Per-node check of the relaxation time tau against the oracle.

tau comes from the strain rate through the modified power law (Eq. MPL):
tau = 3 nu_ref D(gamma*) + 1/2.  The strain rate is a small difference of O(1)
moments (non-equilibrium parts ~1e-4 of the moments), so its rounding error
is an absolute bound ``dgam`` rather than a relative one, and the literal law
jumps at gamma_1.  A node's tau is therefore unique only where the oracle's
strain rate is resolved; elsewhere several values are correct, and the check
is that the GPU's tau is the law evaluated at some strain rate within
``dgam`` of the oracle's.

``dgam`` for an input that already differs by ``df`` (max population
difference): the strain-rate moments are e (coefficients 4, 1, 2 over the
populations, plus the equilibrium term 2 rho), p_xx (4 terms) and p_xy
(4 terms); gamma = (3/rho) sqrt(A^2 + B^2 + C^2) with A = (1.4/6) e_neq,
B = w p_xx_neq / 2, C = w p_xy_neq, so |d gamma| <= (3/rho)(|dA| + |dB| + |dC|)
<= 3 (0.234 * 34 + 0.5 * 2 * 8 + 2 * 8) df ~ 100 df for w = 1/tau <= 2; the
arithmetic adds about 100 unit roundoffs.
"""
import numpy as np

EPS = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "f32d": 2.0 ** -24, "bf16d": 2.0 ** -24, "f16d": 2.0 ** -24,
       "f16s": 2.0 ** -24, "bf16s": 2.0 ** -24}


def law_tau(gs, lat):
    """tau from the non-dimensional shear rate (vectorised), per clamp mode."""
    gs = np.asarray(gs, dtype=np.float64)
    nm1 = lat.n - 1.0
    if lat.clamp_mode == 0:
        with np.errstate(divide="ignore"):
            D = np.where(gs < lat.gamma1, 1.0,
                         np.where(gs <= lat.gamma2, np.power(np.maximum(gs, 1e-300), nm1),
                                  lat.gamma2 ** nm1))
    else:
        D = np.power(np.clip(gs, lat.gamma1, lat.gamma2), nm1)
    return 3.0 * lat.nu_ref * D + 0.5


def tau_interval(gam_ref, dgam, lat):
    """Min and max of the law over [gamma* - d, gamma* + d] (pieces are monotone,
    so the extremes sit at the ends or at the one-sided limits of a jump)."""
    gs = gam_ref * lat.gamma_scale
    d = dgam * lat.gamma_scale
    lo_g = np.maximum(gs - d, 0.0)
    hi_g = gs + d
    cands = [law_tau(lo_g, lat), law_tau(hi_g, lat)]
    for b in (lat.gamma1, lat.gamma2):
        inside = (lo_g <= b) & (b <= hi_g)
        below = law_tau(np.full_like(gs, b * (1 - 1e-15)), lat)
        at = law_tau(np.full_like(gs, b), lat)
        cands.append(np.where(inside, below, cands[0]))
        cands.append(np.where(inside, at, cands[0]))
    c = np.stack(cands)
    return c.min(axis=0), c.max(axis=0)


def check_tau(tau, tau_ref, gam_ref, lat, prec, df):
    """Assert tau is valid at every node and close to the oracle where unique.

    tau, tau_ref, gam_ref: arrays of the GPU's tau after the last collision,
    the oracle's, and the oracle's strain rate of that collision; df: max
    population difference of the input to that collision."""
    eps = EPS[prec]
    store = 0.0 if prec == "f64" else 2.0 ** -24   # tau stored in FP32
    dgam = 100.0 * df + 100.0 * eps
    lo, hi = tau_interval(gam_ref, dgam, lat)
    slack = 4 * (eps + store) * hi
    bad = (tau < lo - slack) | (tau > hi + slack)
    assert not bad.any(), f"tau outside the law's range at {np.argwhere(bad)[:5].tolist()}"
    # where the strain rate is resolved and away from the clamp jumps, tau is
    # unique up to the propagated strain-rate error
    gs = gam_ref * lat.gamma_scale
    resolved = (gam_ref > 10 * dgam) & ((gs < lat.gamma1 / 3) | (gs > 3 * lat.gamma1)) & \
        ((gs < lat.gamma2 / 3) | (gs > 3 * lat.gamma2))
    rtol = 2 * abs(lat.n - 1.0) * dgam / np.maximum(gam_ref, 1e-300) + 4 * (eps + store)
    rel = np.abs(tau - tau_ref) / tau_ref
    worst = np.where(resolved, rel - rtol, -1.0)
    assert worst.max() <= 0, f"tau differs beyond its bound at {np.unravel_index(worst.argmax(), worst.shape)}"
    return int(resolved.sum())
