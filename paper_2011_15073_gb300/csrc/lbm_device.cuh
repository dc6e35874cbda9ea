// lbm_device.cuh -- device-side physics of the fused MRT step (sm_103a).
//
// Closed-form moment transforms: the D2Q9 basis rows are mutually orthogonal,
// so M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4) and the
// D2Q5 N^-1 = N^T diag(1/5, 1/2, 1/2, 1/20, 1/4); every product below is
// written out with those integer coefficients instead of a matrix multiply.
// The strain-rate double sum of the power-law section collapses to the three
// non-equilibrium moments that carry second velocity moments (e, p_xx, p_xy).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

#include "lbm_internal.h"

namespace lbm {

// Per-case constants in the compute type R (built on the host from
// lbm_lattice by make_params below).
template <class R>
struct Phys {
    int nx, ny;
    int64_t pitch;   // elements between rows of a plane
    int64_t plane;   // elements between planes
    R nu_ref, gamma_scale, gamma1, gamma2, nm1, D_hi;
    int clamp_mode;
    R eps, inv_eps;
    R half_eps_invK;   // eps / (2 K) / 2 -> c0 = 1/2 + half_eps_invK * nu
    R eps_invK;        // eps / K
    R c1;              // eps F_eps / (2 sqrt K)
    R eFe_isqK;        // eps F_eps / sqrt K
    R gbeta, Tm;
    R omegaT, s_e, s_p;
    R abb_hot, abb_cold;   // 2 w T_wall for the anti-bounce-back (w = 1/6)
};

// ------------------------------------------------------------ parameters
template <class R>
inline Phys<R> make_params(const lbm_ctx *c)
{
    const lbm_lattice &L = c->lat;
    Phys<R> p;
    p.nx = c->nx;
    p.ny = c->ny;
    p.pitch = c->pitch;
    p.plane = c->plane;
    p.nu_ref = R(L.nu_ref);
    p.gamma_scale = R(L.gamma_scale);
    p.gamma1 = R(L.gamma1);
    p.gamma2 = R(L.gamma2);
    p.nm1 = R(L.n - 1.0);
    p.D_hi = R(pow(L.gamma2, L.n - 1.0));
    p.clamp_mode = L.clamp_mode;
    p.eps = R(L.eps);
    p.inv_eps = R(1.0 / L.eps);
    p.half_eps_invK = R(L.eps / (4.0 * L.K));
    p.eps_invK = R(L.eps / L.K);
    p.c1 = R(L.eps * L.Feps / (2.0 * sqrt(L.K)));
    p.eFe_isqK = R(L.eps * L.Feps / sqrt(L.K));
    p.gbeta = R(L.gbeta);
    p.Tm = R(L.Tm);
    p.omegaT = R(1.0 / L.tauT);
    p.s_e = R(L.s_e);
    p.s_p = R(L.s_p);
    p.abb_hot = R(2.0 / 6.0 * L.T_hot);
    p.abb_cold = R(2.0 / 6.0 * L.T_cold);
    return p;
}

// Rest-state values used by the deviation storage forms.
__host__ __device__ constexpr double rest_f(int i)
{
    return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
}
__host__ __device__ constexpr double rest_g(int i)  // w_i T_m with T_m = 1/2
{
    return i == 0 ? 1.0 / 6.0 : 1.0 / 12.0;
}

// ---------------------------------------------------------------- storage
template <int PREC>
struct Store;

template <>
struct Store<LBM_F64> {
    using S = double;
    using R = double;
    using TauS = double;
    static __device__ __forceinline__ R ld(const S *p, int64_t k, R) { return p[k]; }
    static __device__ __forceinline__ void st(S *p, int64_t k, R v, R) { p[k] = v; }
};
template <>
struct Store<LBM_F32> {
    using S = float;
    using R = float;
    using TauS = float;
    static __device__ __forceinline__ R ld(const S *p, int64_t k, R) { return p[k]; }
    static __device__ __forceinline__ void st(S *p, int64_t k, R v, R) { p[k] = v; }
};
template <>
struct Store<LBM_BF16D> {
    using S = __nv_bfloat16;
    using R = float;
    using TauS = float;
    static __device__ __forceinline__ R ld(const S *p, int64_t k, R rest)
    {
        return rest + __bfloat162float(p[k]);
    }
    static __device__ __forceinline__ void st(S *p, int64_t k, R v, R rest)
    {
        p[k] = __float2bfloat16_rn(v - rest);
    }
};
template <>
struct Store<LBM_F16D> {
    using S = __half;
    using R = float;
    using TauS = float;
    static __device__ __forceinline__ R ld(const S *p, int64_t k, R rest)
    {
        return rest + __half2float(p[k]);
    }
    static __device__ __forceinline__ void st(S *p, int64_t k, R v, R rest)
    {
        p[k] = __float2half_rn(v - rest);
    }
};

// D = (gamma*)^(n-1) in the compute precision.
__device__ __forceinline__ double powD(double x, double e) { return pow(x, e); }
__device__ __forceinline__ float powD(float x, float e) { return exp2f(e * __log2f(x)); }

// ----------------------------------------------------------- pull streaming
// Streamed populations of node (x, y): f_i(x) = f*_i(x - e_i) when the source
// node exists, otherwise the link crossed a wall halfway between the node and
// the wall and the population comes back reversed from the node itself
// (bounce-back for the flow; anti-bounce-back -g* + 2 w T_w on the isothermal
// left/right walls and bounce-back on the adiabatic top/bottom walls for the
// heat).  Velocity order: e0 (0,0), e1 (1,0), e2 (0,1), e3 (-1,0), e4 (0,-1),
// e5 (1,1), e6 (-1,1), e7 (-1,-1), e8 (1,-1).
template <int PREC, class R>
__device__ __forceinline__ void pull(const typename Store<PREC>::S *__restrict__ src,
                                     const Phys<R> &p, int x, int y, R f[9], R g[5])
{
    using St = Store<PREC>;
    const int64_t P = p.plane, W = p.pitch;
    const int64_t k = (int64_t)y * W + x;
    const bool xl = x > 0, xr = x < p.nx - 1, yb = y > 0, yt = y < p.ny - 1;
    f[0] = St::ld(src, 0 * P + k, R(rest_f(0)));
    f[1] = xl ? St::ld(src, 1 * P + k - 1, R(rest_f(1))) : St::ld(src, 3 * P + k, R(rest_f(3)));
    f[2] = yb ? St::ld(src, 2 * P + k - W, R(rest_f(2))) : St::ld(src, 4 * P + k, R(rest_f(4)));
    f[3] = xr ? St::ld(src, 3 * P + k + 1, R(rest_f(3))) : St::ld(src, 1 * P + k, R(rest_f(1)));
    f[4] = yt ? St::ld(src, 4 * P + k + W, R(rest_f(4))) : St::ld(src, 2 * P + k, R(rest_f(2)));
    f[5] = (xl && yb) ? St::ld(src, 5 * P + k - W - 1, R(rest_f(5))) : St::ld(src, 7 * P + k, R(rest_f(7)));
    f[6] = (xr && yb) ? St::ld(src, 6 * P + k - W + 1, R(rest_f(6))) : St::ld(src, 8 * P + k, R(rest_f(8)));
    f[7] = (xr && yt) ? St::ld(src, 7 * P + k + W + 1, R(rest_f(7))) : St::ld(src, 5 * P + k, R(rest_f(5)));
    f[8] = (xl && yt) ? St::ld(src, 8 * P + k + W - 1, R(rest_f(8))) : St::ld(src, 6 * P + k, R(rest_f(6)));
    const typename Store<PREC>::S *gs = src + 9 * P;
    g[0] = St::ld(gs, 0 * P + k, R(rest_g(0)));
    g[1] = xl ? St::ld(gs, 1 * P + k - 1, R(rest_g(1))) : p.abb_hot - St::ld(gs, 3 * P + k, R(rest_g(3)));
    g[2] = yb ? St::ld(gs, 2 * P + k - W, R(rest_g(2))) : St::ld(gs, 4 * P + k, R(rest_g(4)));
    g[3] = xr ? St::ld(gs, 3 * P + k + 1, R(rest_g(3))) : p.abb_cold - St::ld(gs, 1 * P + k, R(rest_g(1)));
    g[4] = yt ? St::ld(gs, 4 * P + k + W, R(rest_g(4))) : St::ld(gs, 2 * P + k, R(rest_g(2)));
}

// ------------------------------------------------------ macroscopic moments
template <class R>
struct Macro {
    R rho, irho, jx, jy, T, ux, uy, Fx, Fy, nu_prev;
    R nu;  // apparent viscosity chosen by the collision (set by collide)
};

// Density and temperature (Eqs. macro_fluid_density and the D2Q5 zeroth
// moment), the half-force velocity of Eq. (velo) with buoyancy
// G = g beta (T - T_m) along +y, and the porous velocity solve
// u = v / (c0 + sqrt(c0^2 + c1 |v|)), c0 = (1 + eps nu / (2K)) / 2, with the
// apparent viscosity of the lagged relaxation time; then the total force
// F = -eps nu u / K - eps F_eps |u| u / sqrt K + eps G.
template <class R>
__device__ __forceinline__ Macro<R> macro(const Phys<R> &p, const R f[9], const R g[5], R tau_prev)
{
    Macro<R> m;
    const R sax = (f[1] + f[2]) + (f[3] + f[4]);
    const R sdg = (f[5] + f[6]) + (f[7] + f[8]);
    m.rho = f[0] + sax + sdg;
    m.jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    m.jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    m.T = g[0] + (g[1] + g[2]) + (g[3] + g[4]);
    const R Gy = p.gbeta * (m.T - p.Tm);
    m.irho = R(1) / m.rho;
    const R vx = m.jx * m.irho;
    const R vy = m.jy * m.irho + R(0.5) * p.eps * Gy;
    m.nu_prev = (tau_prev - R(0.5)) * R(1.0 / 3.0);
    const R c0 = R(0.5) + p.half_eps_invK * m.nu_prev;
    const R vmag = sqrt(vx * vx + vy * vy);
    const R iden = R(1) / (c0 + sqrt(c0 * c0 + p.c1 * vmag));
    m.ux = vx * iden;
    m.uy = vy * iden;
    const R umag = sqrt(m.ux * m.ux + m.uy * m.uy);
    const R drag = -(p.eps_invK * m.nu_prev + p.eFe_isqK * umag);
    m.Fx = drag * m.ux;
    m.Fy = drag * m.uy + p.eps * Gy;
    return m;
}

// Apparent-viscosity factor of Eq. (MPL) for the non-dimensional shear rate.
template <class R>
__device__ __forceinline__ R apparent(const Phys<R> &p, R gs)
{
    if (p.clamp_mode == 0)
        return gs < p.gamma1 ? R(1) : (gs <= p.gamma2 ? powD(gs, p.nm1) : p.D_hi);
    const R gc = gs < p.gamma1 ? p.gamma1 : (gs > p.gamma2 ? p.gamma2 : gs);
    return powD(gc, p.nm1);
}

// Full node update in place: f, g become the post-collision populations.
// Returns the new relaxation time; m receives the macroscopic moments and the
// apparent lattice viscosity of this collision.
template <class R>
__device__ __forceinline__ R collide(const Phys<R> &p, R f[9], R g[5], R tau_prev, Macro<R> &m)
{
    m = macro<R>(p, f, g, tau_prev);
    const R rho = m.rho, ux = m.ux, uy = m.uy;
    // raw moments
    const R sax = (f[1] + f[2]) + (f[3] + f[4]);
    const R sdg = (f[5] + f[6]) + (f[7] + f[8]);
    const R e = R(-4) * f[0] - sax + R(2) * sdg;
    const R ep = R(4) * f[0] - R(2) * sax + sdg;
    const R qx = R(-2) * (f[1] - f[3]) + ((f[5] - f[6]) + (f[8] - f[7]));
    const R qy = R(-2) * (f[2] - f[4]) + ((f[5] + f[6]) - (f[7] + f[8]));
    const R pxx = (f[1] + f[3]) - (f[2] + f[4]);
    const R pxy = (f[5] + f[7]) - (f[6] + f[8]);
    // equilibria
    const R u2e = (ux * ux + uy * uy) * p.inv_eps;
    const R e_eq = rho * (R(-2) + R(3) * u2e);
    const R ep_eq = rho * (R(1) - R(3) * u2e);
    const R pxx_eq = rho * (ux * ux - uy * uy) * p.inv_eps;
    const R pxy_eq = rho * ux * uy * p.inv_eps;
    // strain rate from the non-equilibrium moments with the lagged tau:
    // gamma_xx,yy = -3/(2 rho) (s1 e_neq / 6 +- w pxx_neq / 2),
    // gamma_xy = -3/(2 rho) w pxy_neq, |gamma| = sqrt(2 gamma:gamma)
    const R wp = R(1) / tau_prev;
    const R A = R(1.4 / 6.0) * (e - e_eq);
    const R B = R(0.5) * wp * (pxx - pxx_eq);
    const R C = wp * (pxy - pxy_eq);
    const R gam = R(3) * m.irho * sqrt(A * A + B * B + C * C);
    const R nu = p.nu_ref * apparent<R>(p, gam * p.gamma_scale);
    const R tau = R(3) * nu + R(0.5);
    const R w = R(1) / tau;
    m.nu = nu;
    // forcing moments (M applied to the velocity-space porous force term)
    const R uF = ux * m.Fx + uy * m.Fy;
    const R Fe = R(6) * rho * uF * p.inv_eps;
    const R Fxx = R(2) * rho * (ux * m.Fx - uy * m.Fy) * p.inv_eps;
    const R Fxy = rho * (ux * m.Fy + uy * m.Fx) * p.inv_eps;
    // post-collision moments, m* = m - S (m - m_eq) + (I - S/2) F
    const R es = e - R(1.4) * (e - e_eq) + R(0.3) * Fe;
    const R eps_s = ep - R(1.4) * (ep - ep_eq) - R(0.3) * Fe;
    const R jxs = rho * (ux + R(0.5) * m.Fx);
    const R jys = rho * (uy + R(0.5) * m.Fy);
    const R qxs = qx - R(1.2) * (qx + rho * ux) - R(0.4) * rho * m.Fx;
    const R qys = qy - R(1.2) * (qy + rho * uy) - R(0.4) * rho * m.Fy;
    const R hw = R(1) - R(0.5) * w;
    const R pxxs = pxx - w * (pxx - pxx_eq) + hw * Fxx;
    const R pxys = pxy - w * (pxy - pxy_eq) + hw * Fxy;
    // f* = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4) m*
    const R a0 = rho * R(1.0 / 9.0), a1 = es * R(1.0 / 36.0), a2 = eps_s * R(1.0 / 36.0);
    const R a3 = jxs * R(1.0 / 6.0), a4 = qxs * R(1.0 / 12.0);
    const R a5 = jys * R(1.0 / 6.0), a6 = qys * R(1.0 / 12.0);
    const R a7 = pxxs * R(0.25), a8 = pxys * R(0.25);
    const R b_ax = a0 - a1 - R(2) * a2;  // common part of f1..f4
    const R b_dg = a0 + R(2) * a1 + a2;  // common part of f5..f8
    const R xa = a3 - R(2) * a4, ya = a5 - R(2) * a6;
    const R xd = a3 + a4, yd = a5 + a6;
    f[0] = a0 - R(4) * a1 + R(4) * a2;
    f[1] = b_ax + xa + a7;
    f[2] = b_ax + ya - a7;
    f[3] = b_ax - xa + a7;
    f[4] = b_ax - ya - a7;
    f[5] = b_dg + xd + yd + a8;
    f[6] = b_dg - xd + yd - a8;
    f[7] = b_dg - xd - yd + a8;
    f[8] = b_dg + xd - yd - a8;
    // thermal MRT: n = N g, n* = n - S_T (n - n_eq), n_eq = (T, T u, -2T/3, 0)
    const R T = m.T;
    const R n1 = g[1] - g[3], n2 = g[2] - g[4];
    const R n3 = R(-4) * g[0] + (g[1] + g[2]) + (g[3] + g[4]);
    const R n4 = (g[1] + g[3]) - (g[2] + g[4]);
    const R n1s = n1 - p.omegaT * (n1 - T * ux);
    const R n2s = n2 - p.omegaT * (n2 - T * uy);
    const R n3s = n3 - p.s_e * (n3 + R(2.0 / 3.0) * T);
    const R n4s = n4 - p.s_p * n4;
    // g* = N^T diag(1/5, 1/2, 1/2, 1/20, 1/4) n*
    const R t0 = T * R(0.2), t3 = n3s * R(0.05), t4 = n4s * R(0.25);
    const R h1 = n1s * R(0.5), h2 = n2s * R(0.5);
    g[0] = t0 - n3s * R(0.2);
    g[1] = t0 + h1 + t3 + t4;
    g[2] = t0 + h2 + t3 - t4;
    g[3] = t0 - h1 + t3 + t4;
    g[4] = t0 - h2 + t3 - t4;
    return tau;
}

}  // namespace lbm
