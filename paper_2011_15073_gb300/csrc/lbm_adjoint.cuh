// lbm_adjoint.cuh -- reverse mode (discrete adjoint) of one node's collision.
//
// collide_adj recomputes the node's forward intermediates exactly as collide
// does (lbm_device.cuh), then propagates the adjoints of the outputs
// (post-collision f*, g* and tau) back, statement by statement, to the
// inputs (the pulled f, g and the lagged tau) and to the parameters: the
// node's porous coefficients (hence its Darcy number), the reference
// viscosity and the power-law exponent (hence n and Ra), and the thermal
// relaxation rate (hence Ra).  Branches of the modified power law take the
// derivative of the branch the forward pass took; at |v| = 0 and |gamma| = 0
// (where the square roots are not differentiable) the subgradient 0 is used.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// Adjoints of the per-node parameters produced by one collision.
template <class V>
struct ParamAdj {
    V heK, eK, c1, eFsK;  // porous coefficients of this node
    V nu_ref, nm1, omegaT;
};

template <class V>
__device__ __forceinline__ void collide_adj(const Phys<V> &p, const V f[9], const V g[5], V tau_prev, int64_t k,
                                            const V fb_out[9], const V gb_out[5], V taub_new, V fb[9], V gb[5],
                                            V &taub_prev, ParamAdj<V> &pa)
{
    // ------------------------------------------------------------ forward
    const Porous<V> q = porous_at(p, k);
    const V sax = (f[1] + f[2]) + (f[3] + f[4]);
    const V sdg = (f[5] + f[6]) + (f[7] + f[8]);
    const V rho = f[0] + sax + sdg;
    const V jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    const V jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    const V T = g[0] + (g[1] + g[2]) + (g[3] + g[4]);
    const V Gy = p.gbeta * (T - p.Tm);
    const V irho = vrcp(rho);
    const V vx = jx * irho;
    const V vy = vfma(p.half_eps, Gy, jy * irho);
    const V nu_prev = (tau_prev - V(0.5)) * V(1.0 / 3.0);
    const V c0 = vfma(q.heK, nu_prev, V(0.5));
    const V vmag = vsqrt(vfma(vx, vx, vy * vy));
    const V sq = vsqrt(vfma(c0, c0, q.c1 * vmag));
    const V iden = vrcp(c0 + sq);
    const V ux = vx * iden, uy = vy * iden;
    const V umag = vmag * iden;
    const V drag = -vfma(q.eK, nu_prev, q.eFsK * umag);
    const V Fx = drag * ux;
    const V Fy = vfma(drag, uy, p.eps * Gy);
    const V e = vfma(V(2), sdg, vfma(V(-4), f[0], -sax));
    const V ep = vfma(V(4), f[0], vfma(V(-2), sax, sdg));
    const V qx = vfma(V(-2), f[1] - f[3], (f[5] - f[6]) + (f[8] - f[7]));
    const V qy = vfma(V(-2), f[2] - f[4], (f[5] + f[6]) - (f[7] + f[8]));
    const V pxx = (f[1] + f[3]) - (f[2] + f[4]);
    const V pxy = (f[5] + f[7]) - (f[6] + f[8]);
    const V rie = rho * p.inv_eps;
    const V u2e3 = V(3) * vfma(ux, ux, uy * uy) * p.inv_eps;
    const V e_eq = vfma(rho, u2e3, V(-2) * rho);
    const V ep_eq = rho - rho * u2e3;
    const V pxx_eq = rie * vfma(ux, ux, -(uy * uy));
    const V pxy_eq = rie * (ux * uy);
    const V wp = vrcp(tau_prev);
    const V A = V(1.4 / 6.0) * (e - e_eq);
    const V B = V(0.5) * wp * (pxx - pxx_eq);
    const V C = wp * (pxy - pxy_eq);
    const V sQ = vsqrt(vfma(A, A, vfma(B, B, C * C)));
    const V gam = V(3) * irho * sQ;
    const V gs = gam * p.gamma_scale;
    // the modified power law and its local derivatives
    V D, dD_dgs = V(0), dD_dnm1 = V(0);
    if (p.clamp_mode == 0) {
        if (gs < p.gamma1) {
            D = V(1);
        } else if (gs <= p.gamma2) {
            D = vpow(gs, p.nm1);
            dD_dgs = p.nm1 * D * vrcp(gs);
            dD_dnm1 = D * log(gs);
        } else {
            D = p.D_hi;
            dD_dnm1 = D * log(p.gamma2);
        }
    } else {
        const V gc = gs < p.gamma1 ? p.gamma1 : (gs > p.gamma2 ? p.gamma2 : gs);
        D = vpow(gc, p.nm1);
        dD_dnm1 = D * log(gc);
        if (gs > p.gamma1 && gs < p.gamma2) dD_dgs = p.nm1 * D * vrcp(gs);
    }
    const V nu = p.nu_ref * D;
    const V tau = vfma(V(3), nu, V(0.5));
    const V w = vrcp(tau);
    const V uF = vfma(ux, Fx, uy * Fy);
    const V Fe = V(6) * rie * uF;
    const V Fxx = V(2) * rie * vfma(ux, Fx, -(uy * Fy));
    const V Fxy = rie * vfma(ux, Fy, uy * Fx);
    const V hw = vfma(V(-0.5), w, V(1));

    // ------------------------------------------------------------ reverse
    // g* = N^T diag(1/5, 1/2, 1/2, 1/20, 1/4) n*
    const V nb0 = (gb_out[0] + gb_out[1] + gb_out[2] + gb_out[3] + gb_out[4]) * V(0.2);
    const V nb1s = (gb_out[1] - gb_out[3]) * V(0.5);
    const V nb2s = (gb_out[2] - gb_out[4]) * V(0.5);
    const V nb3s = (V(-4) * gb_out[0] + gb_out[1] + gb_out[2] + gb_out[3] + gb_out[4]) * V(0.05);
    const V nb4s = (gb_out[1] - gb_out[2] + gb_out[3] - gb_out[4]) * V(0.25);
    const V n1 = g[1] - g[3], n2 = g[2] - g[4];
    V Tb = nb0, uxb = V(0), uyb = V(0), rhob = V(0);
    // n1s = n1 - wT (n1 - T ux), n2s likewise, n3s = n3 - s_e (n3 + 2T/3), n4s = (1 - s_p) n4
    const V nb1 = (V(1) - p.omegaT) * nb1s;
    const V nb2 = (V(1) - p.omegaT) * nb2s;
    Tb = Tb + p.omegaT * (ux * nb1s + uy * nb2s);
    uxb = uxb + p.omegaT * T * nb1s;
    uyb = uyb + p.omegaT * T * nb2s;
    pa.omegaT = (T * ux - n1) * nb1s + (T * uy - n2) * nb2s;
    const V nb3 = (V(1) - p.s_e) * nb3s;
    Tb = Tb - V(2.0 / 3.0) * p.s_e * nb3s;
    const V nb4 = (V(1) - p.s_p) * nb4s;
    // n = N g (rows T, j_x, j_y, 5|e|^2-4, e_x^2-e_y^2); T's adjoint joins later
    V gbl[5];
    gbl[0] = V(-4) * nb3;
    gbl[1] = nb1 + nb3 + nb4;
    gbl[2] = nb2 + nb3 - nb4;
    gbl[3] = -nb1 + nb3 + nb4;
    gbl[4] = -nb2 + nb3 - nb4;

    // f* = M^T diag(...) m*: a_k = sum_i M_ki fb_out_i
    const V F0 = fb_out[0], F1 = fb_out[1], F2_ = fb_out[2], F3 = fb_out[3], F4 = fb_out[4];
    const V F5 = fb_out[5], F6 = fb_out[6], F7 = fb_out[7], F8 = fb_out[8];
    const V Sax = (F1 + F2_) + (F3 + F4), Sdg = (F5 + F6) + (F7 + F8);
    const V ab0 = F0 + Sax + Sdg;
    const V ab1 = V(-4) * F0 - Sax + V(2) * Sdg;
    const V ab2 = V(4) * F0 - V(2) * Sax + Sdg;
    const V ab3 = (F1 - F3) + (F5 - F6) - (F7 - F8);
    const V ab4 = V(-2) * (F1 - F3) + (F5 - F6) - (F7 - F8);
    const V ab5 = (F2_ - F4) + (F5 + F6) - (F7 + F8);
    const V ab6 = V(-2) * (F2_ - F4) + (F5 + F6) - (F7 + F8);
    const V ab7 = (F1 + F3) - (F2_ + F4);
    const V ab8 = (F5 + F7) - (F6 + F8);
    rhob = rhob + ab0 * V(1.0 / 9.0);
    const V esb = ab1 * V(1.0 / 36.0), epsb = ab2 * V(1.0 / 36.0);
    const V jxsb = ab3 * V(1.0 / 6.0), qxsb = ab4 * V(1.0 / 12.0);
    const V jysb = ab5 * V(1.0 / 6.0), qysb = ab6 * V(1.0 / 12.0);
    const V pxxsb = ab7 * V(0.25), pxysb = ab8 * V(0.25);
    // post-collision moments
    V eb = V(-0.4) * esb, e_eqb = V(1.4) * esb, Feb = V(0.3) * esb;
    V epb = V(-0.4) * epsb, ep_eqb = V(1.4) * epsb;
    Feb = Feb - V(0.3) * epsb;
    V Fxb = V(0), Fyb = V(0);
    rhob = rhob + (ux + V(0.5) * Fx) * jxsb + (uy + V(0.5) * Fy) * jysb;
    uxb = uxb + rho * jxsb;
    uyb = uyb + rho * jysb;
    Fxb = Fxb + V(0.5) * rho * jxsb;
    Fyb = Fyb + V(0.5) * rho * jysb;
    V qxb = V(-0.2) * qxsb, qyb = V(-0.2) * qysb;
    rhob = rhob + (V(-1.2) * ux - V(0.4) * Fx) * qxsb + (V(-1.2) * uy - V(0.4) * Fy) * qysb;
    uxb = uxb - V(1.2) * rho * qxsb;
    uyb = uyb - V(1.2) * rho * qysb;
    Fxb = Fxb - V(0.4) * rho * qxsb;
    Fyb = Fyb - V(0.4) * rho * qysb;
    V pxxb = (V(1) - w) * pxxsb, pxyb = (V(1) - w) * pxysb;
    V pxx_eqb = w * pxxsb, pxy_eqb = w * pxysb;
    const V Fxxb = hw * pxxsb, Fxyb = hw * pxysb;
    V wb = (pxx_eq - pxx - V(0.5) * Fxx) * pxxsb + (pxy_eq - pxy - V(0.5) * Fxy) * pxysb;
    // forcing moments
    V rieb = V(6) * uF * Feb + V(2) * vfma(ux, Fx, -(uy * Fy)) * Fxxb + vfma(ux, Fy, uy * Fx) * Fxyb;
    const V uFb = V(6) * rie * Feb;
    uxb = uxb + V(2) * rie * Fx * Fxxb + rie * Fy * Fxyb + Fx * uFb;
    uyb = uyb - V(2) * rie * Fy * Fxxb + rie * Fx * Fxyb + Fy * uFb;
    Fxb = Fxb + V(2) * rie * ux * Fxxb + rie * uy * Fxyb + ux * uFb;
    Fyb = Fyb - V(2) * rie * uy * Fxxb + rie * ux * Fxyb + uy * uFb;
    // relaxation time of this collision: w = 1/tau, tau = 3 nu + 1/2, nu = nu_ref D
    V taub = taub_new - w * w * wb;
    const V nub = V(3) * taub;
    pa.nu_ref = D * nub;
    const V Db = p.nu_ref * nub;
    pa.nm1 = dD_dnm1 * Db;
    const V gsb = dD_dgs * Db;
    const V gamb = p.gamma_scale * gsb;
    V irhob = V(3) * sQ * gamb;
    const V sQb = V(3) * irho * gamb;
    const V Qb = sQ > V(0) ? sQb * V(0.5) * vrcp(sQ) : V(0);
    const V Ab = V(2) * A * Qb, Bb = V(2) * B * Qb, Cb = V(2) * C * Qb;
    eb = eb + V(1.4 / 6.0) * Ab;
    e_eqb = e_eqb - V(1.4 / 6.0) * Ab;
    const V wpb = V(0.5) * (pxx - pxx_eq) * Bb + (pxy - pxy_eq) * Cb;
    pxxb = pxxb + V(0.5) * wp * Bb;
    pxx_eqb = pxx_eqb - V(0.5) * wp * Bb;
    pxyb = pxyb + wp * Cb;
    pxy_eqb = pxy_eqb - wp * Cb;
    V taupb = -wp * wp * wpb;
    // equilibria
    rhob = rhob + (u2e3 - V(2)) * e_eqb + (V(1) - u2e3) * ep_eqb;
    const V u2e3b = rho * e_eqb - rho * ep_eqb;
    rieb = rieb + vfma(ux, ux, -(uy * uy)) * pxx_eqb + ux * uy * pxy_eqb;
    uxb = uxb + V(2) * rie * ux * pxx_eqb + rie * uy * pxy_eqb + V(6) * p.inv_eps * ux * u2e3b;
    uyb = uyb - V(2) * rie * uy * pxx_eqb + rie * ux * pxy_eqb + V(6) * p.inv_eps * uy * u2e3b;
    rhob = rhob + p.inv_eps * rieb;
    // macro: forces and the porous velocity solve
    const V dragb = ux * Fxb + uy * Fyb;
    uxb = uxb + drag * Fxb;
    uyb = uyb + drag * Fyb;
    V Gyb = p.eps * Fyb;
    V nupb = -q.eK * dragb;
    const V umagb = -q.eFsK * dragb;
    pa.eK = -nu_prev * dragb;
    pa.eFsK = -umag * dragb;
    V vmagb = iden * umagb;
    V idenb = vmag * umagb + vx * uxb + vy * uyb;
    V vxb = iden * uxb, vyb = iden * uyb;
    const V denb = -iden * iden * idenb;
    V c0b = denb;
    const V sqb = denb;
    const V tb = sq > V(0) ? sqb * V(0.5) * vrcp(sq) : V(0);
    c0b = c0b + V(2) * c0 * tb;
    pa.c1 = vmag * tb;
    vmagb = vmagb + q.c1 * tb;
    if (vmag > V(0)) {
        const V iv = vrcp(vmag);
        vxb = vxb + vx * iv * vmagb;
        vyb = vyb + vy * iv * vmagb;
    }
    pa.heK = nu_prev * c0b;
    nupb = nupb + q.heK * c0b;
    taupb = taupb + nupb * V(1.0 / 3.0);
    Gyb = Gyb + p.half_eps * vyb;
    const V jyb = irho * vyb;
    const V jxb = irho * vxb;
    irhob = irhob + jy * vyb + jx * vxb;
    rhob = rhob - irho * irho * irhob;
    Tb = Tb + p.gbeta * Gyb;
    // raw moments m = M f: rows rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy
    const V mb[9] = {rhob, eb, epb, jxb, qxb, jyb, qyb, pxxb, pxyb};
    fb[0] = mb[0] - V(4) * mb[1] + V(4) * mb[2];
    fb[1] = mb[0] - mb[1] - V(2) * mb[2] + mb[3] - V(2) * mb[4] + mb[7];
    fb[2] = mb[0] - mb[1] - V(2) * mb[2] + mb[5] - V(2) * mb[6] - mb[7];
    fb[3] = mb[0] - mb[1] - V(2) * mb[2] - mb[3] + V(2) * mb[4] + mb[7];
    fb[4] = mb[0] - mb[1] - V(2) * mb[2] - mb[5] + V(2) * mb[6] - mb[7];
    fb[5] = mb[0] + V(2) * mb[1] + mb[2] + mb[3] + mb[4] + mb[5] + mb[6] + mb[8];
    fb[6] = mb[0] + V(2) * mb[1] + mb[2] - mb[3] - mb[4] + mb[5] + mb[6] - mb[8];
    fb[7] = mb[0] + V(2) * mb[1] + mb[2] - mb[3] - mb[4] - mb[5] - mb[6] + mb[8];
    fb[8] = mb[0] + V(2) * mb[1] + mb[2] + mb[3] + mb[4] - mb[5] - mb[6] - mb[8];
    for (int i = 0; i < 5; i++) gb[i] = gbl[i] + Tb;
    taub_prev = taupb;
}

}  // namespace lbm
