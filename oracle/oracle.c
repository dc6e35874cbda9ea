/*
 * oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * Slow on purpose: every node builds its moment vectors with full 9x9 and
 * 5x5 matrix products, and the strain rate is the literal double sum of the
 * paper's strain-rate equation.  Nothing here is blocked, fused or reordered
 * beyond what the equations state.
 *
 * Parity status of every function is recorded in the header of each block
 * below ("pinned by" names the CPU tests that fix it independently).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------------
 * Lattices.
 * D2Q9 velocities in the order of Eq. (particleSpeedMatrix), section
 * "Multiple-Relaxation-Time Lattice Boltzmann Method":
 * e0 = (0,0); e1..e4 = (1,0),(0,1),(-1,0),(0,-1); e5..e8 = (1,1),(-1,1),
 * (-1,-1),(1,-1).  D2Q5 velocities of the thermal section: e0..e4 = the first
 * five of the above.  Weights are the standard ones for c_s^2 = 1/3.
 * Pinned by: test_oracle_matrices (moment sums), the BGK reductions.
 * ------------------------------------------------------------------------- */
static const int EX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double W9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static const int EX5[5] = {0, 1, 0, -1, 0};
static const int EY5[5] = {0, 0, 1, 0, -1};
static const int OPP5[5] = {0, 3, 4, 1, 2};
static const double W5[5] = {1.0 / 3, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6};

/* ---------------------------------------------------------------------------
 * Transformation matrices.
 * M: the D2Q9 moment basis (rho, e, epsilon, j_x, q_x, j_y, q_y, p_xx, p_xy),
 * ordered to match the relaxation rates s0..s8 of Eq. (collisionMatrix).
 * N: the 5x5 D2Q5 matrix of Eq. (thermalMRTequation), rows
 * (T, j_x, j_y, e, p_xx).  Both inverses come from Gauss-Jordan elimination.
 * Pinned by: M M^-1 = I, N N^-1 = I, and the exact integer row norms
 * M M^T = diag(9,36,36,6,12,6,12,4,4), N N^T = diag(5,2,2,20,4).
 * ------------------------------------------------------------------------- */
static const double MROWS[81] = {
    1, 1, 1, 1, 1, 1, 1, 1, 1,
    -4, -1, -1, -1, -1, 2, 2, 2, 2,
    4, -2, -2, -2, -2, 1, 1, 1, 1,
    0, 1, 0, -1, 0, 1, -1, -1, 1,
    0, -2, 0, 2, 0, 1, -1, -1, 1,
    0, 0, 1, 0, -1, 1, 1, -1, -1,
    0, 0, -2, 0, 2, 1, 1, -1, -1,
    0, 1, -1, 1, -1, 0, 0, 0, 0,
    0, 0, 0, 0, 0, 1, -1, 1, -1};
static const double NROWS[25] = {
    1, 1, 1, 1, 1,
    0, 1, 0, -1, 0,
    0, 0, 1, 0, -1,
    -4, 1, 1, 1, 1,
    0, 1, -1, 1, -1};

/* In-place Gauss-Jordan inverse with partial pivoting of an n x n matrix. */
static void invert(const double *a, double *inv, int n)
{
    double w[81 * 2];
    int cols = 2 * n;
    for (int r = 0; r < n; r++)
        for (int c = 0; c < cols; c++)
            w[r * cols + c] = c < n ? a[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int p = 0; p < n; p++) {
        int best = p;
        for (int r = p + 1; r < n; r++)
            if (fabs(w[r * cols + p]) > fabs(w[best * cols + p])) best = r;
        if (best != p)
            for (int c = 0; c < cols; c++) {
                double t = w[p * cols + c];
                w[p * cols + c] = w[best * cols + c];
                w[best * cols + c] = t;
            }
        double piv = w[p * cols + p];
        for (int c = 0; c < cols; c++) w[p * cols + c] /= piv;
        for (int r = 0; r < n; r++) {
            if (r == p) continue;
            double fac = w[r * cols + p];
            for (int c = 0; c < cols; c++) w[r * cols + c] -= fac * w[p * cols + c];
        }
    }
    for (int r = 0; r < n; r++)
        for (int c = 0; c < n; c++) inv[r * n + c] = w[r * cols + n + c];
}

static double MINV[81], NINV[25];
static int matrices_ready = 0;

static void ensure_matrices(void)
{
    if (matrices_ready) return;
    invert(MROWS, MINV, 9);
    invert(NROWS, NINV, 5);
    matrices_ready = 1;
}

void orc_matrices(double M[81], double Minv[81], double N[25], double Ninv[25])
{
    ensure_matrices();
    if (M) memcpy(M, MROWS, sizeof(MROWS));
    if (Minv) memcpy(Minv, MINV, sizeof(MINV));
    if (N) memcpy(N, NROWS, sizeof(NROWS));
    if (Ninv) memcpy(Ninv, NINV, sizeof(NINV));
}

static void matvec(const double *A, const double *x, double *y, int n)
{
    for (int r = 0; r < n; r++) {
        double acc = 0.0;
        for (int c = 0; c < n; c++) acc += A[r * n + c] * x[c];
        y[r] = acc;
    }
}

/* ---------------------------------------------------------------------------
 * Equilibria and forcing.
 * Moment-space flow equilibrium m^eq of the generalized porous model
 * (porosity eps enters the quadratic velocity terms; eps = 1 is the plain
 * fluid):  (rho, rho(-2 + 3|u|^2/eps), rho(1 - 3|u|^2/eps), rho u_x,
 * -rho u_x, rho u_y, -rho u_y, rho(u_x^2 - u_y^2)/eps, rho u_x u_y/eps).
 * Pinned by: M f^eq(velocity space) = m^eq, and the velocity-space moments
 * sum f = rho, sum f e = rho u, sum f e e = rho(I/3 + u u / eps).
 * ------------------------------------------------------------------------- */
void orc_meq(double rho, double ux, double uy, double eps, double out[9])
{
    double u2 = ux * ux + uy * uy;
    out[0] = rho;
    out[1] = rho * (-2.0 + 3.0 * u2 / eps);
    out[2] = rho * (1.0 - 3.0 * u2 / eps);
    out[3] = rho * ux;
    out[4] = -rho * ux;
    out[5] = rho * uy;
    out[6] = -rho * uy;
    out[7] = rho * (ux * ux - uy * uy) / eps;
    out[8] = rho * ux * uy / eps;
}

/* Velocity-space equilibrium w_i rho [1 + 3 e.u + 9 (e.u)^2 / (2 eps)
 * - 3 |u|^2 / (2 eps)], used in the literal strain-rate sum. */
void orc_feq(double rho, double ux, double uy, double eps, double out[9])
{
    double u2 = ux * ux + uy * uy;
    for (int i = 0; i < 9; i++) {
        double eu = EX9[i] * ux + EY9[i] * uy;
        out[i] = W9[i] * rho *
                 (1.0 + 3.0 * eu + 4.5 * eu * eu / eps - 1.5 * u2 / eps);
    }
}

/* Velocity-space body-force term of the generalized model (without the
 * (1 - S/2) factor, which Eq. (normalMRTequation) applies in moment space):
 * F_i = w_i rho [3 e.F + 9 (e.u)(e.F)/eps - 3 u.F/eps].
 * Pinned by: the MRT -> BGK reduction with forcing (all rates equal). */
void orc_forcing_vel(double rho, double ux, double uy, double Fx, double Fy,
                     double eps, double out[9])
{
    double uF = ux * Fx + uy * Fy;
    for (int i = 0; i < 9; i++) {
        double eF = EX9[i] * Fx + EY9[i] * Fy;
        double eu = EX9[i] * ux + EY9[i] * uy;
        out[i] = W9[i] * rho * (3.0 * eF + 9.0 * eu * eF / eps - 3.0 * uF / eps);
    }
}

/* ---------------------------------------------------------------------------
 * Modified power law, Eq. (MPL).  nu = nu_0 D with D the apparent-viscosity
 * factor of the non-dimensional shear rate gamma*:
 *   clamp_mode 0 (literal): D = 1 below gamma1, gamma*^(n-1) on
 *                           [gamma1, gamma2], gamma2^(n-1) above gamma2;
 *   clamp_mode 1:           D = clamp(gamma*, gamma1, gamma2)^(n-1).
 * Pinned by: n = 1 gives nu = nu_0 everywhere; the power-law channel.
 * ------------------------------------------------------------------------- */
static double apparent_factor(const orc_lattice *p, double gstar)
{
    if (p->clamp_mode == 0) {
        if (gstar < p->gamma1) return 1.0;
        if (gstar <= p->gamma2) return pow(gstar, p->n - 1.0);
        return pow(p->gamma2, p->n - 1.0);
    }
    double gc = gstar;
    if (gc < p->gamma1) gc = p->gamma1;
    if (gc > p->gamma2) gc = p->gamma2;
    return pow(gc, p->n - 1.0);
}

/* ---------------------------------------------------------------------------
 * One node: macroscopic moments, porous velocity solve, strain rate,
 * viscosity, flow MRT collision with forcing (Eq. normalMRTequation) and
 * thermal MRT collision (Eq. thermalMRTequation).
 *
 * Steps, in the order the equations use them:
 *  1. rho = sum f_i (Eq. macro_fluid_density), T = sum g_i.
 *  2. Buoyancy acceleration G = g beta (T - T_m) along +y (Eq. velo), plus
 *     any uniform x body acceleration.
 *  3. v = sum f_i e_i / rho + eps G / 2 (half-force shift of Eq. velo).
 *  4. Porous solve: u = v / (c0 + sqrt(c0^2 + c1 |v|)), with
 *     c0 = (1 + eps nu / (2K)) / 2, c1 = eps F_eps / (2 sqrt K), and nu the
 *     apparent viscosity of the relaxation time tau_in that the collision
 *     starts from (the lagged tau_prev, or the node-local implicit solve).
 *  5. Total force per unit mass F = -eps nu u / K - eps F_eps |u| u / sqrt K
 *     + eps G (Darcy drag with the apparent viscosity as in the
 *     non-dimensional momentum equations, Forchheimer, buoyancy).
 *  6. Strain rate gamma_ab = -3/(2 rho) sum_i e_ia e_ib
 *     sum_j (M^-1 S M)_ij (f_j - f_j^eq), with s7 = s8 = 1/tau_in, and
 *     |gamma| = sqrt(2 gamma_ab gamma_ab).
 *  7. gamma* = |gamma| gamma_scale, nu = nu_ref D(gamma*), tau = 3 nu + 1/2.
 *  8. m* = m - S (m - m^eq) + (I - S/2) M F_vel with s7 = s8 = 1/tau;
 *     f* = M^-1 m*.
 *  9. n = N g, n^eq = (T, T u_x, T u_y, -2T/3, 0),
 *     n* = n - S_T (n - n^eq), S_T = diag(1, 1/tauT, 1/tauT, s_e, s_p);
 *     g* = N^-1 n*.
 * Steps 1-6 are strain_state(); steps 7-9 node_update().
 * ------------------------------------------------------------------------- */
typedef struct {
    double rho, ux, uy, T, nu, gamma;
} node_diag;

typedef struct {
    double rho, T, ux, uy, Fx, Fy;
    double gamma;  /* |gamma| of step 6                                   */
    double R;      /* d ln|gamma| / d ln(1/tau_in) at fixed velocity:
                      omega (gamma : gamma_p) / (gamma : gamma), where
                      gamma_p is the strain tensor of step 6 with S replaced
                      by diag(0, ..., 0, 1, 1) (the part that scales with
                      omega = 1/tau_in); 0 where gamma = 0 or when not
                      asked for                                          */
} strain_out;

static void strain_state(const orc_lattice *p, double K, const double f[9],
                         const double g[5], double tau_in, int want_R, strain_out *o)
{
    ensure_matrices();
    /* 1 */
    double rho = 0.0, jx = 0.0, jy = 0.0, T = 0.0;
    for (int i = 0; i < 9; i++) {
        rho += f[i];
        jx += f[i] * EX9[i];
        jy += f[i] * EY9[i];
    }
    for (int i = 0; i < 5; i++) T += g[i];
    /* 2 */
    double Gx = p->Gx;
    double Gy = p->gbeta * (T - p->Tm);
    /* 3 */
    double vx = jx / rho + 0.5 * p->eps * Gx;
    double vy = jy / rho + 0.5 * p->eps * Gy;
    /* 4 */
    double nu_in = (tau_in - 0.5) / 3.0;
    double c0 = 0.5 * (1.0 + p->eps * nu_in / (2.0 * K));
    double c1 = p->eps * p->Feps / (2.0 * sqrt(K));
    double vmag = sqrt(vx * vx + vy * vy);
    double den = c0 + sqrt(c0 * c0 + c1 * vmag);
    double ux = vx / den, uy = vy / den;
    /* 5 */
    double umag = sqrt(ux * ux + uy * uy);
    double Fx = -p->eps * nu_in * ux / K
                - p->eps * p->Feps * umag * ux / sqrt(K) + p->eps * Gx;
    double Fy = -p->eps * nu_in * uy / K
                - p->eps * p->Feps * umag * uy / sqrt(K) + p->eps * Gy;
    /* 6 */
    double feq[9], fneq[9], S[9], P[9], A[81], Ap[81], tmp[81], tmpp[81], h[9], hp[9];
    orc_feq(rho, ux, uy, p->eps, feq);
    for (int i = 0; i < 9; i++) fneq[i] = f[i] - feq[i];
    for (int i = 0; i < 9; i++) {
        S[i] = p->s[i];
        P[i] = 0.0;
    }
    S[7] = S[8] = 1.0 / tau_in;
    P[7] = P[8] = 1.0;
    for (int r = 0; r < 9; r++) /* tmp = S M, tmpp = P M */
        for (int c = 0; c < 9; c++) {
            tmp[r * 9 + c] = S[r] * MROWS[r * 9 + c];
            tmpp[r * 9 + c] = P[r] * MROWS[r * 9 + c];
        }
    for (int r = 0; r < 9; r++) /* A = M^-1 (S M), Ap = M^-1 (P M) */
        for (int c = 0; c < 9; c++) {
            double acc = 0.0, accp = 0.0;
            for (int k = 0; k < 9; k++) {
                acc += MINV[r * 9 + k] * tmp[k * 9 + c];
                if (want_R) accp += MINV[r * 9 + k] * tmpp[k * 9 + c];
            }
            A[r * 9 + c] = acc;
            Ap[r * 9 + c] = accp;
        }
    matvec(A, fneq, h, 9);
    matvec(Ap, fneq, hp, 9);
    double gab[2][2], gabp[2][2];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) {
            double acc = 0.0, accp = 0.0;
            for (int i = 0; i < 9; i++) {
                double ea = a == 0 ? EX9[i] : EY9[i];
                double eb = b == 0 ? EX9[i] : EY9[i];
                acc += ea * eb * h[i];
                accp += ea * eb * hp[i];
            }
            gab[a][b] = -3.0 / (2.0 * rho) * acc; /* c = 1 */
            gabp[a][b] = -3.0 / (2.0 * rho) * accp;
        }
    double gg = 0.0, ggp = 0.0;
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) {
            gg += gab[a][b] * gab[a][b];
            ggp += gab[a][b] * gabp[a][b];
        }
    o->rho = rho;
    o->T = T;
    o->ux = ux;
    o->uy = uy;
    o->Fx = Fx;
    o->Fy = Fy;
    o->gamma = sqrt(2.0 * gg);
    o->R = want_R && gg > 0.0 ? (1.0 / tau_in) * ggp / gg : 0.0;
}

/* ---------------------------------------------------------------------------
 * Node-local implicit relaxation time (an extension: the paper does not say
 * how the tau used in the strain rate is obtained; the lagged reading uses
 * the node's previous tau).  The implicit tau is the root of
 *   tau = Phi(tau),  Phi(tau) = 3 nu_ref D(gamma*(tau)) + 1/2,
 * with gamma(tau) = steps 1-6 above taken with tau_in = tau.  It is found by
 * p->tau_iters Newton steps on ln tau, starting from the rest-state tau0:
 *   J_k = 1 - (1 - n) R_k (Phi_k - 1/2) / Phi_k   where D has slope, i.e.
 *         gamma1 < gamma* < gamma2,  else J_k = 1,
 *   tau_{k+1} = tau_k (Phi_k / tau_k)^(1 / J_k)
 * (d ln Phi / d ln tau = -(n - 1) R (Phi - 1/2) / Phi with the velocity held;
 * the slope of the drag through the velocity is left out of J only, so the
 * root is exact but convergence there is linear with a small rate).
 * J lies between n and 1, so the step is defined for every n > 0.
 * Pinned by: n = 1 reproduces the lagged update bit for bit; the converged
 * tau satisfies tau = Phi(tau) and equals the root found by bisection on
 * ln tau; a lagged steady state is a fixed point of the implicit step.
 * ------------------------------------------------------------------------- */
static double phi_of(const orc_lattice *p, double K, const double f[9],
                     const double g[5], double tau, double *J)
{
    strain_out st;
    strain_state(p, K, f, g, tau, J != NULL, &st);
    double gs = st.gamma * p->gamma_scale;
    double phi = 3.0 * p->nu_ref * apparent_factor(p, gs) + 0.5;
    if (J) {
        if (gs > p->gamma1 && gs < p->gamma2)
            *J = 1.0 - (1.0 - p->n) * st.R * (phi - 0.5) / phi;
        else
            *J = 1.0;
    }
    return phi;
}

static double implicit_tau(const orc_lattice *p, double K, const double f[9],
                           const double g[5])
{
    double tau = p->tau0;
    for (int it = 0; it < p->tau_iters; it++) {
        double J;
        double phi = phi_of(p, K, f, g, tau, &J);
        if (J == 1.0)
            tau = phi;
        else
            tau = tau * pow(phi / tau, 1.0 / J);
    }
    return tau;
}

static void node_update(const orc_lattice *p, double K, const double f[9],
                        const double g[5], double tau_in, double fo[9],
                        double go[5], double *tau_new, node_diag *d)
{
    strain_out st;
    strain_state(p, K, f, g, tau_in, 0, &st);
    double rho = st.rho, T = st.T, ux = st.ux, uy = st.uy;
    /* 7 */
    double nu_new = p->nu_ref * apparent_factor(p, st.gamma * p->gamma_scale);
    double tau = 3.0 * nu_new + 0.5;
    /* 8 */
    double m[9], meq[9], Fv[9], Fh[9], ms[9], S[9];
    for (int i = 0; i < 9; i++) S[i] = p->s[i];
    matvec(MROWS, f, m, 9);
    orc_meq(rho, ux, uy, p->eps, meq);
    orc_forcing_vel(rho, ux, uy, st.Fx, st.Fy, p->eps, Fv);
    matvec(MROWS, Fv, Fh, 9);
    S[7] = S[8] = 1.0 / tau;
    for (int k = 0; k < 9; k++)
        ms[k] = m[k] - S[k] * (m[k] - meq[k]) + (1.0 - 0.5 * S[k]) * Fh[k];
    matvec(MINV, ms, fo, 9);
    /* 9 */
    double nT[5], nTeq[5], ST[5], nTs[5];
    matvec(NROWS, g, nT, 5);
    nTeq[0] = T;
    nTeq[1] = T * ux;
    nTeq[2] = T * uy;
    nTeq[3] = -2.0 * T / 3.0;
    nTeq[4] = 0.0;
    ST[0] = 1.0;
    ST[1] = ST[2] = 1.0 / p->tauT;
    ST[3] = p->s_e;
    ST[4] = p->s_p;
    for (int k = 0; k < 5; k++) nTs[k] = nT[k] - ST[k] * (nT[k] - nTeq[k]);
    matvec(NINV, nTs, go, 5);

    *tau_new = tau;
    if (d) {
        d->rho = rho;
        d->ux = ux;
        d->uy = uy;
        d->T = T;
        d->nu = nu_new;
        d->gamma = st.gamma;
    }
}

/* tau the collision of a node starts from: the stored lagged tau, or the
 * implicit solve when tau_iters > 0. */
static double tau_start(const orc_lattice *p, double K, const double f[9],
                        const double g[5], double tau_stored)
{
    return p->tau_iters > 0 ? implicit_tau(p, K, f, g) : tau_stored;
}

double orc_phi(const orc_lattice *lat, const double f[9], const double g[5],
               double tau, double *J)
{
    return phi_of(lat, lat->K, f, g, tau, J);
}

double orc_implicit_tau(const orc_lattice *lat, const double f[9], const double g[5])
{
    return implicit_tau(lat, lat->K, f, g);
}

void orc_collide_node(const orc_lattice *lat, const double f[9],
                      const double g[5], double tau_prev, double fo[9],
                      double go[5], double *tau_new, double *gamma)
{
    node_diag d;
    node_update(lat, lat->K, f, g, tau_prev, fo, go, tau_new, &d);
    if (gamma) *gamma = d.gamma;
}

/* ---------------------------------------------------------------------------
 * Lattice-unit mapping of the non-dimensional problem (the paper defers the
 * mapping to earlier work, so this is a stated reading):
 *   U_c = Ma c_s (c_s = 1/sqrt 3), L = nx (hot-to-cold distance);
 *   thermal diffusivity alpha = U_c L / sqrt(Ra), tauT = 3 alpha + 1/2
 *     (energy equation with diffusivity 1/sqrt(Ra));
 *   nu_0 = Pr / sqrt(Ra)^(2-n) (power-law section), nu_ref = nu_0 U_c L;
 *   gamma* = |gamma| L / U_c;
 *   g beta (T_h - T_c) = Pr U_c^2 / L (buoyancy Pr theta of the
 *     non-dimensional v-momentum equation), T_m = (T_h + T_c) / 2;
 *   K = Da L^2;  tau = 3 nu + 1/2 (Eq. kinematic_viscosity, c_s^2 = 1/3).
 * Porous model 1 uses the Ergun factor F_eps = 1.75 / sqrt(150 eps^3).
 * Pinned by tests/test_oracle_mapping.py, which measures the viscosity a
 * sheared node takes, the momentum one collision adds through buoyancy and
 * drag, and the diffusion rate of transient conduction, and checks them
 * against the dimensional groups of Eq. (non_dim_var), the non-dimensional
 * equations, Eq. (MPL) and a Fourier-series conduction solution.
 * ------------------------------------------------------------------------- */
int orc_map_params(int nx, int ny, double n, double Da, double Ra, double Pr,
                   double porosity, double Ma, int porous_model,
                   int clamp_mode, double s_e, double s_p, orc_lattice *o)
{
    if (!o || nx < 2 || ny < 2 || !(n > 0) || !(Da > 0) || !(Ra > 0) ||
        !(Pr > 0) || !(porosity > 0) || porosity > 1 || !(Ma > 0) ||
        (porous_model != 0 && porous_model != 1) ||
        (clamp_mode != 0 && clamp_mode != 1) || !(s_e > 0) || !(s_p > 0))
        return -1;
    memset(o, 0, sizeof(*o));
    double Uc = Ma / sqrt(3.0);
    double L = (double)nx;
    o->nx = nx;
    o->ny = ny;
    o->n = n;
    double nu0 = Pr / pow(sqrt(Ra), 2.0 - n);
    o->nu_ref = nu0 * Uc * L;
    o->gamma_scale = L / Uc;
    o->gamma1 = 0.01;
    o->gamma2 = 1.0e6;
    o->clamp_mode = clamp_mode;
    o->K = Da * L * L;
    if (porous_model == 1) {
        o->eps = porosity;
        o->Feps = 1.75 / sqrt(150.0 * porosity * porosity * porosity);
    } else {
        o->eps = 1.0;
        o->Feps = 0.0;
    }
    o->T_hot = 1.0;
    o->T_cold = 0.0;
    o->Tm = 0.5 * (o->T_hot + o->T_cold);
    o->gbeta = Pr * Uc * Uc / L / (o->T_hot - o->T_cold);
    o->Gx = 0.0;
    double alpha = Uc * L / sqrt(Ra);
    o->tauT = 3.0 * alpha + 0.5;
    double s[9] = {1.0, 1.4, 1.4, 1.0, 1.2, 1.0, 1.2, 0.0, 0.0};
    memcpy(o->s, s, sizeof(s));
    o->s_e = s_e;
    o->s_p = s_p;
    o->periodic_x = 0;
    o->L = L;
    o->rho0 = 1.0;
    o->T0 = o->Tm;
    o->tau0 = 3.0 * o->nu_ref * apparent_factor(o, 0.0) + 0.5;
    return 0;
}

/* ---------------------------------------------------------------------------
 * Run state and push streaming.
 * ------------------------------------------------------------------------- */
struct orc_ctx {
    orc_lattice p;
    size_t nn;
    double *f, *g, *tau;  /* post-collision state          */
    double *fs, *gs;      /* streamed (pre-collision) work */
    double *Kf;           /* per-node permeability or NULL */
};

static double K_at(const orc_ctx *c, size_t q) { return c->Kf ? c->Kf[q] : c->p.K; }

/* Per-node permeability K(x) = Da(x) L^2 (reading R17 of the Darcy term of
 * the momentum equations, node by node).  Pinned by: a uniform field equals
 * the uniform-K run bit for bit (and the uniform K is pinned against
 * Da = K / L^2), and a field differing at one node changes that node's
 * collision into the one of a uniform run at the node's Da and no other. */
void orc_set_darcy_field(orc_ctx *c, const double *Da)
{
    if (!Da) {
        free(c->Kf);
        c->Kf = NULL;
        return;
    }
    if (!c->Kf) c->Kf = (double *)malloc(sizeof(double) * c->nn);
    for (size_t q = 0; q < c->nn; q++) c->Kf[q] = Da[q] * c->p.L * c->p.L;
}

int orc_create(orc_ctx **out, const orc_lattice *lat)
{
    if (!out || !lat || lat->nx < 1 || lat->ny < 1) return -1;
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    if (!c) return -2;
    ensure_matrices(); /* before any parallel region reads them */
    c->p = *lat;
    c->nn = (size_t)lat->nx * lat->ny;
    c->f = (double *)malloc(sizeof(double) * 9 * c->nn);
    c->g = (double *)malloc(sizeof(double) * 5 * c->nn);
    c->tau = (double *)malloc(sizeof(double) * c->nn);
    c->fs = (double *)malloc(sizeof(double) * 9 * c->nn);
    c->gs = (double *)malloc(sizeof(double) * 5 * c->nn);
    if (!c->f || !c->g || !c->tau || !c->fs || !c->gs) {
        orc_destroy(c);
        return -2;
    }
    /* Rest state: f = f^eq(rho0, 0), g = g^eq(T0, 0), tau = tau0. */
    for (int i = 0; i < 9; i++)
        for (size_t k = 0; k < c->nn; k++) c->f[i * c->nn + k] = W9[i] * lat->rho0;
    for (int i = 0; i < 5; i++)
        for (size_t k = 0; k < c->nn; k++) c->g[i * c->nn + k] = W5[i] * lat->T0;
    for (size_t k = 0; k < c->nn; k++) c->tau[k] = lat->tau0;
    *out = c;
    return 0;
}

void orc_destroy(orc_ctx *c)
{
    if (!c) return;
    free(c->f);
    free(c->g);
    free(c->tau);
    free(c->fs);
    free(c->gs);
    free(c->Kf);
    free(c);
}

void orc_get_lattice(const orc_ctx *c, orc_lattice *out) { *out = c->p; }

/* Push every post-collision population one link along its velocity.  A link
 * that would leave the domain crosses a wall halfway between the boundary node
 * and the wall and returns to the node it left:
 *   flow: halfway bounce-back on a resting wall, f_opp(x) = f*_i(x);
 *   heat: left/right walls (Dirichlet) anti-bounce-back,
 *         g_opp(x) = -g*_i(x) + 2 w_opp T_wall; top/bottom (adiabatic)
 *         bounce-back, g_opp(x) = g*_i(x).
 * With periodic_x the x coordinate wraps instead. */
static void stream(const orc_ctx *c, double *fs, double *gs)
{
    const orc_lattice *p = &c->p;
    int nx = p->nx, ny = p->ny;
    size_t nn = c->nn;
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            size_t k = (size_t)y * nx + x;
            for (int i = 0; i < 9; i++) {
                int xd = x + EX9[i], yd = y + EY9[i];
                if (p->periodic_x) xd = (xd + nx) % nx;
                double val = c->f[i * nn + k];
                if (xd >= 0 && xd < nx && yd >= 0 && yd < ny)
                    fs[i * nn + (size_t)yd * nx + xd] = val;
                else
                    fs[OPP9[i] * nn + k] = val;
            }
            for (int i = 0; i < 5; i++) {
                int xd = x + EX5[i], yd = y + EY5[i];
                if (p->periodic_x) xd = (xd + nx) % nx;
                double val = c->g[i * nn + k];
                if (xd >= 0 && xd < nx && yd >= 0 && yd < ny)
                    gs[i * nn + (size_t)yd * nx + xd] = val;
                else if (xd < 0)
                    gs[OPP5[i] * nn + k] = -val + 2.0 * W5[OPP5[i]] * p->T_hot;
                else if (xd >= nx)
                    gs[OPP5[i] * nn + k] = -val + 2.0 * W5[OPP5[i]] * p->T_cold;
                else
                    gs[OPP5[i] * nn + k] = val;
            }
        }
}

static void gather(const double *a, int planes, size_t nn, size_t k, double *out)
{
    for (int i = 0; i < planes; i++) out[i] = a[i * nn + k];
}

int orc_step(orc_ctx *c, int64_t k)
{
    size_t nn = c->nn;
    for (int64_t t = 0; t < k; t++) {
        stream(c, c->fs, c->gs);
#pragma omp parallel for schedule(static)
        for (long q = 0; q < (long)nn; q++) {
            double f[9], g[5], fo[9], go[5], tnew;
            gather(c->fs, 9, nn, (size_t)q, f);
            gather(c->gs, 5, nn, (size_t)q, g);
            double Kq = K_at(c, (size_t)q);
            node_update(&c->p, Kq, f, g, tau_start(&c->p, Kq, f, g, c->tau[q]), fo, go, &tnew, NULL);
            for (int i = 0; i < 9; i++) c->f[i * nn + q] = fo[i];
            for (int i = 0; i < 5; i++) c->g[i * nn + q] = go[i];
            if (c->p.tau_iters == 0) c->tau[q] = tnew; /* implicit runs keep no tau */
        }
    }
    return 0;
}

void orc_get_state(const orc_ctx *c, double *f, double *g, double *tau)
{
    if (f) memcpy(f, c->f, sizeof(double) * 9 * c->nn);
    if (g) memcpy(g, c->g, sizeof(double) * 5 * c->nn);
    if (tau) memcpy(tau, c->tau, sizeof(double) * c->nn);
}

void orc_set_state(orc_ctx *c, const double *f, const double *g, const double *tau)
{
    if (f) memcpy(c->f, f, sizeof(double) * 9 * c->nn);
    if (g) memcpy(c->g, g, sizeof(double) * 5 * c->nn);
    if (tau) memcpy(c->tau, tau, sizeof(double) * c->nn);
}

void orc_fields(const orc_ctx *c, double *rho, double *ux, double *uy,
                double *T, double *nu, double *gamma)
{
    size_t nn = c->nn;
    double *fs = (double *)malloc(sizeof(double) * 9 * nn);
    double *gs = (double *)malloc(sizeof(double) * 5 * nn);
    if (!fs || !gs) {
        free(fs);
        free(gs);
        return;
    }
    stream(c, fs, gs);
    for (size_t q = 0; q < nn; q++) {
        double f[9], g[5], fo[9], go[5], tnew;
        node_diag d;
        gather(fs, 9, nn, q, f);
        gather(gs, 5, nn, q, g);
        node_update(&c->p, K_at(c, q), f, g, tau_start(&c->p, K_at(c, q), f, g, c->tau[q]), fo, go,
                    &tnew, &d);
        if (rho) rho[q] = d.rho;
        if (ux) ux[q] = d.ux;
        if (uy) uy[q] = d.uy;
        if (T) T[q] = d.T;
        if (nu) nu[q] = d.nu;
        if (gamma) gamma[q] = d.gamma;
    }
    free(fs);
    free(gs);
}

/* ---------------------------------------------------------------------------
 * Average Nusselt number, Eq. (avgNu): Nu(Y) = -d theta / dX at X = 0 and
 * its mean over the wall.  The derivative at the halfway wall is the
 * second-order one-sided difference through the wall value and the first two
 * node temperatures (at 1/2 and 3/2 lattice units from the wall):
 *   d theta/dx|wall = (9 theta_0 - theta_1 - 8 theta_w) / 3,
 * scaled by L to non-dimensional X.  The wall integral is the midpoint sum.
 * The cold wall uses the mirror formula (outward flux).
 * Pinned by: the conduction limit (Nu = 1 exactly for a linear profile).
 * ------------------------------------------------------------------------- */
void orc_nusselt(const orc_ctx *c, double *hot, double *cold, double *nu_local)
{
    const orc_lattice *p = &c->p;
    int nx = p->nx, ny = p->ny;
    size_t nn = c->nn;
    double *fs = (double *)malloc(sizeof(double) * 9 * nn);
    double *gs = (double *)malloc(sizeof(double) * 5 * nn);
    if (!fs || !gs) {
        free(fs);
        free(gs);
        return;
    }
    stream(c, fs, gs);
    double dT = p->T_hot - p->T_cold;
    double sh = 0.0, sc = 0.0;
    for (int y = 0; y < ny; y++) {
        double th[4];
        int cols[4] = {0, 1, nx - 1, nx - 2};
        for (int q = 0; q < 4; q++) {
            size_t k = (size_t)y * nx + cols[q];
            double T = 0.0;
            for (int i = 0; i < 5; i++) T += gs[i * nn + k];
            th[q] = (T - p->T_cold) / dT;
        }
        double nh = -p->L * (9.0 * th[0] - th[1] - 8.0 * 1.0) / 3.0;
        double nc = p->L * (9.0 * th[2] - th[3] - 8.0 * 0.0) / 3.0;
        if (nu_local) nu_local[y] = nh;
        sh += nh;
        sc += nc;
    }
    if (hot) *hot = sh / ny;
    if (cold) *cold = sc / ny;
    free(fs);
    free(gs);
}
