/*
 * oracle.h -- plain FP64 CPU oracle of the coupled MRT lattice Boltzmann
 * update for natural convection of a power-law fluid in a porous cavity
 * (Islam, Nag & Molla, ICME2019, "GPU Accelerated Lattice Boltzmann
 * Simulation of Non-Newtonian Power-Law Fluid in a Porous Enclosure").
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library
 * against a slow, literal restatement of the paper's algorithm.  Only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark may load
 * it.  It shares no code, header, table or helper with the CUDA path.
 *
 * Form: the literal moment-space MRT of Eq. (normalMRTequation) with explicit
 * 9x9 M and its inverse, the 5x5 thermal N and its inverse
 * (Eq. thermalMRTequation), the strain rate as the literal double sum over
 * (M^-1 S M)(f - f^eq) of the strain-rate equation in the power-law section,
 * the modified power law of Eq. (MPL), and push streaming with an explicit
 * per-link wall rule.  Arrays are [plane][y][x] with x fastest.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Lattice-unit parameters of one run.  orc_map_params fills them from the
 * paper's non-dimensional groups; tests may also fill them directly (e.g. the
 * channel-flow pins with periodic x and a body force). */
typedef struct {
    int    nx, ny;
    double n;            /* power-law index                                */
    double nu_ref;       /* lattice viscosity at D = 1  (nu_0 U_c L)       */
    double gamma_scale;  /* lattice |gamma| -> non-dimensional  (L / U_c)  */
    double gamma1;       /* lower shear-rate threshold (non-dimensional)   */
    double gamma2;       /* upper shear-rate threshold (non-dimensional)   */
    int    clamp_mode;   /* 0 literal Eq. MPL, 1 continuous clamp          */
    double K;            /* permeability in lattice units (may be +inf)    */
    double eps;          /* porosity                                       */
    double Feps;         /* Forchheimer geometric factor                   */
    double gbeta;        /* g*beta in lattice units (buoyancy per unit T)  */
    double Tm;           /* reference temperature of the buoyancy term     */
    double Gx;           /* extra uniform body acceleration along x        */
    double tauT;         /* thermal relaxation time                        */
    double s[9];         /* flow rates s0..s8 (s7, s8 set per node)        */
    double s_e, s_p;     /* thermal rates of the 4th and 5th moments       */
    int    periodic_x;   /* 1: periodic in x instead of side walls         */
    double T_hot, T_cold;/* Dirichlet wall temperatures (left, right)      */
    double L;            /* length unit for Nu (distance hot -> cold wall) */
    double tau0;         /* initial relaxation time                        */
    double rho0, T0;     /* initial density and temperature                */
    int    tau_iters;    /* 0: lagged tau (stored per node); k > 0: node-
                            local implicit tau by k Newton steps from tau0,
                            no stored tau (orc_implicit_tau)               */
} orc_lattice;

typedef struct orc_ctx orc_ctx;

/* Map the paper's groups (n, Da, Ra, Pr, porosity) and the Mach number to
 * lattice units.  porous_model 0: paper-literal Darcy drag (eps = 1, no
 * Forchheimer); 1: generalized (Brinkman-Forchheimer) porous model.
 * Returns 0, or -1 on an invalid argument. */
int orc_map_params(int nx, int ny, double n, double Da, double Ra, double Pr,
                   double porosity, double Ma, int porous_model,
                   int clamp_mode, double s_e, double s_p, orc_lattice *out);

int  orc_create(orc_ctx **out, const orc_lattice *lat);
void orc_destroy(orc_ctx *c);
void orc_get_lattice(const orc_ctx *c, orc_lattice *out);
/* Advance k time steps (push stream + collide). */
int  orc_step(orc_ctx *c, int64_t k);
/* State after the last collision: f[9][ny][nx], g[5][ny][nx], tau[ny][nx]. */
void orc_get_state(const orc_ctx *c, double *f, double *g, double *tau);
void orc_set_state(orc_ctx *c, const double *f, const double *g, const double *tau);
/* Streamed (pre-collision) macroscopic fields that the next collision sees:
 * density, velocity (after the porous solve), temperature, the apparent
 * lattice viscosity the next collision will use, and the lattice |gamma|.
 * Any pointer may be NULL. */
void orc_fields(const orc_ctx *c, double *rho, double *ux, double *uy,
                double *T, double *nu, double *gamma);
/* Hot- and cold-wall average Nusselt numbers from the streamed temperature;
 * nu_local (NULL or ny values) gets the hot-wall local Nu. */
void orc_nusselt(const orc_ctx *c, double *hot, double *cold, double *nu_local);

/* Per-node Darcy numbers (nx*ny values, [ny][nx]); K(x) = Da(x) L^2 replaces
 * the uniform K.  NULL restores the uniform permeability. */
void orc_set_darcy_field(orc_ctx *c, const double *Da);

/* Pieces exposed for the unit pins. */
void orc_matrices(double M[81], double Minv[81], double N[25], double Ninv[25]);
void orc_meq(double rho, double ux, double uy, double eps, double out[9]);
void orc_feq(double rho, double ux, double uy, double eps, double out[9]);
void orc_forcing_vel(double rho, double ux, double uy, double Fx, double Fy,
                     double eps, double out[9]);
/* One flow + thermal collision of a single node from streamed f, g and the
 * lagged tau.  Outputs post-collision f, g, the new tau and |gamma|. */
void orc_collide_node(const orc_lattice *lat, const double f[9],
                      const double g[5], double tau_prev, double fo[9],
                      double go[5], double *tau_new, double *gamma);

/* The implicit-tau map of one node (uniform K of lat): Phi(tau) =
 * 3 nu_ref D(gamma*(tau)) + 1/2, gamma(tau) the strain rate of the collision
 * started from tau; *J (may be NULL) receives the Newton factor
 * 1 - d ln Phi / d ln tau at fixed velocity (1 where D is flat). */
double orc_phi(const orc_lattice *lat, const double f[9], const double g[5],
               double tau, double *J);
/* lat->tau_iters Newton steps on ln tau from lat->tau0 toward tau = Phi(tau). */
double orc_implicit_tau(const orc_lattice *lat, const double f[9], const double g[5]);

#ifdef __cplusplus
}
#endif
#endif
