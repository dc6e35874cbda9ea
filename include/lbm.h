/*
 * lbm.h -- C ABI of the GB300 (sm_103a) fused MRT lattice Boltzmann step for
 * natural convection of a power-law fluid in a porous square cavity
 * (Islam, Nag & Molla, "GPU Accelerated Lattice Boltzmann Simulation of
 * Non-Newtonian Power-Law Fluid in a Porous Enclosure", ICME2019).
 *
 * The problem (section "Mathematical formulations"): a cavity of side L with
 * the left wall hot (theta = 1), the right wall cold (theta = 0), adiabatic
 * top and bottom walls and no-slip everywhere, filled with a porous medium
 * (Darcy number Da, porosity) saturated by a power-law fluid (index n), driven
 * by Boussinesq buoyancy (Rayleigh number Ra, Prandtl number Pr).
 *
 * Conventions for every call:
 *  - Return value 0 on success, a negative LBM_ERR_* code otherwise; no
 *    exception or signal crosses this boundary.  lbm_strerror() names a code.
 *  - A node (i, j) sits at x = i + 1/2, y = j + 1/2 in lattice units; the
 *    walls lie halfway between the boundary nodes and the domain edge.
 *    Every host array of per-node values is row-major [ny][nx] (x fastest).
 *  - Host buffers are owned by the caller and must stay valid for the call.
 *    Device memory is owned by the library (allocated in lbm_init, released
 *    in lbm_destroy); no device pointer is exposed.
 *  - lbm_step only enqueues work on the context's stream; every call that
 *    returns host data synchronises that stream before returning.
 *  - A context may be used by one host thread at a time.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,       /* invalid argument, size or state             */
    LBM_ERR_UNSTABLE = -2,  /* a relaxation time maps to <= 1/2 + 1e-6     */
    LBM_ERR_NONFINITE = -3, /* NaN or Inf found in the fields              */
    LBM_ERR_CUDA = -4,      /* a CUDA runtime call failed                  */
    LBM_ERR_OOM = -5,       /* device memory allocation failed             */
    LBM_ERR_TIMEOUT = -6,   /* a bounded device wait gave up (reserved: no
                               kernel of this version waits)          */
    LBM_ERR_UNSUPPORTED = -7,/* option combination not built              */
    LBM_ERR_SIZE = -8       /* grid larger than a fixed-size scratch area  */
};

/* Rows (ny) that lbm_residual_noalloc's fixed scratch area can serve. */
#define LBM_NOALLOC_MAX_ROWS 16384
#define LBM_TAU_ITERS_MAX 16   /* largest lbm_opts.tau_iters */

/* Storage precision of the distributions.  Arithmetic is FP64 for LBM_F64
 * and FP32 otherwise.  The *D forms store the deviation of each population
 * from its rest-state value (w_i for the flow, w_i T_m for the heat): in 16
 * bits for BF16D and F16D, in 32 bits for F32D; the per-node relaxation time
 * is then stored as FP32.  F16S and BF16S store the same 16-bit deviations
 * rounded stochastically (up or down with probability given by the distance
 * to the two neighbours; the random bits are hashed from a per-step seed
 * and the node's offset), so that updates below the 16-bit spacing are not
 * lost on average near a steady state; the paper has no counterpart (its
 * storage is not stated).  Not built with the adjoint. */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_BF16D = 2, LBM_F16D = 3, LBM_F32D = 4,
               LBM_F16S = 5, LBM_BF16S = 6 } lbm_prec;

/* Options; lbm_default_opts() fills the defaults listed per field. */
typedef struct {
    int prec;          /* lbm_prec                                   [F64]  */
    double Ma;         /* Mach number of the velocity scale U_c      [0.1]  */
    int clamp_mode;    /* 0: literal modified power law, Eq. (MPL);
                          1: continuous clamp of the shear rate      [0]    */
    int porous_model;  /* 0: the paper's Darcy drag (porosity 1, no
                          Forchheimer term); 1: generalized Brinkman-
                          Forchheimer model with the porosity        [1]    */
    double s_e, s_p;   /* free thermal MRT rates (4th, 5th moment)   [1.5]  */
    int resid_interval;/* steps between convergence checks           [1000] */
    int layout;        /* 0: two-buffer pull scheme; 1: one buffer,
                          in-place AA-pattern streaming (half the
                          memory, same bytes per update)             [0]    */
    void *cuda_stream; /* cudaStream_t to run on; NULL: the library
                          creates and owns one                       [NULL] */
    int device;        /* CUDA device ordinal the context lives on and
                          every call selects; -1: the device current
                          in the calling thread at lbm_init          [-1]   */
    double stag_floor; /* lbm_run_to_steady stops on stagnation only
                          below this residual (the storage's noise
                          floor); < 0: 0 for F64 (never), 1e-6 for
                          F32 and F32D, 1e-3 for F16S, 1e-2 for F16D
                          and BF16S, 1e-1 for BF16D                  [-1]   */
    int tau_iters;     /* how the relaxation time of the strain rate and
                          the velocity solve is obtained (the paper
                          does not say: section "Power-law fluid"):
                          0: lagged -- each node stores the tau of its
                          last collision (one value per node read and
                          written every step);
                          1..LBM_TAU_ITERS_MAX: node-local implicit --
                          the root of tau = 3 nu_ref D(gamma*(tau)) +
                          1/2 (Eq. MPL, gamma from the collision started
                          at tau), by that many Newton steps on ln tau
                          from tau0; no tau is stored, so a step moves
                          8 bytes per node less in FP32 storage.  2
                          reach FP32 rounding, 4 FP64 rounding on
                          developed flows.  Not built with the
                          adjoint                                    [0]    */
    int staging;       /* how the step kernel of the two-buffer layout
                          gets its inputs: 1 straight into registers,
                          two nodes per thread; 3 straight into
                          registers, four nodes per thread (16-bit
                          storages only, else LBM_ERR_UNSUPPORTED);
                          2 is not built (LBM_ERR_UNSUPPORTED); 0 the fastest
                          measured: 3 for the 16-bit storages on grids
                          of at least 2048 x 2048 nodes (4096 x 4096
                          with tau_iters > 0), else 1.  The update is
                          the same; with
                          stochastic rounding, the random bits of the
                          nodes a mode updates one at a time (at the
                          walls) differ between modes               [0]    */
    int graph_steps;   /* lbm_step replays a CUDA graph of this many
                          steps (rounded up to even) instead of one
                          launch per step, which pays on small,
                          launch-bound grids: 0 auto (64 steps for
                          grids of at most 512 x 512 nodes, none for
                          F16S / BF16S in layout 1), -1 never, G > 0
                          always (F16S / BF16S with layout 1 get
                          LBM_ERR_UNSUPPORTED).  With F16S / BF16S the
                          captured kernels compute each step's seed on
                          the device from the step count the replay
                          starts at, so the seeds are a plain launch's.
                          Results are identical either way.  The graph
                          is captured on the context's stream at the
                          first use (and again after
                          lbm_set_darcy_field); none is used while the
                          stream is already being captured          [0]    */
    uint64_t seed;     /* stream of the stochastic rounding (F16S,
                          BF16S): mixed into every step's seed, so runs
                          with different seeds round independently;
                          0 is the default stream.  Other storages
                          ignore it                                  [0]    */
} lbm_opts;

/* Lattice-unit parameters the library derived from the problem groups
 * (a reading of the paper, which defers the mapping to earlier work):
 *   U_c = Ma / sqrt(3), L = nx;
 *   nu_ref = nu_0 U_c L with nu_0 = Pr / sqrt(Ra)^(2-n) (power-law section);
 *   gamma* = |gamma| L / U_c (non-dimensional shear rate for Eq. MPL);
 *   tauT = 3 U_c L / sqrt(Ra) + 1/2 (diffusivity 1/sqrt(Ra) of the energy
 *   equation); g beta = Pr U_c^2 / L (buoyancy term Pr theta); K = Da L^2;
 *   tau = 3 nu + 1/2 (Eq. kinematic_viscosity with c_s^2 = 1/3). */
typedef struct {
    int nx, ny;
    double n, nu_ref, gamma_scale, gamma1, gamma2;
    int clamp_mode;
    double K, eps, Feps, gbeta, Tm, tauT, s_e, s_p;
    double T_hot, T_cold, L, tau0;
    int prec;
    int64_t pitch;     /* elements between rows of a device plane           */
} lbm_lattice;

typedef struct lbm_ctx lbm_ctx;

/* Fill *opts with the defaults above.  Never fails. */
void lbm_default_opts(lbm_opts *opts);

/* Create a cavity run: nx x ny nodes, power-law index n, Darcy number Da,
 * Rayleigh number Ra, Prandtl number Pr and porosity (problem statement of
 * section "Mathematical formulations"; groups of Eq. non_dim_var).  The
 * state starts at rest: rho = 1, u = 0, T = (T_h + T_c)/2, f = f^eq,
 * g = g^eq, tau = tau0.  opts may be NULL (defaults).
 * Errors: LBM_ERR_ARG (nx or ny < 2, ny > 65535, n, Da, Ra or Pr <= 0, porosity outside
 * (0, 1], bad option), LBM_ERR_UNSTABLE, LBM_ERR_OOM, LBM_ERR_CUDA.
 * On error *out is set to NULL and nothing is leaked. */
int lbm_init(lbm_ctx **out, int nx, int ny, double n, double Da, double Ra,
             double Pr, double porosity, const lbm_opts *opts);

/* Release every device and host resource of ctx (NULL is ignored). */
void lbm_destroy(lbm_ctx *ctx);

/* Set a per-node Darcy number Da(x) (host array of nx*ny doubles, [ny][nx],
 * caller-owned, copied): the permeability K(x) = Da(x) L^2 then replaces the
 * uniform K of lbm_init in the drag of the momentum equations (the term
 * -U D / Da of Eqs. par_sim_u/v:momentum, node by node).  NULL returns to the
 * uniform Da.  Errors: LBM_ERR_ARG (a value not finite or <= 0), LBM_ERR_OOM,
 * LBM_ERR_CUDA.  Synchronous. */
int lbm_set_darcy_field(lbm_ctx *ctx, const double *Da_xy);

/* Copy the lattice-unit parameters of ctx into *out. */
int lbm_get_lattice(const lbm_ctx *ctx, lbm_lattice *out);

/* Advance k >= 0 time steps.  Each step is one launch of the fused kernel:
 * pull streaming with the wall rules, macroscopic moments (Eqs.
 * macro_fluid_density, velo), porous velocity solve, strain rate from the
 * non-equilibrium moments and the modified power law (Eq. MPL and the
 * strain-rate equation), forced MRT flow collision (Eq. normalMRTequation)
 * and MRT thermal collision (Eq. thermalMRTequation).  Asynchronous on the
 * context's stream.  Errors: LBM_ERR_ARG (k < 0), LBM_ERR_CUDA. */
int lbm_step(lbm_ctx *ctx, int64_t k);

/* Wait for all work queued on the context's stream. */
int lbm_synchronize(lbm_ctx *ctx);

/* Streamed (pre-collision) macroscopic fields at the current step, i.e. the
 * values the next collision sees: density, velocity after the porous solve,
 * temperature, and the apparent lattice viscosity the next collision will
 * use.  Each pointer is NULL (skipped) or a host array of nx*ny doubles.
 * Synchronous.  Errors: LBM_ERR_OOM, LBM_ERR_CUDA. */
int lbm_fields(lbm_ctx *ctx, double *rho, double *ux, double *uy, double *T,
               double *nu);

/* Average Nusselt number on the hot wall (Eq. avgNu: the mean over the wall
 * of Nu(Y) = -d theta/dX at X = 0) and the outward one on the cold wall,
 * from the streamed temperature, accumulated in FP64.  The wall derivative is
 * the second-order one-sided difference through the wall value and the two
 * nearest nodes: -L (9 theta_0 - theta_1 - 8 theta_w) / 3.  nu_local is NULL
 * or a host array of ny doubles (hot-wall local Nu).  Synchronous. */
int lbm_nusselt(lbm_ctx *ctx, double *nu_hot, double *nu_cold,
                double *nu_local);

/* Convergence residual against the fields of the previous call:
 * r = max over phi in {u_x, u_y, T} of ||phi - phi_prev||_2 / ||phi||_2,
 * accumulated in FP64, plus a flag for any non-finite value.  The first call
 * after lbm_init or lbm_set_state only stores the snapshot and returns
 * *resid = +inf.  Synchronous.  Returns LBM_ERR_NONFINITE if the flag is set. */
int lbm_residual(lbm_ctx *ctx, double *resid);

/* Run until the residual (checked every resid_interval steps) falls below
 * tol, stagnates (below stag_floor with no new minimum over 10 checks), or
 * max_steps is reached.
 * *steps_done, *resid and *reason (0 tol reached, 1 stagnated, 2 max_steps)
 * may be NULL.  Returns LBM_ERR_NONFINITE on NaN or Inf. */
int lbm_run_to_steady(lbm_ctx *ctx, double tol, int64_t max_steps,
                      int64_t *steps_done, double *resid, int *reason);

/* Size in bytes of the native state: 14 planes of nx*ny distribution values
 * in the storage type (f0..f8, then g0..g4; 16-bit forms hold deviations),
 * followed by one plane of nx*ny relaxation times (double for LBM_F64, float
 * otherwise), each plane row-major [ny][nx]. */
size_t lbm_state_bytes(const lbm_ctx *ctx);

/* Copy the native state (layout of lbm_state_bytes) to / from host memory.
 * bytes must equal lbm_state_bytes(ctx).  Pinned host memory gives
 * asynchronous-speed copies.  Synchronous.  Errors: LBM_ERR_ARG, LBM_ERR_CUDA. */
int lbm_get_state(lbm_ctx *ctx, void *host, size_t bytes);
int lbm_set_state(lbm_ctx *ctx, const void *host, size_t bytes);

/* Checkpoint / resume.  A checkpoint is a self-describing byte blob in host
 * memory (caller-owned, lbm_checkpoint_bytes long): a versioned header
 * (magic "LBMCKPT1", grid, storage, layout, tau scheme, slab rows, the
 * lattice-unit parameters, the step count and lbm_opts.seed) followed by
 * the native state of lbm_get_state.  Loading it into a context created
 * with the same grid, parameters and options restores the state and the
 * step count, so the run continues exactly as the saved one would have
 * after the save (the stochastic rounding's seeds included).  A per-node
 * Darcy field is not part of it: set it again.  Both calls are synchronous.
 * Errors: LBM_ERR_ARG (size, or a blob that is not a checkpoint of a run
 * with the same grid, storage, options and parameters), LBM_ERR_CUDA. */
size_t lbm_checkpoint_bytes(const lbm_ctx *ctx);
int lbm_checkpoint_save(lbm_ctx *ctx, void *host, size_t bytes);
int lbm_checkpoint_load(lbm_ctx *ctx, const void *host, size_t bytes);

/* The post-collision state as FP64 host arrays: f[9][ny][nx], g[5][ny][nx]
 * and tau[ny][nx] (full population values, deviations resolved).  The
 * import rounds to the storage precision.  Any pointer may be NULL (skipped
 * on export, left unchanged on import).  With tau_iters > 0 tau is not part
 * of the state: the export gives the implicit tau each node's next
 * collision starts from, and the import ignores it.  Synchronous. */
int lbm_get_state_f64(lbm_ctx *ctx, double *f, double *g, double *tau);
int lbm_set_state_f64(lbm_ctx *ctx, const double *f, const double *g,
                      const double *tau);

/* Discrete adjoint (reverse mode) of the hot-wall average Nusselt number J
 * (Eq. avgNu) after `steps` fused steps, with respect to the per-node Darcy
 * number Da(x) (the field of lbm_set_darcy_field, or the uniform Da seen as
 * a field), the power-law index n and the Rayleigh number Ra.  The forward
 * run keeps a checkpoint every ckpt_every steps; the reverse sweep
 * recomputes one segment of states at a time from its checkpoint and runs
 * the hand-written reverse of the fused step over it, recomputing the next
 * segment on a second stream meanwhile (the result does not depend on
 * ckpt_every or on that overlap).  from_rest = 1 first
 * resets the state to the rest state of lbm_init and includes the
 * dependence of its relaxation time tau_0 on n and Ra; from_rest = 0 starts
 * from the current state, held fixed.  Afterwards the context holds s_T.
 * Outputs (any may be NULL): *J, dDa (host, nx*ny doubles, [ny][nx]), *dn,
 * *dRa, and *peak_bytes, the device memory the run used (state buffers,
 * checkpoints, two segments of states, or one if there is a single segment
 * or no memory for a second, two adjoint buffers, FP64 gradient planes).  Parameter gradients accumulate in FP64.  Two-buffer layout with
 * FP64 or FP32 storage; other storages get LBM_ERR_UNSUPPORTED.
 * Synchronous.  Errors: LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA. */
int lbm_adjoint_nu(lbm_ctx *ctx, int64_t steps, int ckpt_every, int from_rest,
                   double *J, double *dDa, double *dn, double *dRa,
                   double *peak_bytes);

/* ------------------------------------------------------------- sweeps
 * The paper's results are a sweep of independent cavities over n, Da and Ra
 * (section "Results and discussions", Tables 1-2).  A batch runs such a sweep
 * as one workload: each time step covers the row tiles of every active case
 * (grids may differ) in one launch, or all steps between two checks run in
 * one persistent launch (lbm_batch_set_plan); every resid_interval steps each
 * case's residual is checked on the device and converged cases stop being
 * stepped.  All cases share the storage precision and the options of
 * lbm_batch_create (the two-buffer layout; resid_interval must be even; the
 * lagged or the implicit tau).  With the stochastic-rounding storages each
 * step's seed is computed on the device from the case's step count, so a
 * case draws the same random bits in a batch as stepped alone. */
typedef struct {
    int nx, ny;
    double n, Da, Ra, Pr, porosity;
} lbm_case;

typedef struct lbm_batch lbm_batch;

/* Create one context per case (validated as by lbm_init) on one stream.
 * Errors as lbm_init; LBM_ERR_ARG also for an odd resid_interval;
 * LBM_ERR_UNSUPPORTED for layout 1. */
int lbm_batch_create(lbm_batch **out, const lbm_case *cases, int ncases,
                     const lbm_opts *opts);
void lbm_batch_destroy(lbm_batch *batch);

/* Borrow case i's context for state I/O, fields or Nu (do not destroy it). */
int lbm_batch_get_case(lbm_batch *batch, int i, lbm_ctx **ctx);

/* Advance every case k steps (one launch per step). Asynchronous. */
int lbm_batch_step(lbm_batch *batch, int64_t k);

/* Run every case until its residual (as lbm_run_to_steady) falls below tol,
 * stagnates below the storage's noise floor, or reaches max_steps.
 * graph_mode 0: the host relaunches a CUDA graph of one resid_interval chunk
 * (all cases' steps, residuals and the convergence update) while any case is
 * active; 1: a single CUDA graph launch runs the whole sweep, looping on the
 * device (a conditional while node), bounded by max_steps.  steps, resid,
 * reason (per case, caller-owned, ncases entries; NULL skips) receive the
 * steps run, the last residual, and 0 tol / 1 stagnated / 2 max_steps /
 * 3 non-finite.  Synchronous.  Returns LBM_ERR_NONFINITE if any case blew up. */
int lbm_batch_run_to_steady(lbm_batch *batch, double tol, int64_t max_steps,
                            int graph_mode, int64_t *steps, double *resid,
                            int *reason);

/* Hot- and cold-wall average Nu of every case (host arrays of ncases). */
int lbm_batch_nusselt(lbm_batch *batch, double *nu_hot, double *nu_cold);

/* Execution plan of the batched steps.  The row tiles of the active cases
 * form one list (compacted on the device when cases retire), and a grid of
 * blocks_per_sm x (SM count) blocks strides over it every step, so a block
 * takes several tiles -- of one or several cases -- per step.
 *   LBM_BATCH_PER_STEP: one launch per time step;
 *   LBM_BATCH_PERSISTENT: one cooperative launch runs all steps between two
 *     convergence checks, with a grid barrier between steps (blocks_per_sm
 *     is capped at the blocks that fit on an SM).  Every wait at the
 *     barrier is bounded (lbm_batch_set_wait_budget); a block that gives up
 *     raises the batch's error word and every block leaves, after which the
 *     calls that step the batch return LBM_ERR_TIMEOUT (sticky: the states
 *     are no longer valid).  If a CUDA graph with the cooperative launch
 *     cannot be built, lbm_batch_run_to_steady falls back to the per-step
 *     form.
 * Both modes run the same tile code: results are identical.
 * Defaults: per-step, 128 threads, 8 blocks per SM. */
enum { LBM_BATCH_PER_STEP = 0, LBM_BATCH_PERSISTENT = 1 };

/* Set the plan: mode as above, threads 64, 128 or 256 (tile = 2 x threads
 * nodes, or threads nodes in FP64), blocks_per_sm 1..64.  Errors:
 * LBM_ERR_ARG, LBM_ERR_UNSUPPORTED (no block of the persistent kernel fits
 * on an SM), LBM_ERR_CUDA. */
int lbm_batch_set_plan(lbm_batch *batch, int mode, int threads, int blocks_per_sm);
/* Read the plan in effect (blocks_per_sm after the residency cap). */
int lbm_batch_get_plan(const lbm_batch *batch, int *mode, int *threads, int *blocks_per_sm);
/* Clock cycles a persistent block waits at a barrier before it gives up
 * (default 2^31, about one second); cycles >= 1. */
int lbm_batch_set_wait_budget(lbm_batch *batch, int64_t cycles);

/* Autotune the plan: time `steps` batched steps for every mode x block size
 * (64, 128, 256) x blocks per SM (2, 4, 8, 16, 32; persistent: those that
 * fit) on copies of the current states (restored afterwards) and keep the
 * fastest; *threads_out (may be NULL) receives its block size and
 * lbm_batch_get_plan the rest. */
int lbm_batch_tune(lbm_batch *batch, int steps, int *threads_out);

/* ------------------------------------------------- row-slab decomposition
 * One cavity split into horizontal slabs of rows, one per context (and per
 * GPU or rank), as a domain decomposition of the fused step: the pull
 * scheme reads each node's neighbours from the previous state, so a slab
 * needs, per step, only the populations that cross its cut rows -- per cut
 * node 3 D2Q9 populations (f2, f5, f6 upward; f4, f7, f8 downward) and 1
 * D2Q5 population (g2 upward, g4 downward) each way.  A slab context keeps
 * one ghost row beyond each cut; after every step the caller packs the
 * outgoing populations (lbm_halo_pack), moves them to the neighbours
 * (device copies, peer copies or NCCL send/recv), and unpacks what arrives
 * into the ghost rows (lbm_halo_unpack).  Interior nodes then compute
 * exactly what the undivided cavity computes (bit for bit with FP64 and FP32
 * storage; with stochastic rounding the random bits depend on the slab's
 * own node offsets).  Wall Nusselt numbers and residuals become sums over
 * each slab's interior rows that the caller adds up across slabs
 * (lbm_nusselt_sums, lbm_residual_sums: an all-reduce of a few doubles).
 * Slab contexts take lbm_step, lbm_fields, lbm_nusselt (average over the
 * slab's interior rows), the state calls and lbm_set_darcy_field (arrays
 * of the context's local rows, ghost rows included); lbm_run_to_steady,
 * lbm_adjoint_nu and lbm_residual_noalloc return LBM_ERR_UNSUPPORTED. */

/* Create the slab of global rows [y0, y1) of an nx x ny cavity (the other
 * arguments as lbm_init; L = nx, so the lattice mapping is the cavity's).
 * The context has (y1 - y0) local rows plus a ghost row below if y0 > 0 and
 * above if y1 < ny.  The two-buffer layout only (layout 1 gets
 * LBM_ERR_UNSUPPORTED).  Errors: as lbm_init; LBM_ERR_ARG for a bad range. */
int lbm_init_slab(lbm_ctx **out, int nx, int ny, int y0, int y1, double n, double Da, double Ra,
                  double Pr, double porosity, const lbm_opts *opts);

/* The slab's first global row *y0, its interior local rows [*row_lo,
 * *row_hi) and its local row count *ny_local (a whole cavity: 0, 0, ny, ny).
 * Any pointer may be NULL. */
int lbm_slab_rows(const lbm_ctx *ctx, int *y0, int *row_lo, int *row_hi, int *ny_local);

/* Bytes of one halo message: 4 planes x nx values in the storage type. */
size_t lbm_halo_bytes(const lbm_ctx *ctx);

/* Copy the populations leaving the current state through the lower cut
 * (f4, f7, f8, g4 of the bottom interior row) into d_lo and through the
 * upper cut (f2, f5, f6, g2 of the top interior row) into d_hi: device
 * buffers of lbm_halo_bytes each, plane-major [4][nx]; NULL skips a side.
 * Asynchronous on the context's stream.  Errors: LBM_ERR_ARG (a buffer for a
 * side with no neighbour), LBM_ERR_CUDA. */
int lbm_halo_pack(lbm_ctx *ctx, void *d_lo, void *d_hi);

/* Write the lower neighbour's d_hi message (its upward populations) into
 * the ghost row below and the upper neighbour's d_lo message into the ghost
 * row above; NULL skips a side.  Asynchronous.  Errors as lbm_halo_pack. */
int lbm_halo_unpack(lbm_ctx *ctx, const void *d_lo, const void *d_hi);

/* Sums over the interior rows of the hot- and cold-wall Nu_j of
 * lbm_nusselt (the cavity's average is the sum over all slabs / ny).
 * Synchronous. */
int lbm_nusselt_sums(lbm_ctx *ctx, double *hot_sum, double *cold_sum);

/* The seven sums of lbm_residual over the interior rows, against the
 * previous call's snapshot: sums[2c] = sum (phi_c - phi_c,prev)^2,
 * sums[2c + 1] = sum phi_c^2 for phi = u_x, u_y, T, and sums[6] the count of
 * non-finite values.  Across slabs: add the sums, then r = max over c of
 * sqrt(sum[2c] / sum[2c+1]).  The first call stores the snapshot and
 * returns +inf in sums[0], sums[2], sums[4].  Synchronous. */
int lbm_residual_sums(lbm_ctx *ctx, double *sums);

/* Allocation-free form of lbm_residual, for callers that cannot call
 * cudaMalloc at the point where they check convergence: host code that must
 * not block (cudaMalloc and cudaFree can synchronise the device and stall
 * work already queued), and applications whose device memory is handed out
 * by their own pool allocator, where a stray allocation can fail or fragment
 * the pool.  The paper has no counterpart; it is an interface addition.
 *
 * It computes the same quantity as lbm_residual -- for phi in {u_x, u_y, T},
 * ||phi - phi_prev||_2 / ||phi||_2 accumulated in FP64 -- but every buffer
 * is the caller's and nothing is allocated, freed or synchronised:
 *   d_snapshot  device memory of the context's device, 3*nx*ny doubles
 *               ([3][ny][nx]: u_x, u_y, T); read as the previous fields
 *               unless `first` is non-zero, then overwritten with the
 *               current ones;
 *   first       non-zero: only store the snapshot (results are +inf);
 *   d_result    device memory, 4 doubles, written on the context's stream:
 *               [0..2] the relative change of u_x, u_y, T, [3] the number of
 *               non-finite values seen.
 * The work is queued on the context's stream; synchronise before reading
 * d_result.  The partial sums live in a fixed device array of
 * LBM_NOALLOC_MAX_ROWS rows (1 MiB) inside the library, kept on every GPU
 * that loaded it until the process exits; grids with more rows are refused
 * with LBM_ERR_SIZE.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress), so make it before any stream
 * capture; a call that finds the device's context replaced since (after a
 * cudaDeviceReset) looks it up again.  All calls share the array and it keeps the last call's contents
 * (every slot a call reads is written earlier in the same call); calls that
 * overlap on the GPU, e.g. on two streams, race on it.
 * Contexts with the in-place layout (layout = 1) get LBM_ERR_UNSUPPORTED.
 * Errors: LBM_ERR_ARG (NULL pointer), LBM_ERR_SIZE, LBM_ERR_UNSUPPORTED,
 * LBM_ERR_CUDA. */
int lbm_residual_noalloc(lbm_ctx *ctx, double *d_snapshot, int first,
                         double *d_result);

/* Name of an LBM_* code (static storage). */
const char *lbm_strerror(int code);

/* Text of the last CUDA runtime error seen by this host thread inside the
 * library ("" if none); thread-local storage, valid until the next call. */
const char *lbm_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif
