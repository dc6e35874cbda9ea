// lbm_capi.cu -- the C ABI of include/lbm.h: argument checks, the mapping of
// the paper's non-dimensional groups to lattice units, device memory, and the
// host-side control of the kernels in lbm_kernels.cu.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "lbm_internal.h"
#include "lbm_trace.h"

static thread_local char g_last_cuda[256] = "";

#define CK(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            snprintf(g_last_cuda, sizeof(g_last_cuda), "%s: %s", #call,               \
                     cudaGetErrorString(e_));                                          \
            return e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;       \
        }                                                                              \
    } while (0)

namespace {

// ---- replayed step graphs (lbm_opts.graph_steps)
void drop_graphs(lbm_ctx *c)
{
    for (int i = 0; i < 2; i++)
        if (c->step_graph[i]) {
            cudaGraphExecDestroy(c->step_graph[i]);
            c->step_graph[i] = nullptr;
        }
}

int graph_len_for(const lbm_ctx *c)
{
    const int g = c->opts.graph_steps;
    if (g < 0) return 0;
    if (g > 0) return (g + 1) & ~1;
    // the stochastic-rounding storages take their seeds from the device in a
    // graph: built for the two-buffer kernels, not the in-place ones
    const bool sr_aa = lbm::rounds_stochastically(c->opts.prec) && c->opts.layout == 1;
    return (!sr_aa && (int64_t)c->nx * c->ny <= 512 * 512) ? 64 : 0;
}

int graph_parity(const lbm_ctx *c) { return c->opts.layout == 1 ? (c->aa_form_o ? 1 : 0) : c->cur; }

// Capture G step launches on the context's stream into an executable graph
// for the current parity.  Launching records nothing while capturing, and G
// is even, so the buffer state is back where it started afterwards.
int capture_steps(lbm_ctx *c, int G, int par)
{
    cudaGraph_t g = nullptr;
    if (lbm::rounds_stochastically(c->opts.prec) && !c->d_step_base &&
        cudaMalloc(&c->d_step_base, sizeof(long long)) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_OOM;
    }
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_UNSUPPORTED;
    }
    cudaError_t e = cudaSuccess;
    const bool sr = lbm::rounds_stochastically(c->opts.prec);
    for (int i = 0; i < G && e == cudaSuccess; i++) {
        c->capture_s = sr ? i : -1;   // seeds from d_step_base + i (lbm_kernels.cu)
        e = lbm::launch_step(c);
    }
    c->capture_s = -1;
    const cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->step_graph[par], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) c->step_graph[par] = nullptr;
    CK(e);
    return LBM_OK;
}


size_t store_elem(int prec) { return prec == LBM_F64 ? 8 : ((prec == LBM_F32 || prec == LBM_F32D) ? 4 : 2); }
size_t tau_elem(int prec) { return prec == LBM_F64 ? 8 : 4; }

// Mapping of the non-dimensional problem to lattice units.  The paper defers
// it to earlier work, so this is a stated reading:
//   velocity scale U_c = Ma c_s (c_s^2 = 1/3), length scale L = nx;
//   alpha = U_c L / sqrt(Ra) (energy equation: diffusivity 1/sqrt(Ra)),
//   tauT = 3 alpha + 1/2;
//   nu_0 = Pr / sqrt(Ra)^(2 - n) (power-law section), nu_ref = nu_0 U_c L;
//   gamma* = |gamma| L / U_c is the shear rate the thresholds gamma_1 = 0.01,
//   gamma_2 = 1e6 of Eq. (MPL) apply to;
//   g beta (T_h - T_c) = Pr U_c^2 / L (buoyancy Pr theta of the
//   non-dimensional v-momentum equation), T_m = (T_h + T_c)/2;
//   K = Da L^2 (Eq. non_dim_var); tau = 3 nu + 1/2 (Eq. kinematic_viscosity).
//   Porous model 1 (generalized Brinkman-Forchheimer): porosity eps and
//   Ergun's F_eps = 1.75 / sqrt(150 eps^3); model 0: eps = 1, F_eps = 0.
int map_lattice(int nx, int ny, double n, double Da, double Ra, double Pr, double porosity,
                const lbm_opts &o, lbm_lattice *L)
{
    if (nx < 2 || ny < 2 || ny > 65535 || nx > (1 << 30) || !(n > 0) || !(Da > 0) || !(Ra > 0) || !(Pr > 0) || !(porosity > 0) ||
        porosity > 1 || !isfinite(n) || !isfinite(Da) || !isfinite(Ra) || !isfinite(Pr))
        return LBM_ERR_ARG;
    if (o.prec < LBM_F64 || o.prec > LBM_BF16S || !(o.Ma > 0) || o.Ma > 1 ||
        (o.clamp_mode != 0 && o.clamp_mode != 1) || (o.porous_model != 0 && o.porous_model != 1) ||
        !(o.s_e > 0) || !(o.s_e < 2) || !(o.s_p > 0) || !(o.s_p < 2) || o.resid_interval < 1 ||
        o.device < -1 || o.tau_iters < 0 || o.tau_iters > LBM_TAU_ITERS_MAX || o.staging < 0 ||
        o.staging > 3 || o.graph_steps < -1)
        return LBM_ERR_ARG;
    if (o.graph_steps > 0 && (o.prec == LBM_F16S || o.prec == LBM_BF16S) && o.layout == 1)
        return LBM_ERR_UNSUPPORTED;
    if (o.staging == 2) return LBM_ERR_UNSUPPORTED;  // the staged kernel is not built
    if (o.staging == 3 && !(o.prec == LBM_BF16D || o.prec == LBM_F16D || o.prec == LBM_F16S || o.prec == LBM_BF16S))
        return LBM_ERR_UNSUPPORTED;
    if (o.layout != 0 && o.layout != 1) return LBM_ERR_UNSUPPORTED;
    memset(L, 0, sizeof(*L));
    const double Uc = o.Ma / sqrt(3.0);
    const double len = (double)nx;
    L->nx = nx;
    L->ny = ny;
    L->n = n;
    L->nu_ref = Pr / pow(sqrt(Ra), 2.0 - n) * Uc * len;
    L->gamma_scale = len / Uc;
    L->gamma1 = 0.01;
    L->gamma2 = 1.0e6;
    L->clamp_mode = o.clamp_mode;
    L->K = Da * len * len;
    L->eps = o.porous_model == 1 ? porosity : 1.0;
    L->Feps = o.porous_model == 1 ? 1.75 / sqrt(150.0 * porosity * porosity * porosity) : 0.0;
    L->T_hot = 1.0;
    L->T_cold = 0.0;
    L->Tm = 0.5;
    L->gbeta = Pr * Uc * Uc / len;
    L->tauT = 3.0 * Uc * len / sqrt(Ra) + 0.5;
    L->s_e = o.s_e;
    L->s_p = o.s_p;
    L->L = len;
    // at rest gamma* = 0: D = 1 for the literal law, gamma_1^(n-1) for the clamp
    const double D0 = o.clamp_mode == 0 ? 1.0 : pow(L->gamma1, n - 1.0);
    L->tau0 = 3.0 * L->nu_ref * D0 + 0.5;
    L->prec = o.prec;
    if (!(L->tau0 > 0.5 + 1e-6) || !(L->tauT > 0.5 + 1e-6)) return LBM_ERR_UNSTABLE;
    return LBM_OK;
}

void free_ctx(lbm_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    for (int b = 0; b < 2; b++) {
        cudaFree(c->buf.dist[b]);
        cudaFree(c->buf.tau[b]);
    }
    cudaFree(c->d_small);
    cudaFreeHost(c->h_small);
    cudaFree(c->d_stage);
    cudaFree(c->d_snap);
    cudaFree(c->d_part);
    cudaFree(c->d_nuloc);
    cudaFree(c->d_da);
    cudaFree(c->d_step_base);
    drop_graphs(c);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

// The in-place layout leaves the state in its odd-step form after an odd
// number of steps; every call that reads or writes the state first brings it
// back to the canonical form (one in-place pass, no allocation).
int canonical(lbm_ctx *c)
{
    if (c->opts.layout == 1 && c->aa_form_o) CK(lbm::launch_aa_normalize(c));
    return LBM_OK;
}

double stag_floor(const lbm_ctx *c)
{
    if (c->opts.stag_floor >= 0) return c->opts.stag_floor;
    switch (c->opts.prec) {
    case LBM_F64: return 0.0;
    case LBM_F32:
    case LBM_F32D: return 1e-6;
    case LBM_F16D: return 1e-2;
    case LBM_F16S: return 1e-3;
    case LBM_BF16S: return 1e-2;
    default: return 1e-1;
    }
}

// Copy `rows` rows of `row_bytes` between host (packed rows) and device
// (rows `pitch_bytes` apart).  Unpadded rows are one linear copy: the
// strided form moved a 1 GB state at a small fraction of the link's rate.
cudaError_t copy_rows(lbm_ctx *c, void *host, void *dev, size_t row_bytes, size_t pitch_bytes, size_t rows,
                      bool to_host)
{
    const cudaMemcpyKind kind = to_host ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice;
    if (row_bytes == pitch_bytes)
        return to_host ? cudaMemcpyAsync(host, dev, row_bytes * rows, kind, c->stream)
                       : cudaMemcpyAsync(dev, host, row_bytes * rows, kind, c->stream);
    return to_host ? cudaMemcpy2DAsync(host, row_bytes, dev, pitch_bytes, row_bytes, rows, kind, c->stream)
                   : cudaMemcpy2DAsync(dev, pitch_bytes, host, row_bytes, row_bytes, rows, kind, c->stream);
}

// Copy the 14 distribution planes between host (canonical order, unpadded)
// and device.  In the in-place layout's canonical form population i of a
// node lives in plane opp(i).
int copy_planes(lbm_ctx *c, void *host, bool to_host)
{
    const size_t es = c->dist_elem, n = (size_t)c->nx * c->ny;
    if (c->opts.layout == 0) {
        CK(copy_rows(c, host, c->buf.dist[c->cur], c->nx * es, c->pitch * es, 14 * (size_t)c->ny, to_host));
        return LBM_OK;
    }
    static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    for (int i = 0; i < 14; i++) {
        const int j = i < 9 ? OPP[i] : 9 + OPP[i - 9];
        char *h = (char *)host + (size_t)i * n * es;
        char *d = (char *)c->buf.dist[0] + (size_t)j * c->plane * es;
        CK(copy_rows(c, h, d, c->nx * es, c->pitch * es, (size_t)c->ny, to_host));
    }
    return LBM_OK;
}

int ensure_stage(lbm_ctx *c)
{
    if (c->d_stage) return LBM_OK;
    CK(cudaMalloc(&c->d_stage, sizeof(double) * 15 * (size_t)c->nx * c->ny));
    return LBM_OK;
}

int init_ctx(lbm_ctx *c)
{
    if (c->opts.device >= 0) {
        CK(cudaSetDevice(c->opts.device));
        c->device = c->opts.device;
    } else {
        CK(cudaGetDevice(&c->device));
    }
    const size_t es = store_elem(c->opts.prec), ts = tau_elem(c->opts.prec);
    c->pitch = ((int64_t)c->nx + 63) / 64 * 64;
    c->plane = c->pitch * c->ny;
    c->dist_elem = es;
    c->tau_elem = ts;
    if (c->opts.cuda_stream) {
        c->stream = (cudaStream_t)c->opts.cuda_stream;
    } else {
        CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    const int nbuf = c->opts.layout == 1 ? 1 : 2;   // in-place layout: one buffer
    for (int b = 0; b < nbuf; b++) {
        CK(cudaMalloc(&c->buf.dist[b], es * 14 * (size_t)c->plane));
        CK(cudaMalloc(&c->buf.tau[b], ts * (size_t)c->plane));
        CK(cudaMemsetAsync(c->buf.dist[b], 0, es * 14 * (size_t)c->plane, c->stream));
        CK(cudaMemsetAsync(c->buf.tau[b], 0, ts * (size_t)c->plane, c->stream));
    }
    CK(cudaMalloc(&c->d_small, sizeof(double) * 16));
    CK(cudaMallocHost(&c->h_small, sizeof(double) * 16));
    CK(cudaMalloc(&c->d_nuloc, sizeof(double) * (size_t)c->ny));
    c->n_part = lbm::residual_blocks(c);
    CK(cudaMalloc(&c->d_part, sizeof(double) * 8 * (size_t)c->n_part));
    c->lat.pitch = c->pitch;
    CK(lbm::launch_init(c));
    CK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

}  // namespace

extern "C" {

void lbm_default_opts(lbm_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->prec = LBM_F64;
    o->Ma = 0.1;
    o->clamp_mode = 0;
    o->porous_model = 1;
    o->s_e = 1.5;
    o->s_p = 1.5;
    o->resid_interval = 1000;
    o->layout = 0;
    o->cuda_stream = nullptr;
    o->device = -1;
    o->stag_floor = -1.0;
    o->tau_iters = 0;
    o->staging = 0;
    o->graph_steps = 0;
    o->seed = 0;
}

// A context of ny local rows; rows [row_lo, row_hi) are global rows
// [y0, ...) of a cavity of ny_glob rows (a whole cavity: 0, ny, 0, ny).
static int create_ctx(lbm_ctx **out, int nx, int ny, double n, double Da, double Ra, double Pr, double porosity,
                      const lbm_opts *opts, int row_lo, int row_hi, int y0, int ny_glob)
{
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    lbm_opts o;
    if (opts)
        o = *opts;
    else
        lbm_default_opts(&o);
    lbm_lattice L;
    int rc = map_lattice(nx, ny, n, Da, Ra, Pr, porosity, o, &L);
    if (rc != LBM_OK) return rc;
    lbm_ctx *c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ERR_OOM;
    c->nx = nx;
    c->ny = ny;
    c->row_lo = row_lo;
    c->row_hi = row_hi;
    c->y0 = y0;
    c->ny_glob = ny_glob;
    c->opts = o;
    c->lat = L;
    rc = init_ctx(c);
    if (rc != LBM_OK) {
        free_ctx(c);
        return rc;
    }
    *out = c;
    return LBM_OK;
}

int lbm_init(lbm_ctx **out, int nx, int ny, double n, double Da, double Ra, double Pr,
             double porosity, const lbm_opts *opts)
{
    return create_ctx(out, nx, ny, n, Da, Ra, Pr, porosity, opts, 0, ny, 0, ny);
}

int lbm_init_slab(lbm_ctx **out, int nx, int ny, int y0, int y1, double n, double Da, double Ra, double Pr,
                  double porosity, const lbm_opts *opts)
{
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (ny < 2 || y0 < 0 || y1 > ny || y1 <= y0) return LBM_ERR_ARG;
    if (opts && opts->layout != 0) return LBM_ERR_UNSUPPORTED;
    const int glo = y0 > 0 ? 1 : 0, ghi = y1 < ny ? 1 : 0;
    const int local = y1 - y0 + glo + ghi;
    if (local < 2) return LBM_ERR_ARG;
    return create_ctx(out, nx, local, n, Da, Ra, Pr, porosity, opts, glo, glo + (y1 - y0), y0, ny);
}

int lbm_slab_rows(const lbm_ctx *c, int *y0, int *row_lo, int *row_hi, int *ny_local)
{
    if (!c) return LBM_ERR_ARG;
    if (y0) *y0 = c->y0;
    if (row_lo) *row_lo = c->row_lo;
    if (row_hi) *row_hi = c->row_hi;
    if (ny_local) *ny_local = c->ny;
    return LBM_OK;
}

size_t lbm_halo_bytes(const lbm_ctx *c) { return c ? 4 * (size_t)c->nx * c->dist_elem : 0; }

static bool is_slab(const lbm_ctx *c) { return c->row_lo != 0 || c->row_hi != c->ny || c->ny_glob != c->ny; }

int lbm_halo_pack(lbm_ctx *c, void *d_lo, void *d_hi)
{
    LBM_TRACE("lbm_halo_pack");
    if (!c) return LBM_ERR_ARG;
    if ((d_lo && c->row_lo == 0) || (d_hi && c->row_hi == c->ny)) return LBM_ERR_ARG;   // no neighbour there
    CK(cudaSetDevice(c->device));
    CK(lbm::launch_halo_pack(c, d_lo, d_hi));
    return LBM_OK;
}

int lbm_halo_unpack(lbm_ctx *c, const void *d_lo, const void *d_hi)
{
    LBM_TRACE("lbm_halo_unpack");
    if (!c) return LBM_ERR_ARG;
    if ((d_lo && c->row_lo == 0) || (d_hi && c->row_hi == c->ny)) return LBM_ERR_ARG;
    CK(cudaSetDevice(c->device));
    CK(lbm::launch_halo_unpack(c, d_lo, d_hi));
    return LBM_OK;
}

int lbm_nusselt_sums(lbm_ctx *c, double *hot_sum, double *cold_sum)
{
    if (!c) return LBM_ERR_ARG;
    CK(cudaSetDevice(c->device));
    if (int rc0 = canonical(c)) return rc0;
    CK(lbm::launch_nusselt(c));
    CK(cudaMemcpyAsync(c->h_small + 6, c->d_small + 6, sizeof(double) * 2, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (hot_sum) *hot_sum = c->h_small[6];
    if (cold_sum) *cold_sum = c->h_small[7];
    return LBM_OK;
}

int lbm_residual_sums(lbm_ctx *c, double *sums)
{
    if (!c || !sums) return LBM_ERR_ARG;
    CK(cudaSetDevice(c->device));
    if (int rc0 = canonical(c)) return rc0;
    if (!c->d_snap) CK(cudaMalloc(&c->d_snap, sizeof(double) * 3 * (size_t)c->nx * c->ny));
    const bool first = !c->have_snap;
    CK(lbm::launch_residual(c, first));
    CK(cudaMemcpyAsync(c->h_small + 8, c->d_small + 8, sizeof(double) * 7, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->have_snap = true;
    for (int i = 0; i < 7; i++) sums[i] = c->h_small[8 + i];
    if (first)
        for (int i = 0; i < 3; i++) sums[2 * i] = INFINITY;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_ctx(c);
}

int lbm_set_darcy_field(lbm_ctx *c, const double *Da)
{
    if (!c) return LBM_ERR_ARG;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    drop_graphs(c);   // captured launches hold the old field pointer
    if (!Da) {
        CK(cudaStreamSynchronize(c->stream));
        cudaFree(c->d_da);
        c->d_da = nullptr;
        return LBM_OK;
    }
    const size_t n = (size_t)c->nx * c->ny;
    for (size_t q = 0; q < n; q++)
        if (!(Da[q] > 0) || !isfinite(Da[q])) return LBM_ERR_ARG;
    const size_t es = c->opts.prec == LBM_F64 ? 8 : 4;
    if (!c->d_da) {
        CK(cudaMalloc(&c->d_da, es * (size_t)c->plane));
        CK(cudaMemsetAsync(c->d_da, 0, es * (size_t)c->plane, c->stream));
    }
    if (es == 8) {
        CK(cudaMemcpy2DAsync(c->d_da, c->pitch * es, Da, c->nx * es, c->nx * es, c->ny, cudaMemcpyHostToDevice,
                             c->stream));
        CK(cudaStreamSynchronize(c->stream));
    } else {
        float *tmp = new (std::nothrow) float[n];
        if (!tmp) return LBM_ERR_OOM;
        for (size_t q = 0; q < n; q++) tmp[q] = (float)Da[q];
        const cudaError_t e1 = cudaMemcpy2DAsync(c->d_da, c->pitch * es, tmp, c->nx * es, c->nx * es, c->ny,
                                                 cudaMemcpyHostToDevice, c->stream);
        const cudaError_t e2 = cudaStreamSynchronize(c->stream);
        delete[] tmp;
        CK(e1);
        CK(e2);
    }
    return LBM_OK;
}

int lbm_get_lattice(const lbm_ctx *c, lbm_lattice *out)
{
    if (!c || !out) return LBM_ERR_ARG;
    *out = c->lat;
    return LBM_OK;
}

int lbm_step(lbm_ctx *c, int64_t k)
{
    LBM_TRACE("lbm_step");
    if (!c || k < 0) return LBM_ERR_ARG;
    CK(cudaSetDevice(c->device));
    int64_t t = 0;
    const int G = graph_len_for(c);
    if (G > 0 && k >= G) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        CK(cudaStreamIsCapturing(c->stream, &cs));
        while (cs == cudaStreamCaptureStatusNone && k - t >= G) {
            const int par = graph_parity(c);
            if (!c->step_graph[par]) {
                const int rc = capture_steps(c, G, par);
                if (rc == LBM_ERR_UNSUPPORTED) break;   // this stream cannot be captured: plain launches
                if (rc) return rc;
            }
            if (c->d_step_base) CK(lbm::launch_set_step_base(c));   // the replay's seeds start here
            CK(cudaGraphLaunch(c->step_graph[par], c->stream));
            c->steps += G;   // an even number of steps leaves the parity as it was
            t += G;
        }
    }
    for (; t < k; t++) {
        CK(lbm::launch_step(c));
        c->steps++;   // also the stochastic rounding's step counter
    }
    return LBM_OK;
}

int lbm_synchronize(lbm_ctx *c)
{
    if (!c) return LBM_ERR_ARG;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_fields(lbm_ctx *c, double *rho, double *ux, double *uy, double *T, double *nu)
{
    LBM_TRACE("lbm_fields");
    if (!c) return LBM_ERR_ARG;
    CK(cudaSetDevice(c->device));
    if (int rc0 = canonical(c)) return rc0;
    int rc = ensure_stage(c);
    if (rc) return rc;
    CK(lbm::launch_fields(c, c->d_stage));
    const size_t n = (size_t)c->nx * c->ny;
    double *outs[5] = {rho, ux, uy, T, nu};
    for (int i = 0; i < 5; i++)
        if (outs[i])
            CK(cudaMemcpyAsync(outs[i], c->d_stage + i * n, sizeof(double) * n, cudaMemcpyDeviceToHost,
                               c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_nusselt(lbm_ctx *c, double *hot, double *cold, double *local)
{
    LBM_TRACE("lbm_nusselt");
    if (!c) return LBM_ERR_ARG;
    CK(cudaSetDevice(c->device));
    if (int rc0 = canonical(c)) return rc0;
    CK(lbm::launch_nusselt(c));
    CK(cudaMemcpyAsync(c->h_small, c->d_small, sizeof(double) * 2, cudaMemcpyDeviceToHost, c->stream));
    if (local)
        CK(cudaMemcpyAsync(local, c->d_nuloc, sizeof(double) * c->ny, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (hot) *hot = c->h_small[0];
    if (cold) *cold = c->h_small[1];
    return LBM_OK;
}

int lbm_residual(lbm_ctx *c, double *resid)
{
    LBM_TRACE("lbm_residual");
    if (!c) return LBM_ERR_ARG;
    CK(cudaSetDevice(c->device));
    if (int rc0 = canonical(c)) return rc0;
    if (!c->d_snap) CK(cudaMalloc(&c->d_snap, sizeof(double) * 3 * (size_t)c->nx * c->ny));
    const bool first = !c->have_snap;
    CK(lbm::launch_residual(c, first));
    CK(cudaMemcpyAsync(c->h_small + 2, c->d_small + 2, sizeof(double) * 4, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->have_snap = true;
    double r = c->h_small[2];
    if (c->h_small[3] > r) r = c->h_small[3];
    if (c->h_small[4] > r) r = c->h_small[4];
    if (first) r = INFINITY;
    if (resid) *resid = r;
    if (c->h_small[5] > 0.0) return LBM_ERR_NONFINITE;
    return LBM_OK;
}

int lbm_run_to_steady(lbm_ctx *c, double tol, int64_t max_steps, int64_t *steps_done, double *resid,
                      int *reason)
{
    LBM_TRACE("lbm_run_to_steady");
    if (!c || max_steps < 0 || !(tol >= 0)) return LBM_ERR_ARG;
    if (is_slab(c)) return LBM_ERR_UNSUPPORTED;   // its ghost rows need an exchange every step
    c->have_snap = false;
    double r = INFINITY, best = INFINITY;
    int rc = lbm_residual(c, &r);
    int64_t done = 0;
    int why = 2, since_best = 0;
    while (rc == LBM_OK && done < max_steps) {
        int64_t k = max_steps - done;
        if (k > c->opts.resid_interval) k = c->opts.resid_interval;
        rc = lbm_step(c, k);
        if (rc) break;
        done += k;
        rc = lbm_residual(c, &r);
        if (rc) break;
        if (r < tol) {
            why = 0;
            break;
        }
        if (r < best) {
            best = r;
            since_best = 0;
        } else if (++since_best >= 10 && r < stag_floor(c)) {
            why = 1;
            break;
        }
    }
    if (steps_done) *steps_done = done;
    if (resid) *resid = r;
    if (reason) *reason = why;
    return rc;
}

size_t lbm_state_bytes(const lbm_ctx *c)
{
    if (!c) return 0;
    const size_t n = (size_t)c->nx * c->ny;
    return 14 * n * c->dist_elem + n * c->tau_elem;
}

int lbm_get_state(lbm_ctx *c, void *host, size_t bytes)
{
    if (!c || !host || bytes != lbm_state_bytes(c)) return LBM_ERR_ARG;
    CK(cudaSetDevice(c->device));
    if (int rc0 = canonical(c)) return rc0;
    const size_t es = c->dist_elem, ts = c->tau_elem, n = (size_t)c->nx * c->ny;
    if (int rc0 = copy_planes(c, host, true)) return rc0;
    CK(copy_rows(c, (char *)host + 14 * n * es, c->buf.tau[c->cur], c->nx * ts, c->pitch * ts, (size_t)c->ny,
                 true));
    CK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_set_state(lbm_ctx *c, const void *host, size_t bytes)
{
    if (!c || !host || bytes != lbm_state_bytes(c)) return LBM_ERR_ARG;
    CK(cudaSetDevice(c->device));
    const size_t es = c->dist_elem, ts = c->tau_elem, n = (size_t)c->nx * c->ny;
    c->aa_form_o = false;   // the whole state is replaced by a canonical one
    if (int rc0 = copy_planes(c, const_cast<void *>(host), false)) return rc0;
    CK(copy_rows(c, (char *)const_cast<void *>(host) + 14 * n * es, c->buf.tau[c->cur], c->nx * ts, c->pitch * ts,
                 (size_t)c->ny, false));
    CK(cudaStreamSynchronize(c->stream));
    c->have_snap = false;
    return LBM_OK;
}

// ---- checkpoints: a versioned header, then the native state.
namespace {
const char kCkptMagic[8] = {'L', 'B', 'M', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kCkptVersion = 1;
struct CkptHeader {
    char magic[8];
    uint32_t version, header_bytes;
    int32_t nx, ny, prec, layout, tau_iters, row_lo, row_hi, ny_glob;
    int64_t steps;
    uint64_t seed, state_bytes;
    lbm_lattice lat;
};

bool same_lattice(const lbm_lattice &a, const lbm_lattice &b)
{
    // every parameter the step uses, compared exactly
    return a.nx == b.nx && a.ny == b.ny && a.n == b.n && a.nu_ref == b.nu_ref && a.gamma_scale == b.gamma_scale &&
           a.gamma1 == b.gamma1 && a.gamma2 == b.gamma2 && a.clamp_mode == b.clamp_mode && a.K == b.K &&
           a.eps == b.eps && a.Feps == b.Feps && a.gbeta == b.gbeta && a.Tm == b.Tm && a.tauT == b.tauT &&
           a.s_e == b.s_e && a.s_p == b.s_p && a.T_hot == b.T_hot && a.T_cold == b.T_cold && a.L == b.L &&
           a.tau0 == b.tau0 && a.prec == b.prec;
}
}  // namespace

size_t lbm_checkpoint_bytes(const lbm_ctx *c) { return c ? sizeof(CkptHeader) + lbm_state_bytes(c) : 0; }

int lbm_checkpoint_save(lbm_ctx *c, void *host, size_t bytes)
{
    if (!c || !host || bytes != lbm_checkpoint_bytes(c)) return LBM_ERR_ARG;
    CkptHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kCkptMagic, 8);
    h.version = kCkptVersion;
    h.header_bytes = (uint32_t)sizeof(CkptHeader);
    h.nx = c->nx;
    h.ny = c->ny;
    h.prec = c->opts.prec;
    h.layout = c->opts.layout;
    h.tau_iters = c->opts.tau_iters;
    h.row_lo = c->row_lo;
    h.row_hi = c->row_hi;
    h.ny_glob = c->ny_glob;
    h.steps = c->steps;
    h.seed = c->opts.seed;
    h.state_bytes = lbm_state_bytes(c);
    h.lat = c->lat;
    const int rc = lbm_get_state(c, (char *)host + sizeof(CkptHeader), lbm_state_bytes(c));
    if (rc != LBM_OK) return rc;
    memcpy(host, &h, sizeof(h));
    return LBM_OK;
}

int lbm_checkpoint_load(lbm_ctx *c, const void *host, size_t bytes)
{
    if (!c || !host || bytes != lbm_checkpoint_bytes(c)) return LBM_ERR_ARG;
    CkptHeader h;
    memcpy(&h, host, sizeof(h));
    if (memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != kCkptVersion || h.header_bytes != sizeof(CkptHeader) ||
        h.nx != c->nx || h.ny != c->ny || h.prec != c->opts.prec || h.layout != c->opts.layout ||
        h.tau_iters != c->opts.tau_iters || h.row_lo != c->row_lo || h.row_hi != c->row_hi ||
        h.ny_glob != c->ny_glob || h.seed != c->opts.seed || h.state_bytes != lbm_state_bytes(c) ||
        !same_lattice(h.lat, c->lat) || h.steps < 0)
        return LBM_ERR_ARG;
    const int rc = lbm_set_state(c, (const char *)host + sizeof(CkptHeader), lbm_state_bytes(c));
    if (rc != LBM_OK) return rc;
    c->steps = h.steps;   // the stochastic rounding's seed sequence resumes where it was
    return LBM_OK;
}

int lbm_get_state_f64(lbm_ctx *c, double *f, double *g, double *tau)
{
    if (!c) return LBM_ERR_ARG;
    CK(cudaSetDevice(c->device));
    if (int rc0 = canonical(c)) return rc0;
    int rc = ensure_stage(c);
    if (rc) return rc;
    CK(lbm::launch_export_f64(c, c->d_stage));
    const size_t n = (size_t)c->nx * c->ny;
    if (f) CK(cudaMemcpyAsync(f, c->d_stage, sizeof(double) * 9 * n, cudaMemcpyDeviceToHost, c->stream));
    if (g)
        CK(cudaMemcpyAsync(g, c->d_stage + 9 * n, sizeof(double) * 5 * n, cudaMemcpyDeviceToHost, c->stream));
    if (tau)
        CK(cudaMemcpyAsync(tau, c->d_stage + 14 * n, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_set_state_f64(lbm_ctx *c, const double *f, const double *g, const double *tau)
{
    if (!c) return LBM_ERR_ARG;
    CK(cudaSetDevice(c->device));
    if (int rc0 = canonical(c)) return rc0;
    int rc = ensure_stage(c);
    if (rc) return rc;
    const size_t n = (size_t)c->nx * c->ny;
    int mask = 0;
    if (f) {
        CK(cudaMemcpyAsync(c->d_stage, f, sizeof(double) * 9 * n, cudaMemcpyHostToDevice, c->stream));
        mask |= 1;
    }
    if (g) {
        CK(cudaMemcpyAsync(c->d_stage + 9 * n, g, sizeof(double) * 5 * n, cudaMemcpyHostToDevice, c->stream));
        mask |= 2;
    }
    if (tau) {
        CK(cudaMemcpyAsync(c->d_stage + 14 * n, tau, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
        mask |= 4;
    }
    if (mask) CK(lbm::launch_import_f64(c, c->d_stage, mask));
    CK(cudaStreamSynchronize(c->stream));
    c->have_snap = false;
    return LBM_OK;
}

const char *lbm_strerror(int code)
{
    switch (code) {
    case LBM_OK: return "LBM_OK";
    case LBM_ERR_ARG: return "LBM_ERR_ARG: invalid argument";
    case LBM_ERR_UNSTABLE: return "LBM_ERR_UNSTABLE: relaxation time <= 1/2";
    case LBM_ERR_NONFINITE: return "LBM_ERR_NONFINITE: NaN or Inf in the fields";
    case LBM_ERR_CUDA: return "LBM_ERR_CUDA: CUDA runtime error";
    case LBM_ERR_OOM: return "LBM_ERR_OOM: device allocation failed";
    case LBM_ERR_TIMEOUT: return "LBM_ERR_TIMEOUT: bounded device wait gave up";
    case LBM_ERR_UNSUPPORTED: return "LBM_ERR_UNSUPPORTED: option not built";
    case LBM_ERR_SIZE: return "LBM_ERR_SIZE: grid larger than the fixed scratch area";
    default: return "unknown lbm error";
    }
}

const char *lbm_last_cuda_error(void) { return g_last_cuda; }

}  // extern "C"
