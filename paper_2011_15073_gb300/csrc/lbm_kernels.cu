// lbm_kernels.cu -- kernels of the fused MRT step and its reductions, with
// their host launchers, instantiated for every storage precision.
#include <math.h>

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_step.cuh"

namespace lbm {

// ---------------------------------------------------------------- kernels
template <int PREC>
__global__ void init_kernel(typename Store<PREC>::S *__restrict__ dist,
                            typename Store<PREC>::TauS *__restrict__ tau,
                            Phys<typename Store<PREC>::R> p, double tau0, double T0)
{
    using St = Store<PREC>;
    using R = typename St::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= p.nx) return;
    const int64_t k = (int64_t)y * p.pitch + x;
    for (int i = 0; i < 9; i++) St::st(dist, i * p.plane + k, R(rest_f(i)), R(rest_f(i)));
    for (int i = 0; i < 5; i++) {
        const R v = R(rest_g(i) * 2.0 * T0);  // w_i T0 (rest_g holds w_i / 2)
        St::st(dist + 9 * p.plane, i * p.plane + k, v, R(rest_g(i)));
    }
    tau[k] = typename St::TauS(tau0);
}

// One time step of the whole cavity (pull scheme, two buffers); the node
// and tile bodies are in lbm_step.cuh.  TAU 1: node-local implicit tau (the
// tau planes are neither read nor written).
template <int PREC, int FIELD, int TAU>
__global__ void __launch_bounds__(128)
step_kernel(const typename Store<PREC>::S *__restrict__ src, typename Store<PREC>::S *__restrict__ dst,
            const typename Store<PREC>::TauS *__restrict__ tsrc, typename Store<PREC>::TauS *__restrict__ tdst,
            Phys<typename Store<PREC>::R> p)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= p.nx) return;
    step_node<PREC, typename Store<PREC>::R, FIELD, TAU>(src, dst, tsrc, tdst, p, x, y, p.seed);
}

template <int PREC, int FIELD, int TAU>
__global__ void __launch_bounds__(128)
step2_kernel(const typename Store<PREC>::S *__restrict__ src, typename Store<PREC>::S *__restrict__ dst,
             const float *__restrict__ tsrc, float *__restrict__ tdst, Phys<float> p, Phys<F2> p2)
{
    step2_tile<PREC, FIELD, TAU>(src, dst, tsrc, tdst, p, p2, blockIdx.x * 256, blockIdx.y, p.seed);
}

// Four nodes per thread (16-bit storages): 64-thread blocks of 256 nodes,
// at most 96 registers so that ten blocks (20 warps) fit on an SM: more
// bytes in flight per SM than the 64-80-register blocks of step2_kernel
// (measured against caps of 80 and 128 registers: both slower; 128-thread
// blocks at five per SM: 2 % slower).
template <int PREC, int FIELD, int TAU>
__global__ void __launch_bounds__(64, 10)
step4_kernel(const typename Store<PREC>::S *__restrict__ src, typename Store<PREC>::S *__restrict__ dst,
             const float *__restrict__ tsrc, float *__restrict__ tdst, Phys<float> p, Phys<F2> p2)
{
    step4_tile<PREC, FIELD, TAU>(src, dst, tsrc, tdst, p, p2, blockIdx.x * 256, blockIdx.y, [&] { return p.seed; });
}

// The step kernels of a replayed step graph with the stochastic-rounding
// storages.  A graph replays its launches' arguments, so the seed cannot be
// one: it is computed here from the step count the replay starts at (*base,
// written on the device before each replay) plus the launch's place s in the
// graph -- the seed a plain launch gets from the host at that step.  Plain
// launches keep the constant seed (reading it from memory costs the hot
// kernels a register and 3-5 %).
struct GraphSeed {
    const long long *base;
    int s;
    uint32_t run;
};
__device__ __forceinline__ uint32_t graph_seed(GraphSeed g) { return step_seed((uint64_t)(*g.base + g.s), g.run); }

template <int PREC, int FIELD, int TAU>
__global__ void __launch_bounds__(128)
step2_graph_kernel(const typename Store<PREC>::S *__restrict__ src, typename Store<PREC>::S *__restrict__ dst,
                   const float *__restrict__ tsrc, float *__restrict__ tdst, Phys<float> p, Phys<F2> p2,
                   GraphSeed g)
{
    step2_tile<PREC, FIELD, TAU>(src, dst, tsrc, tdst, p, p2, blockIdx.x * 256, blockIdx.y, graph_seed(g));
}

template <int PREC, int FIELD, int TAU>
__global__ void __launch_bounds__(64, 10)
step4_graph_kernel(const typename Store<PREC>::S *__restrict__ src, typename Store<PREC>::S *__restrict__ dst,
                   const float *__restrict__ tsrc, float *__restrict__ tdst, Phys<float> p, Phys<F2> p2,
                   GraphSeed g)
{
    step4_tile<PREC, FIELD, TAU>(src, dst, tsrc, tdst, p, p2, blockIdx.x * 256, blockIdx.y,
                                 [&] { return graph_seed(g); });
}

__global__ void set_step_base_kernel(long long *base, long long steps)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *base = steps;
}

// tau the next collision of every node starts from, in implicit mode (the
// solve of implicit_tau on the streamed populations) -> out[ny][nx].
template <int PREC, bool REV>
__global__ void tau_next_kernel(const typename Store<PREC>::S *__restrict__ src,
                                Phys<typename Store<PREC>::R> p, double *__restrict__ out)
{
    using R = typename Store<PREC>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= p.nx) return;
    R f[9], g[5];
    pull<PREC, R, REV>(src, p, x, y, f, g);
    out[(int64_t)y * p.nx + x] = double(implicit_tau<R>(p, f, g, (int64_t)y * p.pitch + x));
}

// Streamed macroscopic fields: rho, u_x, u_y, T, nu -> out[5][ny][nx].
// REV: the state is in the in-place layout's canonical form (f*_i in plane
// opp(i)).
template <int PREC, bool REV>
__global__ void fields_kernel(const typename Store<PREC>::S *__restrict__ src,
                              const typename Store<PREC>::TauS *__restrict__ tsrc,
                              Phys<typename Store<PREC>::R> p, double *__restrict__ out)
{
    using St = Store<PREC>;
    using R = typename St::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= p.nx) return;
    const int64_t k = (int64_t)y * p.pitch + x;
    const int64_t q = (int64_t)y * p.nx + x, n = (int64_t)p.nx * p.ny;
    R f[9], g[5];
    pull<PREC, R, REV>(src, p, x, y, f, g);
    Macro<R> m;
    collide<R>(p, f, g, p.tau_iters ? implicit_tau<R>(p, f, g, k) : R(tsrc[k]), m, k);
    out[q] = double(m.rho);
    out[n + q] = double(m.ux);
    out[2 * n + q] = double(m.uy);
    out[3 * n + q] = double(m.T);
    out[4 * n + q] = double(m.nu);
}

// FP64 block sum of one value (blockDim.x a multiple of 32, <= 1024); the
// reduction tree is fixed, so results are reproducible run to run.
__device__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < nw ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

// Streamed temperature of node (x, y) in FP64 (thermal part of the pull).
template <int PREC, bool REV>
__device__ double streamed_T(const typename Store<PREC>::S *__restrict__ src,
                             const Phys<typename Store<PREC>::R> &p, int x, int y)
{
    using R = typename Store<PREC>::R;
    R f[9], g[5];
    pull<PREC, R, REV>(src, p, x, y, f, g);
    return (double)g[0] + (double)g[1] + (double)g[2] + (double)g[3] + (double)g[4];
}

// Wall Nusselt numbers: one block; row j of the hot wall gets
// Nu_j = -L (9 theta_0 - theta_1 - 8) / 3, the cold wall the outward
// L (9 theta_{nx-1} - theta_{nx-2}) / 3, theta = (T - T_c) / (T_h - T_c).
// Rows [row_lo, row_hi) (all rows of a whole cavity, the interior rows of a
// slab); small[0..1] the averages over them, small[6..7] the sums.
template <int PREC, bool REV>
__global__ void __launch_bounds__(256)
nusselt_kernel(const typename Store<PREC>::S *__restrict__ src, Phys<typename Store<PREC>::R> p,
               double T_hot, double T_cold, double Lw, double *__restrict__ small,
               double *__restrict__ nuloc, int row_lo, int row_hi)
{
    __shared__ double sh[32];
    const double dT = T_hot - T_cold;
    double sh_hot = 0.0, sh_cold = 0.0;
    for (int j = row_lo + threadIdx.x; j < row_hi; j += blockDim.x) {
        const double t0 = (streamed_T<PREC, REV>(src, p, 0, j) - T_cold) / dT;
        const double t1 = (streamed_T<PREC, REV>(src, p, 1, j) - T_cold) / dT;
        const double ta = (streamed_T<PREC, REV>(src, p, p.nx - 1, j) - T_cold) / dT;
        const double tb = (streamed_T<PREC, REV>(src, p, p.nx - 2, j) - T_cold) / dT;
        const double nh = -Lw * (9.0 * t0 - t1 - 8.0) / 3.0;
        const double nc = Lw * (9.0 * ta - tb) / 3.0;
        nuloc[j] = nh;
        sh_hot += nh;
        sh_cold += nc;
    }
    const double a = block_sum(sh_hot, sh);
    const double b = block_sum(sh_cold, sh);
    if (threadIdx.x == 0) {
        small[0] = a / (row_hi - row_lo);
        small[1] = b / (row_hi - row_lo);
        small[6] = a;
        small[7] = b;
    }
}

// Convergence residual, pass 1: each block accumulates, over a fixed
// grid-stride set of the nodes of rows [row_lo, row_hi), sum (phi -
// phi_prev)^2 and sum phi^2 for phi in {u_x, u_y, T} plus a count of
// non-finite values, and writes its seven partial sums to
// part[blockIdx.x * 8 + 0..6].  The snapshot is updated.
template <int PREC, bool REV>
__global__ void __launch_bounds__(256)
residual_kernel(const typename Store<PREC>::S *__restrict__ src,
                const typename Store<PREC>::TauS *__restrict__ tsrc, Phys<typename Store<PREC>::R> p,
                double *__restrict__ snap, double *__restrict__ part, int first, int row_lo, int row_hi)
{
    using R = typename Store<PREC>::R;
    __shared__ double sh[32];
    const int64_t n = (int64_t)p.nx * p.ny;
    const int64_t q_end = (int64_t)p.nx * row_hi;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t q = (int64_t)p.nx * row_lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < q_end;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(q / p.nx), x = (int)(q - (int64_t)y * p.nx);
        R f[9], g[5];
        pull<PREC, R, REV>(src, p, x, y, f, g);
        const int64_t k = (int64_t)y * p.pitch + x;
        const Macro<R> m = macro<R>(p, f, g, p.tau_iters ? implicit_tau<R>(p, f, g, k) : R(tsrc[k]), k);
        const double v[3] = {double(m.ux), double(m.uy), double(m.T)};
        for (int c = 0; c < 3; c++) {
            const double old = first ? v[c] : snap[c * n + q];
            const double d = v[c] - old;
            acc[2 * c] += d * d;
            acc[2 * c + 1] += v[c] * v[c];
            if (!isfinite(v[c])) acc[6] += 1.0;
            snap[c * n + q] = v[c];
        }
    }
    for (int c = 0; c < 7; c++) {
        const double s = block_sum(acc[c], sh);
        if (threadIdx.x == 0) part[blockIdx.x * 8 + c] = s;
    }
}

// Pass 2: one block sums the partials in block order and writes
// small[2..4] = relative change of u_x, u_y, T, small[5] = non-finite count
// and small[8..14] the seven totals (the sums a decomposed run adds up).
__global__ void __launch_bounds__(256)
residual_final_kernel(const double *__restrict__ part, int nb, double *__restrict__ small)
{
    __shared__ double sh[32];
    double tot[7];
    for (int c = 0; c < 7; c++) {
        double a = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) a += part[b * 8 + c];
        tot[c] = block_sum(a, sh);
    }
    if (threadIdx.x == 0) {
        for (int c = 0; c < 3; c++) {
            const double num = tot[2 * c], den = tot[2 * c + 1];
            small[2 + c] = den > 0.0 ? sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
        }
        small[5] = tot[6];
        for (int c = 0; c < 7; c++) small[8 + c] = tot[c];
    }
}

// FP64 staging [15][ny][nx] (f0..f8, g0..g4, tau) <-> device state.
template <int PREC, bool REV>
__global__ void import_kernel(const double *__restrict__ in, typename Store<PREC>::S *__restrict__ dist,
                              typename Store<PREC>::TauS *__restrict__ tau, int nx, int ny,
                              int64_t pitch, int64_t plane, int mask)
{
    using St = Store<PREC>;
    using R = typename St::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    const int64_t k = (int64_t)y * pitch + x, q = (int64_t)y * nx + x, n = (int64_t)nx * ny;
    if (mask & 1)
        for (int i = 0; i < 9; i++) {
            const int j = REV ? opp(i) : i;
            St::st(dist, j * plane + k, R(in[i * n + q]), R(rest_f(j)));
        }
    if (mask & 2)
        for (int i = 0; i < 5; i++) {
            const int j = REV ? opp(i) : i;
            St::st(dist + 9 * plane, j * plane + k, R(in[(9 + i) * n + q]), R(rest_g(j)));
        }
    if (mask & 4) tau[k] = typename St::TauS(in[14 * n + q]);
}

template <int PREC, bool REV>
__global__ void export_kernel(double *__restrict__ out, const typename Store<PREC>::S *__restrict__ dist,
                              const typename Store<PREC>::TauS *__restrict__ tau, int nx, int ny,
                              int64_t pitch, int64_t plane)
{
    using St = Store<PREC>;
    using R = typename St::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    const int64_t k = (int64_t)y * pitch + x, q = (int64_t)y * nx + x, n = (int64_t)nx * ny;
    for (int i = 0; i < 9; i++) {
        const int j = REV ? opp(i) : i;
        out[i * n + q] = double(St::ld(dist, j * plane + k, R(rest_f(j))));
    }
    for (int i = 0; i < 5; i++) {
        const int j = REV ? opp(i) : i;
        out[(9 + i) * n + q] = double(St::ld(dist + 9 * plane, j * plane + k, R(rest_g(j))));
    }
    out[14 * n + q] = double(tau[k]);
}

// ------------------------------------------------------------- launchers
static dim3 node_grid(const lbm_ctx *c, int bx) { return dim3((c->nx + bx - 1) / bx, c->ny); }

// Seed source of a launch being captured into a step graph (capture_s: its
// place in the graph).
static GraphSeed graph_seed_of(const lbm_ctx *c)
{
    return GraphSeed{c->d_step_base, c->capture_s, run_word(c->opts.seed)};
}

int residual_blocks(const lbm_ctx *c)
{
    const int64_t n = (int64_t)c->nx * c->ny;
    int64_t nb = (n + 255) / 256;
    if (nb > 152 * 8) nb = 152 * 8;
    return (int)(nb < 1 ? 1 : nb);
}

template <int PREC>
static cudaError_t init_t(lbm_ctx *c)
{
    using St = Store<PREC>;
    for (int b = 0; b < 2; b++)
        if (c->buf.dist[b])
        init_kernel<PREC><<<node_grid(c, 128), 128, 0, c->stream>>>(
            (typename St::S *)c->buf.dist[b], (typename St::TauS *)c->buf.tau[b],
            make_params<typename St::R>(c), c->lat.tau0, 0.5 * (c->lat.T_hot + c->lat.T_cold));
    return cudaGetLastError();
}

template <int PREC, int TAU>
static cudaError_t step_buffers_tau(lbm_ctx *c, const void *src, void *dst, const void *tsrc, void *tdst)
{
    using St = Store<PREC>;
    if constexpr (PREC == LBM_F64) {
        auto *kern = c->d_da ? step_kernel<PREC, 1, TAU> : step_kernel<PREC, 0, TAU>;
        kern<<<node_grid(c, 128), 128, 0, c->stream>>>(
            (const typename St::S *)src, (typename St::S *)dst, (const typename St::TauS *)tsrc,
            (typename St::TauS *)tdst, make_params<typename St::R>(c));
    } else {
        if constexpr (rounds_stochastically(PREC)) {
            if (c->capture_s >= 0) {   // a launch captured into a step graph
                auto *kern = c->d_da ? step2_graph_kernel<PREC, 1, TAU> : step2_graph_kernel<PREC, 0, TAU>;
                kern<<<node_grid(c, 256), 128, 0, c->stream>>>(
                    (const typename St::S *)src, (typename St::S *)dst, (const float *)tsrc, (float *)tdst,
                    make_params<float>(c), make_params<F2>(c), graph_seed_of(c));
                return cudaGetLastError();
            }
        }
        auto *kern = c->d_da ? step2_kernel<PREC, 1, TAU> : step2_kernel<PREC, 0, TAU>;
        kern<<<node_grid(c, 256), 128, 0, c->stream>>>(
            (const typename St::S *)src, (typename St::S *)dst, (const float *)tsrc, (float *)tdst,
            make_params<float>(c), make_params<F2>(c));
    }
    return cudaGetLastError();
}

// How the step kernel gets its inputs (lbm_opts.staging, resolved): 1
// straight into registers, two nodes per thread; 3 straight into registers,
// four nodes per thread (16-bit storages only; lbm_init refuses it elsewhere,
// and refuses 2 everywhere).  0 picks 3 for those
// storages on grids of at least 2048 x 2048 nodes with lagged tau, or
// 4096 x 4096 with the implicit tau, else 1.  Measured: 8-21 % faster at
// 4096^2 (the Darcy-field form gains most), 8 % at 2048^2 with lagged tau
// but 2 % slower with the implicit one, and slower at 1024^2, where the
// 128-node warps at the side walls update a larger share of each row one
// node at a time.
static int staging_of(const lbm_ctx *c)
{
    if (c->opts.prec == LBM_F64) return 1;
    if (c->opts.staging != 0) return c->opts.staging;
    const bool p16 = c->opts.prec == LBM_BF16D || c->opts.prec == LBM_F16D || c->opts.prec == LBM_F16S ||
                     c->opts.prec == LBM_BF16S;
    const int min_side = c->opts.tau_iters > 0 ? 4096 : 2048;
    if (p16 && c->nx >= min_side && c->ny_glob >= min_side) return 3;
    return 1;
}

template <int PREC, int TAU>
static cudaError_t step4_buffers_tau(lbm_ctx *c, const void *src, void *dst, const void *tsrc, void *tdst)
{
    using St = Store<PREC>;
    if constexpr (rounds_stochastically(PREC)) {
        if (c->capture_s >= 0) {   // a launch captured into a step graph
            auto *kern = c->d_da ? step4_graph_kernel<PREC, 1, TAU> : step4_graph_kernel<PREC, 0, TAU>;
            kern<<<node_grid(c, 256), 64, 0, c->stream>>>((const typename St::S *)src, (typename St::S *)dst,
                                                          (const float *)tsrc, (float *)tdst, make_params<float>(c),
                                                          make_params<F2>(c), graph_seed_of(c));
            return cudaGetLastError();
        }
    }
    auto *kern = c->d_da ? step4_kernel<PREC, 1, TAU> : step4_kernel<PREC, 0, TAU>;
    kern<<<node_grid(c, 256), 64, 0, c->stream>>>((const typename St::S *)src, (typename St::S *)dst,
                                                  (const float *)tsrc, (float *)tdst, make_params<float>(c),
                                                  make_params<F2>(c));
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t step4_buffers(lbm_ctx *c, const void *src, void *dst, const void *tsrc, void *tdst)
{
    if constexpr (is16<PREC>())
        return c->opts.tau_iters > 0 ? step4_buffers_tau<PREC, 1>(c, src, dst, tsrc, tdst)
                                     : step4_buffers_tau<PREC, 0>(c, src, dst, tsrc, tdst);
    return cudaErrorInvalidValue;
}

template <int PREC>
static cudaError_t step_buffers_t(lbm_ctx *c, const void *src, void *dst, const void *tsrc, void *tdst)
{
    const int how = staging_of(c);
    if (how == 3) return step4_buffers<PREC>(c, src, dst, tsrc, tdst);
    return c->opts.tau_iters > 0 ? step_buffers_tau<PREC, 1>(c, src, dst, tsrc, tdst)
                                 : step_buffers_tau<PREC, 0>(c, src, dst, tsrc, tdst);
}

template <int PREC>
static cudaError_t step_t(lbm_ctx *c)
{
    using St = Store<PREC>;
    if (c->opts.layout == 1) return launch_aa_step(c);
    const int s = c->cur, d = 1 - c->cur;
    const cudaError_t e = step_buffers_t<PREC>(c, c->buf.dist[s], c->buf.dist[d], c->buf.tau[s], c->buf.tau[d]);
    c->cur = d;
    return e;
}

template <int PREC>
static cudaError_t fields_t(lbm_ctx *c, double *out)
{
    using St = Store<PREC>;
    auto *kern = c->opts.layout == 1 ? fields_kernel<PREC, true> : fields_kernel<PREC, false>;
    kern<<<node_grid(c, 128), 128, 0, c->stream>>>(
        (const typename St::S *)c->buf.dist[c->cur], (const typename St::TauS *)c->buf.tau[c->cur],
        make_params<typename St::R>(c), out);
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t nusselt_t(lbm_ctx *c)
{
    using St = Store<PREC>;
    auto *kern = c->opts.layout == 1 ? nusselt_kernel<PREC, true> : nusselt_kernel<PREC, false>;
    kern<<<1, 256, 0, c->stream>>>(
        (const typename St::S *)c->buf.dist[c->cur], make_params<typename St::R>(c), c->lat.T_hot,
        c->lat.T_cold, c->lat.L, c->d_small, c->d_nuloc, c->row_lo, c->row_hi);
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t residual_t(lbm_ctx *c, bool first)
{
    using St = Store<PREC>;
    const int nb = residual_blocks(c);
    auto *kern = c->opts.layout == 1 ? residual_kernel<PREC, true> : residual_kernel<PREC, false>;
    kern<<<nb, 256, 0, c->stream>>>(
        (const typename St::S *)c->buf.dist[c->cur], (const typename St::TauS *)c->buf.tau[c->cur],
        make_params<typename St::R>(c), c->d_snap, c->d_part, first ? 1 : 0, c->row_lo, c->row_hi);
    residual_final_kernel<<<1, 256, 0, c->stream>>>(c->d_part, nb, c->d_small);
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t import_t(lbm_ctx *c, const double *in, int mask)
{
    using St = Store<PREC>;
    auto *kern = c->opts.layout == 1 ? import_kernel<PREC, true> : import_kernel<PREC, false>;
    kern<<<node_grid(c, 128), 128, 0, c->stream>>>(
        in, (typename St::S *)c->buf.dist[c->cur], (typename St::TauS *)c->buf.tau[c->cur], c->nx, c->ny,
        c->pitch, c->plane, mask);
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t export_t(lbm_ctx *c, double *out)
{
    using St = Store<PREC>;
    auto *kern = c->opts.layout == 1 ? export_kernel<PREC, true> : export_kernel<PREC, false>;
    kern<<<node_grid(c, 128), 128, 0, c->stream>>>(
        out, (const typename St::S *)c->buf.dist[c->cur], (const typename St::TauS *)c->buf.tau[c->cur],
        c->nx, c->ny, c->pitch, c->plane);
    if (c->opts.tau_iters > 0) {  // no stored tau: report the next collision's implicit tau
        auto *tk = c->opts.layout == 1 ? tau_next_kernel<PREC, true> : tau_next_kernel<PREC, false>;
        tk<<<node_grid(c, 128), 128, 0, c->stream>>>((const typename St::S *)c->buf.dist[c->cur],
                                                     make_params<typename St::R>(c),
                                                     out + (int64_t)14 * c->nx * c->ny);
    }
    return cudaGetLastError();
}

// Halo exchange of a row slab.  Populations that leave a slab through its
// upper cut are those with e_y = +1 (f2, f5, f6 and g2: planes 2, 5, 6, 11),
// read from the top interior row; through its lower cut those with e_y = -1
// (f4, f7, f8, g4: planes 4, 7, 8, 13), read from the bottom interior row.
// A neighbour writes what it receives into the ghost row its pull reads
// them from.  Buffers hold 4 x nx values of the storage type, plane-major.
__device__ __forceinline__ int up_plane(int q) { return q == 0 ? 2 : (q == 1 ? 5 : (q == 2 ? 6 : 11)); }
__device__ __forceinline__ int down_plane(int q) { return q == 0 ? 4 : (q == 1 ? 7 : (q == 2 ? 8 : 13)); }

template <class E>
__global__ void halo_pack_kernel(const E *__restrict__ dist, int64_t plane, int64_t pitch, int nx, int row_lo,
                                 int row_hi, E *__restrict__ lo, E *__restrict__ hi)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
    if (x >= nx) return;
    if (hi) hi[(int64_t)q * nx + x] = dist[up_plane(q) * plane + (int64_t)(row_hi - 1) * pitch + x];
    if (lo) lo[(int64_t)q * nx + x] = dist[down_plane(q) * plane + (int64_t)row_lo * pitch + x];
}

template <class E>
__global__ void halo_unpack_kernel(E *__restrict__ dist, int64_t plane, int64_t pitch, int nx, int ny,
                                   const E *__restrict__ lo, const E *__restrict__ hi)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
    if (x >= nx) return;
    // from below: the lower neighbour's upward populations, into ghost row 0
    if (lo) dist[up_plane(q) * plane + x] = lo[(int64_t)q * nx + x];
    // from above: the upper neighbour's downward populations, into ghost row ny - 1
    if (hi) dist[down_plane(q) * plane + (int64_t)(ny - 1) * pitch + x] = hi[(int64_t)q * nx + x];
}

template <class E>
static cudaError_t halo_t(lbm_ctx *c, void *lo, void *hi, const void *rlo, const void *rhi, bool pack)
{
    const dim3 grid((c->nx + 255) / 256, 4);
    E *dist = (E *)c->buf.dist[c->cur];
    if (pack)
        halo_pack_kernel<E><<<grid, 256, 0, c->stream>>>(dist, c->plane, c->pitch, c->nx, c->row_lo, c->row_hi,
                                                         (E *)lo, (E *)hi);
    else
        halo_unpack_kernel<E><<<grid, 256, 0, c->stream>>>(dist, c->plane, c->pitch, c->nx, c->ny,
                                                           (const E *)rlo, (const E *)rhi);
    return cudaGetLastError();
}

static cudaError_t halo(lbm_ctx *c, void *lo, void *hi, const void *rlo, const void *rhi, bool pack)
{
    switch (c->dist_elem) {
    case 2: return halo_t<uint16_t>(c, lo, hi, rlo, rhi, pack);
    case 4: return halo_t<uint32_t>(c, lo, hi, rlo, rhi, pack);
    case 8: return halo_t<uint64_t>(c, lo, hi, rlo, rhi, pack);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_halo_pack(lbm_ctx *c, void *d_lo, void *d_hi) { return halo(c, d_lo, d_hi, nullptr, nullptr, true); }
cudaError_t launch_halo_unpack(lbm_ctx *c, const void *d_lo, const void *d_hi)
{
    return halo(c, nullptr, nullptr, d_lo, d_hi, false);
}

#define LBM_DISPATCH(fn, ...)                                      \
    switch (c->opts.prec) {                                        \
    case LBM_F64: return fn<LBM_F64>(__VA_ARGS__);                 \
    case LBM_F32: return fn<LBM_F32>(__VA_ARGS__);                 \
    case LBM_BF16D: return fn<LBM_BF16D>(__VA_ARGS__);             \
    case LBM_F16D: return fn<LBM_F16D>(__VA_ARGS__);               \
    case LBM_F32D: return fn<LBM_F32D>(__VA_ARGS__);               \
    case LBM_F16S: return fn<LBM_F16S>(__VA_ARGS__);               \
    case LBM_BF16S: return fn<LBM_BF16S>(__VA_ARGS__);             \
    default: return cudaErrorInvalidValue;                         \
    }

cudaError_t launch_init(lbm_ctx *c) { LBM_DISPATCH(init_t, c) }
cudaError_t launch_set_step_base(lbm_ctx *c)
{
    set_step_base_kernel<<<1, 32, 0, c->stream>>>(c->d_step_base, (long long)c->steps);
    return cudaGetLastError();
}

cudaError_t launch_step(lbm_ctx *c) { LBM_DISPATCH(step_t, c) }
cudaError_t launch_step_buffers(lbm_ctx *c, const void *src, void *dst, const void *tsrc, void *tdst)
{
    LBM_DISPATCH(step_buffers_t, c, src, dst, tsrc, tdst)
}
cudaError_t launch_fields(lbm_ctx *c, double *out) { LBM_DISPATCH(fields_t, c, out) }
cudaError_t launch_nusselt(lbm_ctx *c) { LBM_DISPATCH(nusselt_t, c) }
cudaError_t launch_residual(lbm_ctx *c, bool first) { LBM_DISPATCH(residual_t, c, first) }
cudaError_t launch_import_f64(lbm_ctx *c, const double *in, int mask) { LBM_DISPATCH(import_t, c, in, mask) }
cudaError_t launch_export_f64(lbm_ctx *c, double *out) { LBM_DISPATCH(export_t, c, out) }

}  // namespace lbm
