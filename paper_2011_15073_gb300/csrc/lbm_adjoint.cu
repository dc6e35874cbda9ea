// lbm_adjoint.cu -- discrete adjoint of the hot-wall average Nusselt number
// through a run of the fused step (two-buffer layout), with checkpoints.
//
// J = Nu_hot(s_T) after T steps from s_0.  With s_{t+1} = C(P(s_t)) (P the
// pull with the wall rules, C the per-node collision), the adjoint state
// lambda_t = dJ/ds_t obeys lambda_t = P^T C'^T lambda_{t+1}.  P maps every
// post-collision slot to exactly one pulled value (a neighbour, or the node
// itself across a wall, negated by the anti-bounce-back), so P^T is a scatter
// in which every slot is written once: no atomics.  Parameter gradients
// accumulate in FP64 over the steps: the per-node Darcy number in a plane
// that each node owns, n and Ra in one slot per block (fixed order), reduced
// once at the end.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "lbm_adjoint.cuh"
#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_trace.h"
#include "lbm_step.cuh"

namespace {

using namespace lbm;

// Parameters of the chain from (n, Ra, Da) to the lattice coefficients,
// with the per-case constants of the parameter gradients computed once on
// the host: dn = a_nu dJ/dnu_ref + dJ/d(n - 1), dRa = b_nu dJ/dnu_ref +
// b_wT dJ/d(1/tauT), and 1/Da for a uniform Darcy number.
struct Chain {
    double n, Ra, tauT;  // power-law index, Rayleigh number, thermal tau
    double a_nu;         // d nu_ref / dn = nu_ref ln(Ra) / 2
    double b_nu;         // d nu_ref / dRa = -nu_ref (2 - n) / (2 Ra)
    double b_wT;         // d (1/tauT) / dRa = (tauT - 1/2) / (2 Ra tauT^2)
    double inv_Da;       // 1 / Da of a uniform permeability
};

// The constants the reverse step reads, in its compute type: rounded once on
// the host (to nearest, as a conversion in the kernel would), so the FP32
// kernel spends no FP64-pipe conversions on them.
template <class V>
struct ChainV {
    V a_nu, b_nu, b_wT, inv_Da;
};

// Programmatic dependent launch: a reverse step lets the next one be
// launched as soon as all its blocks have started, and that one loads the
// recomputed state (written before the stage began) and then waits for the
// whole previous step to complete before it reads or writes an adjoint or
// gradient buffer.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void allow_dependent_launch() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ void wait_for_previous_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Seed: lambda_T = dJ/ds_T.  Nu_hot = mean_j -L (9 theta_0 - theta_1 - 8)/3
// with theta = (T - T_c)/(T_h - T_c) and T the sum of the pulled g at
// columns 0 and 1; every pulled value there reads exactly one slot.
template <class V>
__global__ void adj_seed_kernel(V *__restrict__ lam, Phys<V> p, double coef0, double coef1)
{
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= p.ny) return;
    const int64_t P = p.plane, W = p.pitch;
    V *G = lam + 9 * P;
    for (int col = 0; col < 2 && col < p.nx; col++) {
        const V a = V(col == 0 ? coef0 : coef1);
        const int x = col;
        const int64_t k = (int64_t)y * W + x;
        const bool xl = x > 0, xr = x < p.nx - 1, yb = y > 0, yt = y < p.ny - 1;
        // pulled g_i(x) reads: g0 own; g1 from x-1 or -(own g3) at the hot wall;
        // g2 from y-1 or own g4; g3 from x+1 or -(own g1); g4 from y+1 or own g2
        G[0 * P + k] += a;
        if (xl) G[1 * P + k - 1] += a; else G[3 * P + k] += -a;
        if (yb) G[2 * P + k - W] += a; else G[4 * P + k] += a;
        if (xr) G[3 * P + k + 1] += a; else G[1 * P + k] += -a;
        if (yt) G[4 * P + k + W] += a; else G[2 * P + k] += a;
    }
}

// Sum of v over a block of 128 threads (fixed order); thread 0 gets it.
// Within a warp the sum runs in the compute type (for the FP32 adjoint:
// FP32 shuffles and adds, where the FP64 pipe of this part runs at 1/64 of
// the FP32 rate and a per-thread FP64 reduction was a serial tail of every
// reverse step), across the four warps in FP64.
template <class V>
__device__ __forceinline__ double block128_sum(V v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = double(v);
    __syncthreads();
    const double t = threadIdx.x == 0 ? (sh[0] + sh[1]) + (sh[2] + sh[3]) : 0.0;
    __syncthreads();
    return t;
}

// One reverse step: lam_out (adjoint of s_{t+1}) -> lam_in (adjoint of s_t),
// recomputing the collision of every node from s_t.  The per-node Darcy
// gradient accumulates in gDa (FP64, one slot per node); the n and Ra
// gradients are summed over the block and accumulate in the block's slot of
// gnb / gRab (FP64; fixed order, so the result is deterministic).
template <int PREC, class V>
__global__ void __launch_bounds__(128)
adj_step_kernel(const typename Store<PREC>::S *__restrict__ st, const typename Store<PREC>::TauS *__restrict__ tst,
                const V *__restrict__ lam_out, V *__restrict__ lam_in, double *__restrict__ gDa,
                double *__restrict__ gnb, double *__restrict__ gRab, Phys<V> p, ChainV<V> ch)
{
    __shared__ double sh[4];
    allow_dependent_launch();
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    const bool in = x < p.nx;
    const int64_t P = p.plane, W = p.pitch;
    const int64_t k = (int64_t)y * W + (in ? x : 0);
    V f[9], g[5];
    V tau_prev = V(1);
    if (in) {
        pull<PREC, V>(st, p, x, y, f, g);
        tau_prev = V(tst[k]);
    }
    wait_for_previous_grid();
    V dn = V(0), dRa = V(0);
    if (in) {
    // the adjoint of s_{t+1}, written by the previous step: read at L2
    // (never from a line an earlier kernel left in this SM's L1)
    V fo[9], go[5];
#pragma unroll
    for (int i = 0; i < 9; i++) fo[i] = __ldcg(lam_out + i * P + k);
#pragma unroll
    for (int i = 0; i < 5; i++) go[i] = __ldcg(lam_out + (9 + i) * P + k);
    const V tb_new = __ldcg(lam_out + 14 * P + k);
    V fb[9], gb[5], tb_prev;
    ParamAdj<V> pa;
    collide_adj<V>(p, f, g, tau_prev, k, fo, go, tb_new, fb, gb, tb_prev, pa);
    // P^T: the pulled f_i(x) came from slot i of x - e_i, or slot opp(i) of x
    const bool xl = x > 0, xr = x < p.nx - 1, yb = y > 0, yt = y < p.ny - 1;
    lam_in[0 * P + k] = fb[0];
    if (xl) lam_in[1 * P + k - 1] = fb[1]; else lam_in[3 * P + k] = fb[1];
    if (yb) lam_in[2 * P + k - W] = fb[2]; else lam_in[4 * P + k] = fb[2];
    if (xr) lam_in[3 * P + k + 1] = fb[3]; else lam_in[1 * P + k] = fb[3];
    if (yt) lam_in[4 * P + k + W] = fb[4]; else lam_in[2 * P + k] = fb[4];
    if (xl && yb) lam_in[5 * P + k - W - 1] = fb[5]; else lam_in[7 * P + k] = fb[5];
    if (xr && yb) lam_in[6 * P + k - W + 1] = fb[6]; else lam_in[8 * P + k] = fb[6];
    if (xr && yt) lam_in[7 * P + k + W + 1] = fb[7]; else lam_in[5 * P + k] = fb[7];
    if (xl && yt) lam_in[8 * P + k + W - 1] = fb[8]; else lam_in[6 * P + k] = fb[8];
    V *G = lam_in + 9 * P;
    G[0 * P + k] = gb[0];
    if (xl) G[1 * P + k - 1] = gb[1]; else G[3 * P + k] = -gb[1];
    if (yb) G[2 * P + k - W] = gb[2]; else G[4 * P + k] = gb[2];
    if (xr) G[3 * P + k + 1] = gb[3]; else G[1 * P + k] = -gb[3];
    if (yt) G[4 * P + k + W] = gb[4]; else G[2 * P + k] = gb[4];
    lam_in[14 * P + k] = tb_prev;
    // parameters: porous coefficients of this node -> Da(x) (K = Da L^2, so
    // every coefficient scales as 1/Da or 1/sqrt(Da)), in the compute type
    const Porous<V> q = porous_at(p, k);
    const V iDa = p.da ? vrcp(load_da(p, k)) : ch.inv_Da;
    const V dDa = -iDa * (vfma(q.heK, pa.heK, q.eK * pa.eK) + V(0.5) * vfma(q.c1, pa.c1, q.eFsK * pa.eFsK));
    // nu_ref = Pr Ra^(-(2-n)/2) U_c L, n - 1, and 1/tauT with tauT - 1/2 ~ Ra^(-1/2)
    dn = vfma(pa.nu_ref, ch.a_nu, pa.nm1);
    dRa = vfma(pa.nu_ref, ch.b_nu, pa.omegaT * ch.b_wT);
    double *gd = gDa + (int64_t)y * p.nx + x;
    *gd = __ldcg(gd) + double(dDa);
    }
    const double sn = block128_sum(dn, sh), sR = block128_sum(dRa, sh);
    if (threadIdx.x == 0) {
        const int64_t b = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
        gnb[b] = __ldcg(gnb + b) + sn;
        gRab[b] = __ldcg(gRab + b) + sR;
    }
}

// Single-block FP64 sum of n values (fixed order).
__global__ void __launch_bounds__(256) sum_kernel(const double *__restrict__ a, int64_t n, double *out)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += a[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// dJ/dtau_0 summed over the nodes (the rest state's tau_0 depends on n, Ra).
template <class V>
__global__ void __launch_bounds__(256) tau0_sum_kernel(const V *__restrict__ lam, Phys<V> p, double *out)
{
    __shared__ double sh[256];
    double s = 0.0;
    const int64_t n = (int64_t)p.nx * p.ny;
    for (int64_t q = threadIdx.x; q < n; q += blockDim.x) {
        const int y = (int)(q / p.nx), x = (int)(q - (int64_t)y * p.nx);
        s += double(lam[14 * p.plane + (int64_t)y * p.pitch + x]);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

template <int PREC>
struct Adj {
    using St = Store<PREC>;
    using S = typename St::S;
    using TauS = typename St::TauS;
    using V = typename St::R;
};

template <int PREC>
int run_adjoint(lbm_ctx *c, int64_t steps, int ckpt, int from_rest, double *J, double *dDa, double *dn,
                double *dRa, double *peak_bytes)
{
    using A = Adj<PREC>;
    using S = typename A::S;
    using TauS = typename A::TauS;
    using V = typename A::V;
    const size_t es = sizeof(S), ts = sizeof(TauS);
    const size_t dist_bytes = es * 14 * (size_t)c->plane, tau_bytes = ts * (size_t)c->plane;
    const size_t lam_bytes = sizeof(V) * 15 * (size_t)c->plane;
    const int64_t nseg = (steps + ckpt - 1) / ckpt;
    const size_t nn = (size_t)c->nx * c->ny;
    std::vector<void *> allocs;
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();   // an allocation failure is reported by the return code
            return nullptr;
        }
        allocs.push_back(p);
        return p;
    };
    // second stream of the reverse sweep and its fork / join events
    cudaStream_t s2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    auto cleanup = [&]() {
        cudaStreamSynchronize(c->stream);
        if (s2) cudaStreamSynchronize(s2);
        for (void *p : allocs) cudaFree(p);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (s2) cudaStreamDestroy(s2);
    };
    int rc = LBM_OK;
    // checkpoints s_{j ckpt}, the states of one segment, two adjoint buffers, gradients
    char *ck = (char *)alloc((dist_bytes + tau_bytes) * (size_t)(nseg > 0 ? nseg : 1));
    const int seg_len = (int)(steps < ckpt ? steps : ckpt);
    const size_t seg_bytes = (dist_bytes + tau_bytes) * (size_t)(seg_len > 0 ? seg_len : 1);
    char *segs[2] = {(char *)alloc(seg_bytes), nullptr};
    V *lam[2] = {(V *)alloc(lam_bytes), (V *)alloc(lam_bytes)};
    const dim3 grid((c->nx + 127) / 128, c->ny);
    const size_t nblk = (size_t)grid.x * grid.y;
    double *g3 = (double *)alloc(sizeof(double) * (nn + 2 * nblk));   // dDa per node, dn / dRa per block
    double *red = (double *)alloc(sizeof(double) * 4);
    if (!ck || !segs[0] || !lam[0] || !lam[1] || !g3 || !red) {
        cleanup();
        return LBM_ERR_OOM;
    }
    // A second segment buffer and stream let the states of segment j - 1 be
    // recomputed while the reverse steps of segment j run (both are small,
    // latency-bound launches at the sizes the adjoint runs at, and share the
    // SMs).  Without them (one segment, or no memory or stream for them) the
    // two run one after the other on the context's stream.  The kernels and
    // their arguments are the same either way, so are the results.
    if (nseg > 1) {
        segs[1] = (char *)alloc(seg_bytes);
        if (segs[1] && (cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                        cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming) != cudaSuccess)) {
            cudaGetLastError();
            segs[1] = nullptr;
        }
    }
    const bool overlap = segs[1] != nullptr;
    // device memory of this run: the context's two state buffers plus the
    // checkpoints, one or two segments of states, two adjoint buffers and the
    // gradients
    const double total = (double)(dist_bytes + tau_bytes) * (double)(nseg + 2) +
                         (double)seg_bytes * (overlap ? 2.0 : 1.0) + 2.0 * lam_bytes +
                         sizeof(double) * (double)(nn + 2 * nblk);
    if (peak_bytes) *peak_bytes = total;
    if (from_rest) {
        c->cur = 0;
        if (lbm::launch_init(c) != cudaSuccess) rc = LBM_ERR_CUDA;
    }
    const Phys<V> pv = make_params<V>(c);
    auto ckd = [&](int64_t j) { return (S *)(ck + (size_t)j * (dist_bytes + tau_bytes)); };
    auto ckt = [&](int64_t j) { return (TauS *)(ck + (size_t)j * (dist_bytes + tau_bytes) + dist_bytes); };
    // state i of the segment held in buffer b
    auto sgd = [&](int b, int i) { return (S *)(segs[b] + (size_t)i * (dist_bytes + tau_bytes)); };
    auto sgt = [&](int b, int i) { return (TauS *)(segs[b] + (size_t)i * (dist_bytes + tau_bytes) + dist_bytes); };
    // forward with checkpoints (the context's own buffers advance to s_T),
    // through lbm_step, so small grids replay the context's step graphs
    // (same kernels and arguments as plain launches: identical states); it
    // also advances the context's step count
    for (int64_t j = 0; j < nseg && rc == LBM_OK; j++) {
        if (cudaMemcpyAsync(ckd(j), c->buf.dist[c->cur], dist_bytes, cudaMemcpyDeviceToDevice, c->stream) ||
            cudaMemcpyAsync(ckt(j), c->buf.tau[c->cur], tau_bytes, cudaMemcpyDeviceToDevice, c->stream)) {
            rc = LBM_ERR_CUDA;
            break;
        }
        const int64_t len = (j + 1) * ckpt <= steps ? ckpt : steps - j * ckpt;
        rc = lbm_step(c, len);
    }
    // J and the seed
    if (rc == LBM_OK && lbm::launch_nusselt(c) != cudaSuccess) rc = LBM_ERR_CUDA;
    double hj = 0.0;
    if (rc == LBM_OK && (cudaMemcpyAsync(&hj, c->d_small, sizeof(double), cudaMemcpyDeviceToHost, c->stream) ||
                         cudaStreamSynchronize(c->stream)))
        rc = LBM_ERR_CUDA;
    if (J) *J = hj;
    const double L = c->lat.L, dT = c->lat.T_hot - c->lat.T_cold;
    int cur = 0;
    if (rc == LBM_OK) {
        cudaMemsetAsync(lam[0], 0, lam_bytes, c->stream);
        cudaMemsetAsync(lam[1], 0, lam_bytes, c->stream);
        cudaMemsetAsync(g3, 0, sizeof(double) * (nn + 2 * nblk), c->stream);
        adj_seed_kernel<V><<<(c->ny + 127) / 128, 128, 0, c->stream>>>(lam[0], pv, -3.0 * L / (c->ny * dT),
                                                                       L / (3.0 * c->ny * dT));
        if (cudaGetLastError() != cudaSuccess) rc = LBM_ERR_CUDA;
    }
    // reverse sweep, one segment at a time, the last one first
    Chain chain{c->lat.n, 0.0, c->lat.tauT, 0.0, 0.0, 0.0, 0.0};
    {
        // Ra from the mapping: tauT - 1/2 = 3 U_c L / sqrt(Ra)
        const double Uc = c->opts.Ma / sqrt(3.0);
        const double r = 3.0 * Uc * L / (c->lat.tauT - 0.5);
        chain.Ra = r * r;
        const double nu_ref = c->lat.nu_ref, wT = 1.0 / c->lat.tauT;
        chain.a_nu = nu_ref * 0.5 * log(chain.Ra);
        chain.b_nu = -nu_ref * (2.0 - chain.n) / (2.0 * chain.Ra);
        chain.b_wT = wT * wT * (chain.tauT - 0.5) / (2.0 * chain.Ra);
        chain.inv_Da = c->lat.L * c->lat.L / c->lat.K;
    }
    const ChainV<V> chain_v{V(chain.a_nu), V(chain.b_nu), V(chain.b_wT), V(chain.inv_Da)};
    auto seg_len_of = [&](int64_t j) { return (j + 1) * ckpt <= steps ? ckpt : steps - j * ckpt; };
    auto buf_of = [&](int64_t j) { return overlap ? (int)(j & 1) : 0; };
    // Checkpoint j into slot 0 of its segment buffer (a plain copy on the
    // context's stream, never part of a graph: its source differs per
    // segment).
    auto copy_ckpt = [&](int64_t j) -> int {
        const int b = buf_of(j);
        if (cudaMemcpyAsync(sgd(b, 0), ckd(j), dist_bytes, cudaMemcpyDeviceToDevice, c->stream) ||
            cudaMemcpyAsync(sgt(b, 0), ckt(j), tau_bytes, cudaMemcpyDeviceToDevice, c->stream))
            return LBM_ERR_CUDA;
        return LBM_OK;
    };
    // The states s_{j ckpt + i}, i = 1..len-1, of segment j recomputed from
    // slot 0 on stream `s` (the context's step launcher, pointed at `s` for
    // these launches).
    auto recompute = [&](int64_t j, cudaStream_t s) -> int {
        const int b = buf_of(j), len = (int)seg_len_of(j);
        const cudaStream_t own = c->stream;
        c->stream = s;
        int r = LBM_OK;
        for (int i = 1; i < len && r == LBM_OK; i++)
            if (lbm::launch_step_buffers(c, sgd(b, i - 1), sgd(b, i), sgt(b, i - 1), sgt(b, i)) != cudaSuccess)
                r = LBM_ERR_CUDA;
        c->stream = own;
        return r;
    };
    // The reverse steps i = len-1..0 of segment j from adjoint buffer c0, on
    // the context's stream.
    auto reverse = [&](int64_t j, int c0) -> int {
        const int b = buf_of(j), len = (int)seg_len_of(j);
        int cc = c0;
        for (int i = len - 1; i >= 0; i--) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = grid;
            cfg.blockDim = dim3(128);
            cfg.stream = c->stream;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            auto launch = [&] {
                return cudaLaunchKernelEx(&cfg, adj_step_kernel<PREC, V>, (const S *)sgd(b, i),
                                          (const TauS *)sgt(b, i), (const V *)lam[cc], lam[cc ^ 1], g3, g3 + nn,
                                          g3 + nn + nblk, pv, chain_v);
            };
            cudaError_t e = launch();
            if (e != cudaSuccess) {   // a stream that refuses the attribute: an ordinary launch
                cudaGetLastError();
                cfg.numAttrs = 0;
                e = launch();
            }
            if (e != cudaSuccess) return LBM_ERR_CUDA;
            cc ^= 1;
        }
        return LBM_OK;
    };
    // Run `body` (launches on the context's stream, and on the second stream
    // forked from and joined back into it) through the cached graph `ex`:
    // captured at first use, replayed afterwards with the same kernels and
    // arguments, so the results are identical.  Pieces that are not
    // `cacheable`, or a stream that is already being captured, run plain.
    cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
    const bool can_capture = cudaStreamIsCapturing(c->stream, &cap_status) == cudaSuccess &&
                             cap_status == cudaStreamCaptureStatusNone && ckpt >= 2;
    std::vector<cudaGraphExec_t> execs;
    auto run = [&](cudaGraphExec_t &ex, bool cacheable, auto &&body) -> int {
        if (can_capture && cacheable) {
            if (!ex) {
                cudaGraph_t g = nullptr;
                if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                    const int rs = body();
                    const cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
                    if (rs == LBM_OK && ee == cudaSuccess && g && cudaGraphInstantiate(&ex, g, 0) == cudaSuccess)
                        execs.push_back(ex);
                    else
                        ex = nullptr;
                    if (g) cudaGraphDestroy(g);
                    cudaGetLastError();
                }
            }
            if (ex) return cudaGraphLaunch(ex, c->stream) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
        }
        return body();
    };
    // Stage j.  With two segment buffers: the reverse steps of segment j on
    // the context's stream and, beside them on the second stream, the
    // recomputation of segment j - 1 into the other buffer, whose last
    // reader (the reverse of segment j + 1) ended with the previous stage;
    // its checkpoint is copied in first.  With one buffer: the reverse steps,
    // then the copy and the recomputation, one after the other.  Only the
    // last segment can be shorter than ckpt, and it comes first; the stage of
    // segment 0, which runs once, is not captured.
    cudaGraphExec_t ex_both[2][2] = {}, ex_rev[2] = {}, ex_rec = nullptr;
    if (rc == LBM_OK && nseg > 0) {
        rc = copy_ckpt(nseg - 1);
        if (rc == LBM_OK) rc = recompute(nseg - 1, c->stream);
    }
    for (int64_t j = nseg - 1; j >= 0 && rc == LBM_OK; j--) {
        const int64_t len = seg_len_of(j);
        const bool full = len == ckpt;
        if (overlap) {
            if (j >= 1) rc = copy_ckpt(j - 1);
            if (rc == LBM_OK)
                rc = run(ex_both[buf_of(j)][cur], full && j >= 1, [&]() -> int {
                    if (cudaEventRecord(ev_fork, c->stream) || cudaStreamWaitEvent(s2, ev_fork, 0))
                        return LBM_ERR_CUDA;
                    if (int r = reverse(j, cur)) return r;
                    if (j >= 1)
                        if (int r = recompute(j - 1, s2)) return r;
                    if (cudaEventRecord(ev_join, s2) || cudaStreamWaitEvent(c->stream, ev_join, 0))
                        return LBM_ERR_CUDA;
                    return LBM_OK;
                });
        } else {
            rc = run(ex_rev[cur], full, [&]() -> int { return reverse(j, cur); });
            if (rc == LBM_OK && j >= 1) rc = copy_ckpt(j - 1);
            if (rc == LBM_OK && j >= 1)
                rc = run(ex_rec, seg_len_of(j - 1) == ckpt, [&]() -> int { return recompute(j - 1, c->stream); });
        }
        if (len & 1) cur ^= 1;
    }
    for (cudaGraphExec_t e : execs) cudaGraphExecDestroy(e);
    // reductions: sum of the n and Ra partials, and lambda_0 on tau for tau_0(n, Ra)
    double h[3] = {0, 0, 0};
    if (rc == LBM_OK) {
        sum_kernel<<<1, 256, 0, c->stream>>>(g3 + nn, (int64_t)nblk, red);
        sum_kernel<<<1, 256, 0, c->stream>>>(g3 + nn + nblk, (int64_t)nblk, red + 1);
        tau0_sum_kernel<V><<<1, 256, 0, c->stream>>>(lam[cur], pv, red + 2);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(h, red, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream) ||
            (dDa && cudaMemcpyAsync(dDa, g3, sizeof(double) * nn, cudaMemcpyDeviceToHost, c->stream)) ||
            cudaStreamSynchronize(c->stream))
            rc = LBM_ERR_CUDA;
    }
    if (rc == LBM_OK) {
        double gn = h[0], gR = h[1];
        if (from_rest) {
            // tau_0 = 3 nu_ref D(0) + 1/2, nu_ref ~ Ra^(-(2-n)/2), D(0) = 1 (literal) or gamma1^(n-1)
            const double nu_ref = c->lat.nu_ref, n = c->lat.n;
            const double D0 = c->lat.clamp_mode == 0 ? 1.0 : pow(c->lat.gamma1, n - 1.0);
            double dtau_dn = 3.0 * D0 * nu_ref * 0.5 * log(chain.Ra);
            if (c->lat.clamp_mode == 1) dtau_dn += 3.0 * nu_ref * D0 * log(c->lat.gamma1);
            const double dtau_dRa = 3.0 * D0 * (-nu_ref * (2.0 - n) / (2.0 * chain.Ra));
            gn += h[2] * dtau_dn;
            gR += h[2] * dtau_dRa;
        }
        if (dn) *dn = gn;
        if (dRa) *dRa = gR;
        c->have_snap = false;
    }
    cleanup();
    return rc;
}

}  // namespace

extern "C" int lbm_adjoint_nu(lbm_ctx *c, int64_t steps, int ckpt_every, int from_rest, double *J, double *dDa,
                              double *dn, double *dRa, double *peak_bytes)
{
    LBM_TRACE("lbm_adjoint_nu");
    if (!c || steps < 1 || ckpt_every < 1) return LBM_ERR_ARG;
    if (c->opts.layout != 0 || c->opts.tau_iters != 0) return LBM_ERR_UNSUPPORTED;
    if (c->row_lo != 0 || c->row_hi != c->ny) return LBM_ERR_UNSUPPORTED;   // whole cavities only
    if (cudaSetDevice(c->device) != cudaSuccess) return LBM_ERR_CUDA;
    switch (c->opts.prec) {
    case LBM_F64: return run_adjoint<LBM_F64>(c, steps, ckpt_every, from_rest, J, dDa, dn, dRa, peak_bytes);
    case LBM_F32: return run_adjoint<LBM_F32>(c, steps, ckpt_every, from_rest, J, dDa, dn, dRa, peak_bytes);
    case LBM_F32D: return run_adjoint<LBM_F32D>(c, steps, ckpt_every, from_rest, J, dDa, dn, dRa, peak_bytes);
    default: return LBM_ERR_UNSUPPORTED;
    }
}
