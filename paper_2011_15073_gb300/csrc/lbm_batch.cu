// lbm_batch.cu -- many independent cavities (a parameter sweep) as one
// workload: every time step is one launch over a flat list of row tiles of
// all active cases; convergence is checked per case on the device every
// resid_interval steps, and converged cases drop out of the tile work.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_step.cuh"

namespace {

using namespace lbm;

// What the batched kernel needs of one case (device memory).
struct CaseDev {
    void *dist[2];
    void *tau[2];
    Phys<double> pd;
    Phys<float> pf;
    Phys<F2> p2;
    int tiles_per_row;
    int tile0;  // first tile of this case in the flat tile list
    int cur;    // buffer holding the case's current state
    int pad;
};

// Per-case convergence state kept on the device.
struct Conv {
    double best, resid;
    long long steps;
    int since, active, reason, pad;
};

// TAU as for step_node: 0 lagged tau (stored per node), 1 node-local
// implicit tau (every case of a batch shares lbm_opts.tau_iters).
template <int PREC, int TAU>
__global__ void __launch_bounds__(256)
batch_step_kernel(const CaseDev *__restrict__ cases, int ncases, const int *__restrict__ active, int parity)
{
    using St = Store<PREC>;
    const int t = blockIdx.x;
    int lo = 0, hi = ncases - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cases[mid].tile0 <= t) lo = mid; else hi = mid - 1;
    }
    if (!active[lo]) return;
    const CaseDev &cd = cases[lo];
    const int local = t - cd.tile0;
    const int y = local / cd.tiles_per_row, xb = local - y * cd.tiles_per_row;
    const int s = cd.cur ^ parity;
    const auto *src = (const typename St::S *)cd.dist[s];
    auto *dst = (typename St::S *)cd.dist[s ^ 1];
    if constexpr (PREC == LBM_F64) {
        const int x = xb * blockDim.x + threadIdx.x;
        if (x < cd.pd.nx)
            step_node<PREC, double, 2, TAU>(src, dst, (const double *)cd.tau[s], (double *)cd.tau[s ^ 1], cd.pd,
                                            x, y);
    } else {
        step2_tile<PREC, 2, TAU>(src, dst, (const float *)cd.tau[s], (float *)cd.tau[s ^ 1], cd.pf, cd.p2,
                                 xb * 2 * (int)blockDim.x, y);
    }
}

// After each chunk: read every active case's residual (written by its
// residual kernels), retire it on tol / stagnation / max_steps / non-finite,
// and decide whether another chunk runs.  The chunk counter falls by one
// per call, so the device loop below ends after at most the number of chunks
// the host allowed, whatever the residuals do.
__global__ void __launch_bounds__(256)
batch_update_kernel(Conv *conv, int *active, double *const *smalls, int n, int delta, double tol,
                    double stag_floor, long long max_steps, int *chunks_left, int *go_out,
                    cudaGraphConditionalHandle handle, int set_condition)
{
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        Conv cv = conv[c];
        if (!cv.active) continue;
        const double *sm = smalls[c];
        const double r = fmax(sm[2], fmax(sm[3], sm[4]));
        cv.steps += delta;
        cv.resid = r;
        if (sm[5] > 0.0) {
            cv.active = 0;
            cv.reason = 3;
        } else if (r < tol) {
            cv.active = 0;
            cv.reason = 0;
        } else {
            if (r < cv.best) {
                cv.best = r;
                cv.since = 0;
            } else if (++cv.since >= 10 && r < stag_floor) {
                cv.active = 0;
                cv.reason = 1;
            }
            if (cv.active && cv.steps >= max_steps) {
                cv.active = 0;
                cv.reason = 2;
            }
        }
        conv[c] = cv;
        active[c] = cv.active;
        if (cv.active) atomicOr(&any, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int left = *chunks_left - 1;
        *chunks_left = left;
        const int go = (any && left > 0) ? 1 : 0;
        *go_out = go;
        if (set_condition) cudaGraphSetConditional(handle, (unsigned)go);
    }
}

}  // namespace

struct lbm_batch {
    std::vector<lbm_ctx *> sub;
    lbm_opts opts{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int threads = 128;        // block size of the batched kernel (tile = 2x nodes, or 1x in FP64)
    int ntiles = 0;
    std::vector<CaseDev> host_cases;
    CaseDev *d_cases = nullptr;
    int *d_active = nullptr;
    Conv *d_conv = nullptr;
    double **d_smalls = nullptr;
    int *d_chunks = nullptr;
    int *d_go = nullptr;
    int *h_go = nullptr;       // pinned
};

static thread_local char g_batch_err[256] = "";
#define BK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            snprintf(g_batch_err, sizeof(g_batch_err), "%s: %s", #call, cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;               \
        }                                                                                     \
    } while (0)

namespace {

int upload_cases(lbm_batch *b)
{
    const int tile = b->opts.prec == LBM_F64 ? b->threads : 2 * b->threads;
    int t0 = 0;
    for (size_t i = 0; i < b->sub.size(); i++) {
        lbm_ctx *c = b->sub[i];
        CaseDev &d = b->host_cases[i];
        d.dist[0] = c->buf.dist[0];
        d.dist[1] = c->buf.dist[1];
        d.tau[0] = c->buf.tau[0];
        d.tau[1] = c->buf.tau[1];
        d.pd = make_params<double>(c);
        d.pf = make_params<float>(c);
        d.p2 = make_params<F2>(c);
        d.tiles_per_row = (c->nx + tile - 1) / tile;
        d.tile0 = t0;
        d.cur = c->cur;
        t0 += d.tiles_per_row * c->ny;
    }
    b->ntiles = t0;
    BK(cudaMemcpyAsync(b->d_cases, b->host_cases.data(), sizeof(CaseDev) * b->sub.size(), cudaMemcpyHostToDevice,
                       b->stream));
    return LBM_OK;
}

template <int TAU>
cudaError_t launch_batch_step_tau(lbm_batch *b, int parity)
{
    const int n = (int)b->sub.size();
    switch (b->opts.prec) {
    case LBM_F64: batch_step_kernel<LBM_F64, TAU><<<b->ntiles, b->threads, 0, b->stream>>>(b->d_cases, n, b->d_active, parity); break;
    case LBM_F32: batch_step_kernel<LBM_F32, TAU><<<b->ntiles, b->threads, 0, b->stream>>>(b->d_cases, n, b->d_active, parity); break;
    case LBM_BF16D: batch_step_kernel<LBM_BF16D, TAU><<<b->ntiles, b->threads, 0, b->stream>>>(b->d_cases, n, b->d_active, parity); break;
    case LBM_F16D: batch_step_kernel<LBM_F16D, TAU><<<b->ntiles, b->threads, 0, b->stream>>>(b->d_cases, n, b->d_active, parity); break;
    default: batch_step_kernel<LBM_F32D, TAU><<<b->ntiles, b->threads, 0, b->stream>>>(b->d_cases, n, b->d_active, parity); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_step(lbm_batch *b, int parity)
{
    return b->opts.tau_iters > 0 ? launch_batch_step_tau<1>(b, parity) : launch_batch_step_tau<0>(b, parity);
}

double default_floor(const lbm_opts &o)
{
    if (o.stag_floor >= 0) return o.stag_floor;
    return o.prec == LBM_F64 ? 0.0 : ((o.prec == LBM_F32 || o.prec == LBM_F32D) ? 1e-6 : (o.prec == LBM_F16D ? 1e-2 : 1e-1));
}

// Enqueue one chunk: `delta` steps of every active case, their residuals and
// the convergence update.
int enqueue_chunk(lbm_batch *b, double tol, long long max_steps, cudaGraphConditionalHandle h, int set_cond)
{
    const int delta = b->opts.resid_interval;
    for (int s = 0; s < delta; s++) BK(launch_batch_step(b, s & 1));
    for (lbm_ctx *c : b->sub) BK(lbm::launch_residual(c, false));
    batch_update_kernel<<<1, 256, 0, b->stream>>>(b->d_conv, b->d_active, b->d_smalls, (int)b->sub.size(), delta,
                                                  tol, default_floor(b->opts), max_steps, b->d_chunks, b->d_go, h,
                                                  set_cond);
    BK(cudaGetLastError());
    return LBM_OK;
}

void free_batch(lbm_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (lbm_ctx *c : b->sub) lbm_destroy(c);
    cudaFree(b->d_cases);
    cudaFree(b->d_active);
    cudaFree(b->d_conv);
    cudaFree(b->d_smalls);
    cudaFree(b->d_chunks);
    cudaFree(b->d_go);
    cudaFreeHost(b->h_go);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int set_all_active(lbm_batch *b, int v)
{
    std::vector<int> a(b->sub.size(), v);
    BK(cudaMemcpyAsync(b->d_active, a.data(), sizeof(int) * a.size(), cudaMemcpyHostToDevice, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(lbm_batch **out, const lbm_case *cases, int ncases, const lbm_opts *opts)
{
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (!cases || ncases < 1) return LBM_ERR_ARG;
    lbm_opts o;
    if (opts) o = *opts; else lbm_default_opts(&o);
    // the batched sweep replays a CUDA graph, which would replay the
    // stochastic rounding's seed too: those storages are not built here
    if (o.layout != 0 || o.prec == LBM_F16S || o.prec == LBM_BF16S) return LBM_ERR_UNSUPPORTED;
    if (o.resid_interval < 2 || (o.resid_interval & 1)) return LBM_ERR_ARG;
    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_OOM;
    b->opts = o;
    int rc = LBM_OK;
    if (o.device >= 0) {
        if (cudaSetDevice(o.device) != cudaSuccess) { delete b; return LBM_ERR_CUDA; }
        b->device = o.device;
    } else if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return LBM_ERR_CUDA;
    }
    if (o.cuda_stream) {
        b->stream = (cudaStream_t)o.cuda_stream;
    } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        return LBM_ERR_CUDA;
    } else {
        b->own_stream = true;
    }
    lbm_opts so = o;
    so.cuda_stream = b->stream;
    so.device = b->device;
    for (int i = 0; i < ncases && rc == LBM_OK; i++) {
        lbm_ctx *c = nullptr;
        rc = lbm_init(&c, cases[i].nx, cases[i].ny, cases[i].n, cases[i].Da, cases[i].Ra, cases[i].Pr,
                      cases[i].porosity, &so);
        if (rc == LBM_OK) b->sub.push_back(c);
    }
    if (rc == LBM_OK) {
        auto alloc = [&]() -> int {
            const size_t n = b->sub.size();
            BK(cudaMalloc(&b->d_cases, sizeof(CaseDev) * n));
            BK(cudaMalloc(&b->d_active, sizeof(int) * n));
            BK(cudaMalloc(&b->d_conv, sizeof(Conv) * n));
            BK(cudaMalloc(&b->d_smalls, sizeof(double *) * n));
            BK(cudaMalloc(&b->d_chunks, sizeof(int)));
            BK(cudaMalloc(&b->d_go, sizeof(int)));
            BK(cudaMallocHost(&b->h_go, sizeof(int)));
            std::vector<double *> sm(n);
            for (size_t i = 0; i < n; i++) sm[i] = b->sub[i]->d_small;
            BK(cudaMemcpy(b->d_smalls, sm.data(), sizeof(double *) * n, cudaMemcpyHostToDevice));
            b->host_cases.resize(n);
            return LBM_OK;
        };
        rc = alloc();
    }
    if (rc == LBM_OK) rc = upload_cases(b);
    if (rc == LBM_OK) rc = set_all_active(b, 1);
    if (rc != LBM_OK) {
        free_batch(b);
        return rc;
    }
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b) { free_batch(b); }

int lbm_batch_get_case(lbm_batch *b, int i, lbm_ctx **ctx)
{
    if (!b || !ctx || i < 0 || i >= (int)b->sub.size()) return LBM_ERR_ARG;
    *ctx = b->sub[i];
    return LBM_OK;
}

int lbm_batch_step(lbm_batch *b, int64_t k)
{
    if (!b || k < 0) return LBM_ERR_ARG;
    BK(cudaSetDevice(b->device));
    int rc = upload_cases(b);   // current buffers of every case
    if (rc) return rc;
    rc = set_all_active(b, 1);
    if (rc) return rc;
    for (int64_t s = 0; s < k; s++) BK(launch_batch_step(b, (int)(s & 1)));
    if (k & 1)
        for (lbm_ctx *c : b->sub) c->cur ^= 1;
    for (lbm_ctx *c : b->sub) c->steps += k;
    return LBM_OK;
}

int lbm_batch_run_to_steady(lbm_batch *b, double tol, int64_t max_steps, int graph_mode, int64_t *steps,
                            double *resid, int *reason)
{
    if (!b || max_steps < 0 || !(tol >= 0) || (graph_mode != 0 && graph_mode != 1)) return LBM_ERR_ARG;
    BK(cudaSetDevice(b->device));
    const int n = (int)b->sub.size();
    const int delta = b->opts.resid_interval;
    int rc = upload_cases(b);
    if (rc) return rc;
    // first residual of every case stores its snapshot
    for (lbm_ctx *c : b->sub) {
        if (!c->d_snap) BK(cudaMalloc(&c->d_snap, sizeof(double) * 3 * (size_t)c->nx * c->ny));
        BK(lbm::launch_residual(c, true));
        c->have_snap = true;
    }
    std::vector<Conv> conv(n);
    for (auto &cv : conv) {
        cv.best = INFINITY;
        cv.resid = INFINITY;
        cv.steps = 0;
        cv.since = 0;
        cv.active = max_steps > 0 ? 1 : 0;
        cv.reason = 2;
        cv.pad = 0;
    }
    BK(cudaMemcpyAsync(b->d_conv, conv.data(), sizeof(Conv) * n, cudaMemcpyHostToDevice, b->stream));
    rc = set_all_active(b, max_steps > 0 ? 1 : 0);
    if (rc) return rc;
    const long long chunks = (long long)((max_steps + delta - 1) / delta);
    const int chunks_i = chunks > 0x7fffffff ? 0x7fffffff : (int)chunks;
    BK(cudaMemcpyAsync(b->d_chunks, &chunks_i, sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BK(cudaStreamSynchronize(b->stream));

    if (chunks_i > 0) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        BK(cudaGraphCreate(&graph, 0));
        int rc2 = LBM_OK;
        if (graph_mode == 0) {
            // one graph = one chunk; the host relaunches it while cases remain
            BK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            rc2 = enqueue_chunk(b, tol, max_steps, 0, 0);
            cudaGraph_t captured = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(b->stream, &captured);
            cudaGraphDestroy(graph);
            graph = captured;
            if (rc2 == LBM_OK && ec != cudaSuccess) rc2 = LBM_ERR_CUDA;
        } else {
            // one graph launch for the whole run: a device-side while loop
            cudaGraphConditionalHandle handle;
            BK(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
            cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
            cp.conditional.handle = handle;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t node;
            BK(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            BK(cudaStreamBeginCaptureToGraph(b->stream, body, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
            rc2 = enqueue_chunk(b, tol, max_steps, handle, 1);
            cudaGraph_t captured = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(b->stream, &captured);
            if (rc2 == LBM_OK && ec != cudaSuccess) rc2 = LBM_ERR_CUDA;
        }
        if (rc2 == LBM_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rc2 = LBM_ERR_CUDA;
        if (rc2 == LBM_OK) {
            if (graph_mode == 0) {
                for (;;) {
                    if (cudaGraphLaunch(exec, b->stream) != cudaSuccess) { rc2 = LBM_ERR_CUDA; break; }
                    if (cudaMemcpyAsync(b->h_go, b->d_go, sizeof(int), cudaMemcpyDeviceToHost, b->stream) !=
                            cudaSuccess ||
                        cudaStreamSynchronize(b->stream) != cudaSuccess) {
                        rc2 = LBM_ERR_CUDA;
                        break;
                    }
                    if (!*b->h_go) break;
                }
            } else if (cudaGraphLaunch(exec, b->stream) != cudaSuccess ||
                       cudaStreamSynchronize(b->stream) != cudaSuccess) {
                rc2 = LBM_ERR_CUDA;
            }
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (rc2 != LBM_OK) {
            snprintf(g_batch_err, sizeof(g_batch_err), "batch graph: %s", cudaGetErrorString(cudaGetLastError()));
            return rc2;
        }
    }
    BK(cudaMemcpyAsync(conv.data(), b->d_conv, sizeof(Conv) * n, cudaMemcpyDeviceToHost, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    int out_rc = LBM_OK;
    for (int i = 0; i < n; i++) {
        b->sub[i]->steps += conv[i].steps;
        if (steps) steps[i] = conv[i].steps;
        if (resid) resid[i] = conv[i].resid;
        if (reason) reason[i] = conv[i].reason;
        if (conv[i].reason == 3) out_rc = LBM_ERR_NONFINITE;
    }
    return out_rc;
}

int lbm_batch_nusselt(lbm_batch *b, double *hot, double *cold)
{
    if (!b) return LBM_ERR_ARG;
    for (size_t i = 0; i < b->sub.size(); i++) {
        int rc = lbm_nusselt(b->sub[i], hot ? hot + i : nullptr, cold ? cold + i : nullptr, nullptr);
        if (rc) return rc;
    }
    return LBM_OK;
}

int lbm_batch_tune(lbm_batch *b, int steps, int *threads_out)
{
    if (!b || steps < 2) return LBM_ERR_ARG;
    BK(cudaSetDevice(b->device));
    steps &= ~1;  // even: every case ends in the buffer it started in
    // keep the states: time on copies, restore afterwards
    std::vector<void *> save_d(b->sub.size(), nullptr), save_t(b->sub.size(), nullptr);
    int rc = LBM_OK;
    for (size_t i = 0; i < b->sub.size() && rc == LBM_OK; i++) {
        lbm_ctx *c = b->sub[i];
        const size_t db = c->dist_elem * 14 * (size_t)c->plane, tb = c->tau_elem * (size_t)c->plane;
        if (cudaMalloc(&save_d[i], db) != cudaSuccess || cudaMalloc(&save_t[i], tb) != cudaSuccess ||
            cudaMemcpyAsync(save_d[i], c->buf.dist[c->cur], db, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess ||
            cudaMemcpyAsync(save_t[i], c->buf.tau[c->cur], tb, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
            rc = LBM_ERR_CUDA;
    }
    const int cand[3] = {64, 128, 256};
    float best_ms = 1e30f;
    int best = b->threads;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == LBM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = LBM_ERR_CUDA;
    if (rc == LBM_OK) rc = set_all_active(b, 1);
    for (int ci = 0; ci < 3 && rc == LBM_OK; ci++) {
        b->threads = cand[ci];
        rc = upload_cases(b);
        if (rc) break;
        for (int s = 0; s < 2 && rc == LBM_OK; s++)
            if (launch_batch_step(b, s & 1) != cudaSuccess) rc = LBM_ERR_CUDA;   // warm-up
        cudaEventRecord(e0, b->stream);
        for (int s = 0; s < steps && rc == LBM_OK; s++)
            if (launch_batch_step(b, s & 1) != cudaSuccess) rc = LBM_ERR_CUDA;
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = LBM_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rc == LBM_OK && ms < best_ms) {
            best_ms = ms;
            best = cand[ci];
        }
    }
    for (size_t i = 0; i < b->sub.size(); i++) {
        lbm_ctx *c = b->sub[i];
        if (save_d[i] && rc == LBM_OK) {
            cudaMemcpyAsync(c->buf.dist[c->cur], save_d[i], c->dist_elem * 14 * (size_t)c->plane,
                            cudaMemcpyDeviceToDevice, b->stream);
            cudaMemcpyAsync(c->buf.tau[c->cur], save_t[i], c->tau_elem * (size_t)c->plane, cudaMemcpyDeviceToDevice,
                            b->stream);
        }
    }
    cudaStreamSynchronize(b->stream);
    for (size_t i = 0; i < b->sub.size(); i++) {
        cudaFree(save_d[i]);
        cudaFree(save_t[i]);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    b->threads = best;
    if (rc == LBM_OK) rc = upload_cases(b);
    if (threads_out) *threads_out = best;
    return rc;
}

}  // extern "C"
