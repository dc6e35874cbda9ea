// lbm_batch.cu -- many independent cavities (a parameter sweep) as one
// workload.  The row tiles of all active cases form one flat list, compacted
// on the device whenever cases retire; a fixed grid (a tuned multiple of the
// SM count) strides over it.  Two execution modes:
//   per-step: one launch per time step (resid_interval launches per chunk);
//   persistent: one cooperative launch per chunk that runs all its steps,
//     with a grid barrier between steps (every wait bounded: a block that
//     gives up raises the batch's error word and every block leaves).
// Convergence is checked per case on the device every resid_interval steps,
// and converged cases drop out of the tile list.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_trace.h"
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
    int ntiles;  // tiles_per_row * ny
    int cur;     // buffer holding the case's current state
    uint32_t run;              // stochastic rounding: the run's stream word (run_word)
    long long step0;           // the case's step count when the batch call began
};

// Per-case convergence state kept on the device.
struct Conv {
    double best, resid;
    long long steps;
    int since, active, reason, pad;
};

// The compacted list of active cases: idx[0..m) the active cases in order,
// t0[j] the first flat tile of idx[j] (t0[m] = total), hdr = {m, total}.
struct ActiveList {
    int *idx;
    int *t0;
    int *hdr;
};

// Grid barrier of the persistent kernel: arrival count and generation.
struct GridBarrier {
    unsigned count, gen;
};

// Rebuild the active list from the per-case flags (one thread; runs once per
// chunk).
__device__ void build_active(const CaseDev *cases, const int *active, int n, ActiveList a)
{
    int m = 0, t = 0;
    for (int c = 0; c < n; c++) {
        if (!active[c]) continue;
        a.idx[m] = c;
        a.t0[m] = t;
        t += cases[c].ntiles;
        m++;
    }
    a.t0[m] = t;
    a.hdr[0] = m;
    a.hdr[1] = t;
}

__global__ void build_active_kernel(const CaseDev *cases, const int *active, int n, ActiveList a)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) build_active(cases, active, n, a);
}

// Where a step of the sweep stands in each case's own step count: step s of
// the current launch or chunk, `off` steps into the batch call, plus (in a
// run to steady state, whose chunks replay one graph) the steps the case's
// convergence record has counted so far.
struct StepAt {
    const Conv *conv;   // nullptr outside run_to_steady
    long long off;
    int s;
};

// One row tile of one case: the same tile bodies as the single-cavity
// kernels (two nodes per thread, or one node per thread in FP64), so every
// case evolves bit for bit as it would alone -- the stochastic-rounding
// storages too, whose seed is computed here from the case's step count as a
// plain launch computes it on the host.  TAU as for step_node; FIELD 0 when
// no case has a per-node Darcy field, else 2 (decided per case).
template <int PREC, int TAU, int FIELD>
__device__ __forceinline__ void batch_tile(const CaseDev &cd, int c, int local, StepAt at)
{
    using St = Store<PREC>;
    const int y = local / cd.tiles_per_row, xb = local - y * cd.tiles_per_row;
    const int s = cd.cur ^ (at.s & 1);
    const auto *src = (const typename St::S *)cd.dist[s];
    auto *dst = (typename St::S *)cd.dist[s ^ 1];
    uint32_t seed = 0;
    if constexpr (rounds_stochastically(PREC)) {
        const long long done = at.conv ? at.conv[c].steps : 0;
        seed = step_seed((uint64_t)(cd.step0 + done + at.off + at.s), cd.run);
    }
    if constexpr (PREC == LBM_F64) {
        const int x = xb * blockDim.x + threadIdx.x;
        if (x < cd.pd.nx)
            step_node<PREC, double, FIELD, TAU>(src, dst, (const double *)cd.tau[s], (double *)cd.tau[s ^ 1],
                                                cd.pd, x, y, seed);
    } else {
        step2_tile<PREC, FIELD, TAU>(src, dst, (const float *)cd.tau[s], (float *)cd.tau[s ^ 1], cd.pf, cd.p2,
                                 xb * 2 * (int)blockDim.x, y, seed);
    }
}

// Every tile of the active list once, striding by the grid.
template <int PREC, int TAU, int FIELD>
__device__ __forceinline__ void batch_sweep(const CaseDev *__restrict__ cases, ActiveList a, int m, int nt,
                                            StepAt at)
{
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        int lo = 0, hi = m - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.t0[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const int c = a.idx[lo];
        batch_tile<PREC, TAU, FIELD>(cases[c], c, t - a.t0[lo], at);
    }
}

template <int PREC, int TAU, int FIELD>
__global__ void __launch_bounds__(256)
batch_step_kernel(const CaseDev *__restrict__ cases, ActiveList a, StepAt at)
{
    batch_sweep<PREC, TAU, FIELD>(cases, a, a.hdr[0], a.hdr[1], at);
}

// Bounded grid barrier.  Thread 0 of each block arrives on the counter; the
// last one resets it and advances the generation, the others poll the
// generation for at most `budget` clock cycles.  A block that gives up sets
// *err; a block that sees *err set after the barrier leaves too, so no block
// waits on one that has gone.  The fences order each block's stores of the
// finished step before any block's loads of the next.
__device__ __forceinline__ bool grid_sync(GridBarrier *bar, long long budget, int *err)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *genp = &bar->gen;
        const unsigned g = *genp;
        __threadfence();
        if (atomicAdd(&bar->count, 1u) == gridDim.x - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*genp == g) {
                if (clock64() - t0 > budget) {
                    atomicExch(err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        if (ok && *(volatile int *)err) ok = 0;
    }
    __syncthreads();
    return ok != 0;
}

// Persistent form: `steps` time steps in one cooperative launch (all blocks
// resident), a grid barrier between consecutive steps.
template <int PREC, int TAU, int FIELD>
__global__ void __launch_bounds__(256)
batch_chunk_kernel(const CaseDev *__restrict__ cases, ActiveList a, StepAt at, int steps, GridBarrier *bar,
                   long long budget, int *err)
{
    if (*(volatile int *)err) return;
    const int m = a.hdr[0], nt = a.hdr[1];
    for (int s = 0; s < steps; s++) {
        at.s = s;
        batch_sweep<PREC, TAU, FIELD>(cases, a, m, nt, at);
        if (s + 1 < steps && !grid_sync(bar, budget, err)) return;
    }
}

// After each chunk: read every active case's residual (written by its
// residual kernels), retire it on tol / stagnation / max_steps / non-finite,
// rebuild the active tile list, and decide whether another chunk runs.  The
// chunk counter falls by one per call, so the device loop below ends after
// at most the number of chunks the host allowed, whatever the residuals do;
// a raised error word (a persistent launch gave up a barrier) ends it too.
__global__ void __launch_bounds__(256)
batch_update_kernel(Conv *conv, int *active, double *const *smalls, int n, int delta, double tol,
                    double stag_floor, long long max_steps, int *chunks_left, int *go_out,
                    const CaseDev *cases, ActiveList a, const int *err,
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
        build_active(cases, active, n, a);
        const int left = *chunks_left - 1;
        *chunks_left = left;
        const int go = (any && left > 0 && !*err) ? 1 : 0;
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
    int sms = 0;
    // execution plan (lbm_batch_tune / lbm_batch_set_plan): block size (tile
    // = 2x nodes, or 1x in FP64), grid = blocks_per_sm x SMs, and the mode
    int threads = 128;
    int blocks_per_sm = 8;
    int mode = LBM_BATCH_PER_STEP;
    long long budget = 1ll << 31;   // clock cycles a persistent block waits at a barrier
    int ntiles = 0;
    bool any_field = false;   // some case has a per-node Darcy field
    std::vector<CaseDev> host_cases;
    CaseDev *d_cases = nullptr;
    int *d_active = nullptr;
    ActiveList act{nullptr, nullptr, nullptr};
    Conv *d_conv = nullptr;
    double **d_smalls = nullptr;
    int *d_chunks = nullptr;
    int *d_go = nullptr;
    int *h_go = nullptr;       // pinned
    GridBarrier *d_bar = nullptr;
    int *d_err = nullptr;      // raised by a persistent block that gave up a barrier (sticky)
    int *h_err = nullptr;      // pinned
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

int tile_nodes(const lbm_batch *b) { return b->opts.prec == LBM_F64 ? b->threads : 2 * b->threads; }

int upload_cases(lbm_batch *b)
{
    const int tile = tile_nodes(b);
    int t0 = 0;
    b->any_field = false;
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
        d.ntiles = d.tiles_per_row * c->ny;
        d.cur = c->cur;
        d.run = run_word(c->opts.seed);
        d.step0 = c->steps;
        if (c->d_da) b->any_field = true;
        t0 += d.ntiles;
    }
    b->ntiles = t0;
    BK(cudaMemcpyAsync(b->d_cases, b->host_cases.data(), sizeof(CaseDev) * b->sub.size(), cudaMemcpyHostToDevice,
                       b->stream));
    build_active_kernel<<<1, 32, 0, b->stream>>>(b->d_cases, b->d_active, (int)b->sub.size(), b->act);
    BK(cudaGetLastError());
    return LBM_OK;
}

// The step and persistent kernels of the batch's storage, tau scheme and
// Darcy-field mode.
template <int PREC>
void *kernel_of(const lbm_batch *b, bool persistent)
{
    const int t = b->opts.tau_iters > 0 ? 1 : 0, f = b->any_field ? 2 : 0;
    if (persistent) {
        if (t) return f ? (void *)batch_chunk_kernel<PREC, 1, 2> : (void *)batch_chunk_kernel<PREC, 1, 0>;
        return f ? (void *)batch_chunk_kernel<PREC, 0, 2> : (void *)batch_chunk_kernel<PREC, 0, 0>;
    }
    if (t) return f ? (void *)batch_step_kernel<PREC, 1, 2> : (void *)batch_step_kernel<PREC, 1, 0>;
    return f ? (void *)batch_step_kernel<PREC, 0, 2> : (void *)batch_step_kernel<PREC, 0, 0>;
}

void *kernel_of(const lbm_batch *b, bool persistent)
{
    switch (b->opts.prec) {
    case LBM_F64: return kernel_of<LBM_F64>(b, persistent);
    case LBM_F32: return kernel_of<LBM_F32>(b, persistent);
    case LBM_BF16D: return kernel_of<LBM_BF16D>(b, persistent);
    case LBM_F16D: return kernel_of<LBM_F16D>(b, persistent);
    case LBM_F16S: return kernel_of<LBM_F16S>(b, persistent);
    case LBM_BF16S: return kernel_of<LBM_BF16S>(b, persistent);
    default: return kernel_of<LBM_F32D>(b, persistent);
    }
}

void *chunk_kernel(const lbm_batch *b) { return kernel_of(b, true); }

// Blocks of `threads` threads of the persistent kernel that fit on one SM
// (a cooperative launch needs every block resident).
int resident_blocks(const lbm_batch *b, int threads)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, chunk_kernel(b), threads, 0) != cudaSuccess) return 0;
    return nb;
}

int grid_blocks(const lbm_batch *b)
{
    int bps = b->blocks_per_sm;
    if (b->mode == LBM_BATCH_PERSISTENT) {
        const int r = resident_blocks(b, b->threads);
        if (bps > r) bps = r;
    }
    return (bps < 1 ? 1 : bps) * b->sms;
}

cudaError_t launch_batch_step(lbm_batch *b, StepAt at)
{
    const CaseDev *cases = b->d_cases;
    ActiveList a = b->act;
    void *args[] = {(void *)&cases, (void *)&a, (void *)&at};
    return cudaLaunchKernel(kernel_of(b, false), dim3(grid_blocks(b)), dim3(b->threads), args, 0, b->stream);
}

// `steps` steps of every active case, `off` steps into the batch call (and
// counted from the convergence records in a run to steady state): per-step
// launches, or one persistent cooperative launch (its barrier reset first).
cudaError_t launch_batch_steps(lbm_batch *b, int steps, long long off = 0, bool counted = false)
{
    if (steps <= 0) return cudaSuccess;
    StepAt at{counted ? b->d_conv : nullptr, off, 0};
    if (b->mode == LBM_BATCH_PER_STEP) {
        for (int s = 0; s < steps; s++) {
            at.s = s;
            const cudaError_t e = launch_batch_step(b, at);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    cudaError_t e = cudaMemsetAsync(b->d_bar, 0, sizeof(GridBarrier), b->stream);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid_blocks(b));
    cfg.blockDim = dim3(b->threads);
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const CaseDev *cases = b->d_cases;
    ActiveList a = b->act;
    GridBarrier *bar = b->d_bar;
    long long budget = b->budget;
    int *err = b->d_err;
    void *args[] = {(void *)&cases, (void *)&a, (void *)&at, (void *)&steps, (void *)&bar, (void *)&budget,
                    (void *)&err};
    return cudaLaunchKernelExC(&cfg, chunk_kernel(b), args);
}

double default_floor(const lbm_opts &o)
{
    if (o.stag_floor >= 0) return o.stag_floor;
    switch (o.prec) {   // as a single context's run_to_steady
    case LBM_F64: return 0.0;
    case LBM_F32:
    case LBM_F32D: return 1e-6;
    case LBM_F16D: return 1e-2;
    case LBM_F16S: return 1e-3;
    case LBM_BF16S: return 1e-2;
    default: return 1e-1;
    }
}

// Enqueue one chunk: `delta` steps of every active case, their residuals and
// the convergence update.
int enqueue_chunk(lbm_batch *b, double tol, long long max_steps, cudaGraphConditionalHandle h, int set_cond)
{
    const int delta = b->opts.resid_interval;
    BK(launch_batch_steps(b, delta, 0, true));
    for (lbm_ctx *c : b->sub) BK(lbm::launch_residual(c, false));
    batch_update_kernel<<<1, 256, 0, b->stream>>>(b->d_conv, b->d_active, b->d_smalls, (int)b->sub.size(), delta,
                                                  tol, default_floor(b->opts), max_steps, b->d_chunks, b->d_go,
                                                  b->d_cases, b->act, b->d_err, h, set_cond);
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
    cudaFree(b->act.idx);
    cudaFree(b->act.t0);
    cudaFree(b->act.hdr);
    cudaFree(b->d_conv);
    cudaFree(b->d_smalls);
    cudaFree(b->d_chunks);
    cudaFree(b->d_go);
    cudaFreeHost(b->h_go);
    cudaFree(b->d_bar);
    cudaFree(b->d_err);
    cudaFreeHost(b->h_err);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int set_all_active(lbm_batch *b, int v)
{
    std::vector<int> a(b->sub.size(), v);
    BK(cudaMemcpyAsync(b->d_active, a.data(), sizeof(int) * a.size(), cudaMemcpyHostToDevice, b->stream));
    build_active_kernel<<<1, 32, 0, b->stream>>>(b->d_cases, b->d_active, (int)b->sub.size(), b->act);
    BK(cudaGetLastError());
    BK(cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

// Read the error word: LBM_ERR_TIMEOUT once a persistent block gave up.
int batch_err(lbm_batch *b)
{
    BK(cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    return *b->h_err ? LBM_ERR_TIMEOUT : LBM_OK;
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
    if (o.layout != 0) return LBM_ERR_UNSUPPORTED;
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
            BK(cudaMemset(b->d_active, 0, sizeof(int) * n));
            BK(cudaMalloc(&b->act.idx, sizeof(int) * n));
            BK(cudaMalloc(&b->act.t0, sizeof(int) * (n + 1)));
            BK(cudaMalloc(&b->act.hdr, sizeof(int) * 2));
            BK(cudaMalloc(&b->d_bar, sizeof(GridBarrier)));
            BK(cudaMalloc(&b->d_err, sizeof(int)));
            BK(cudaMemset(b->d_err, 0, sizeof(int)));
            BK(cudaMallocHost(&b->h_err, sizeof(int)));
            *b->h_err = 0;
            BK(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device));
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
    LBM_TRACE("lbm_batch_step");
    if (!b || k < 0) return LBM_ERR_ARG;
    BK(cudaSetDevice(b->device));
    int rc = upload_cases(b);   // current buffers of every case
    if (rc) return rc;
    rc = set_all_active(b, 1);
    if (rc) return rc;
    if (int e = batch_err(b)) return e;
    // in pieces of an even number of steps (each case then ends a piece in
    // the buffer it started it in), then the odd remainder
    const int64_t piece = 1 << 20;
    for (int64_t done = 0; done < k;) {
        int64_t n = k - done < piece ? k - done : piece;
        if (n > 1) n &= ~int64_t(1);
        BK(launch_batch_steps(b, (int)n, done));
        if (n & 1) {
            for (lbm_ctx *c : b->sub) c->cur ^= 1;
            rc = upload_cases(b);
            if (rc) return rc;
        }
        done += n;
    }
    for (lbm_ctx *c : b->sub) c->steps += k;
    return b->mode == LBM_BATCH_PERSISTENT ? batch_err(b) : LBM_OK;
}

int lbm_batch_run_to_steady(lbm_batch *b, double tol, int64_t max_steps, int graph_mode, int64_t *steps,
                            double *resid, int *reason)
{
    LBM_TRACE("lbm_batch_run_to_steady");
    if (!b || max_steps < 0 || !(tol >= 0) || (graph_mode != 0 && graph_mode != 1)) return LBM_ERR_ARG;
    BK(cudaSetDevice(b->device));
    if (int e = batch_err(b)) return e;
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

    for (int attempt = 0; chunks_i > 0 && attempt < 2; attempt++) {
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
        const bool exec_launched = rc2 == LBM_OK;
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
        if (rc2 == LBM_OK) break;
        const cudaError_t last = cudaGetLastError();
        if (attempt == 0 && b->mode == LBM_BATCH_PERSISTENT && !exec_launched) {
            // the graph with the cooperative launch could not be built here:
            // the per-step form runs the same steps
            b->mode = LBM_BATCH_PER_STEP;
            continue;
        }
        snprintf(g_batch_err, sizeof(g_batch_err), "batch graph: %s", cudaGetErrorString(last));
        return rc2;
    }
    if (int e = batch_err(b)) return e;
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

int lbm_batch_set_plan(lbm_batch *b, int mode, int threads, int blocks_per_sm)
{
    if (!b || (mode != LBM_BATCH_PER_STEP && mode != LBM_BATCH_PERSISTENT) ||
        (threads != 64 && threads != 128 && threads != 256) || blocks_per_sm < 1 || blocks_per_sm > 64)
        return LBM_ERR_ARG;
    BK(cudaSetDevice(b->device));
    const int old_mode = b->mode, old_threads = b->threads;
    b->mode = mode;
    b->threads = threads;
    if (mode == LBM_BATCH_PERSISTENT && resident_blocks(b, threads) < 1) {
        b->mode = old_mode;
        b->threads = old_threads;
        return LBM_ERR_UNSUPPORTED;
    }
    b->blocks_per_sm = blocks_per_sm;
    return upload_cases(b);
}

int lbm_batch_get_plan(const lbm_batch *b, int *mode, int *threads, int *blocks_per_sm)
{
    if (!b) return LBM_ERR_ARG;
    if (mode) *mode = b->mode;
    if (threads) *threads = b->threads;
    if (blocks_per_sm) {
        int bps = b->blocks_per_sm;
        if (b->mode == LBM_BATCH_PERSISTENT) {
            const int r = resident_blocks(b, b->threads);
            if (bps > r) bps = r;
        }
        *blocks_per_sm = bps;
    }
    return LBM_OK;
}

int lbm_batch_set_wait_budget(lbm_batch *b, int64_t cycles)
{
    if (!b || cycles < 1) return LBM_ERR_ARG;
    b->budget = cycles;
    return LBM_OK;
}

int lbm_batch_tune(lbm_batch *b, int steps, int *threads_out)
{
    LBM_TRACE("lbm_batch_tune");
    if (!b || steps < 2) return LBM_ERR_ARG;
    BK(cudaSetDevice(b->device));
    if (int e = batch_err(b)) return e;
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
    // candidates: mode x block size x blocks per SM (the grid is a multiple
    // of the SM count; each block strides over the tiles, so the blocks per
    // SM set how many tiles -- and cases -- one block takes per step)
    struct Plan { int mode, threads, bps; };
    std::vector<Plan> cand;
    for (int mode : {LBM_BATCH_PER_STEP, LBM_BATCH_PERSISTENT})
        for (int th : {64, 128, 256})
            for (int bps : {2, 4, 8, 16, 32}) {
                if (mode == LBM_BATCH_PERSISTENT) {
                    b->mode = mode;
                    const int r = resident_blocks(b, th);
                    b->mode = LBM_BATCH_PER_STEP;
                    if (bps > r) continue;
                }
                cand.push_back({mode, th, bps});
            }
    float best_ms = 1e30f;
    Plan best{b->mode, b->threads, b->blocks_per_sm};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == LBM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = LBM_ERR_CUDA;
    if (rc == LBM_OK) rc = set_all_active(b, 1);
    for (size_t ci = 0; ci < cand.size() && rc == LBM_OK; ci++) {
        b->mode = cand[ci].mode;
        b->threads = cand[ci].threads;
        b->blocks_per_sm = cand[ci].bps;
        rc = upload_cases(b);
        if (rc) break;
        if (launch_batch_steps(b, 2) != cudaSuccess) {   // warm-up; a plan that cannot launch is skipped
            cudaGetLastError();
            continue;
        }
        cudaEventRecord(e0, b->stream);
        const cudaError_t le = launch_batch_steps(b, steps);
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = LBM_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        // a persistent plan that gave up a barrier is not a candidate; its
        // error word is cleared (the states are restored below)
        const bool gave_up = batch_err(b) != LBM_OK;
        if (gave_up && cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
        if (rc == LBM_OK && le == cudaSuccess && !gave_up && ms < best_ms) {
            best_ms = ms;
            best = cand[ci];
        }
        cudaGetLastError();
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
    b->mode = best.mode;
    b->threads = best.threads;
    b->blocks_per_sm = best.bps;
    if (rc == LBM_OK) rc = upload_cases(b);
    if (rc == LBM_OK) rc = batch_err(b);
    if (threads_out) *threads_out = best.threads;
    return rc;
}

}  // extern "C"
