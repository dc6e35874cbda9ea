// lbm_noalloc.cu -- lbm_residual_noalloc: the convergence residual without any
// device allocation, for callers that cannot call cudaMalloc (see lbm.h).
//
// Its only scratch is the file-scope array below: one slot of partial sums
// per grid row, LBM_NOALLOC_MAX_ROWS rows at most (1 MiB).  Every GPU that
// loads this library holds the array until the process exits.
#include <cuda.h>  // CUcontext / CUresult types only; no link against libcuda
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace {

constexpr int kSlot = 8;  // doubles per row: 7 partial sums + padding
static __device__ __align__(256) double g_row_partials[LBM_NOALLOC_MAX_ROWS * kSlot];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};  // context the address belongs to

// cuCtxGetCurrent, fetched through the runtime (the library links only the
// CUDA runtime); null if the driver does not offer it.
typedef CUresult (*ctx_get_current_fn)(CUcontext *);
ctx_get_current_fn ctx_get_current()
{
    static ctx_get_current_fn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<ctx_get_current_fn>(p);
    }();
    return fn;
}

// Device address of g_row_partials on device `dev` (current).  In host code
// the symbol's name is only a host-side stand-in, so the address must come
// from cudaGetSymbolAddress: once per device, and again if the device's
// context was replaced since (a cudaDeviceReset destroys the primary
// context, and the array lives at a new address in the next one).  Without
// cuCtxGetCurrent the address is looked up on every call.
int scratch_address(int dev, double **out)
{
    if (dev < 0 || dev >= kMaxDevices) return LBM_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    CUcontext cur = nullptr;
    const ctx_get_current_fn get = ctx_get_current();
    const bool known = get && get(&cur) == CUDA_SUCCESS && cur;
    if (!g_scratch[dev] || !known || cur != g_scratch_ctx[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_row_partials);
        if (e != cudaSuccess || !p) return LBM_ERR_CUDA;
        g_scratch[dev] = static_cast<double *>(p);
        g_scratch_ctx[dev] = known ? cur : nullptr;
    }
    *out = g_scratch[dev];
    return LBM_OK;
}

__device__ double row_block_sum(double v, double *sh)
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
    return t;
}

// Pass 1: block y sums, over row y, (phi - phi_prev)^2 and phi^2 for
// phi in {u_x, u_y, T} and counts non-finite values; slot y of the scratch
// receives the seven sums.  The caller's snapshot is updated in place.
template <int PREC>
__global__ void __launch_bounds__(256)
residual_rows_kernel(const typename lbm::Store<PREC>::S *__restrict__ src,
                     const typename lbm::Store<PREC>::TauS *__restrict__ tsrc,
                     lbm::Phys<typename lbm::Store<PREC>::R> p, double *__restrict__ snap,
                     double *__restrict__ part, int first)
{
    using R = typename lbm::Store<PREC>::R;
    __shared__ double sh[32];
    const int y = blockIdx.x;
    const int64_t n = (int64_t)p.nx * p.ny;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int x = threadIdx.x; x < p.nx; x += blockDim.x) {
        R f[9], g[5];
        lbm::pull<PREC, R>(src, p, x, y, f, g);
        const int64_t k = (int64_t)y * p.pitch + x;
        const lbm::Macro<R> m =
            lbm::macro<R>(p, f, g, p.tau_iters ? lbm::implicit_tau<R>(p, f, g, k) : R(tsrc[k]), k);
        const double v[3] = {double(m.ux), double(m.uy), double(m.T)};
        const int64_t q = (int64_t)y * p.nx + x;
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
        const double s = row_block_sum(acc[c], sh);
        if (threadIdx.x == 0) part[(int64_t)y * kSlot + c] = s;
    }
}

// Pass 2: one block adds the row slots in row order; out[0..2] = relative
// change of u_x, u_y, T (+inf on a first call), out[3] = non-finite count.
__global__ void __launch_bounds__(256)
residual_rows_final(const double *__restrict__ part, int rows, int first, double *__restrict__ out)
{
    __shared__ double sh[32];
    double tot[7];
    for (int c = 0; c < 7; c++) {
        double a = 0.0;
        for (int r = threadIdx.x; r < rows; r += blockDim.x) a += part[(int64_t)r * kSlot + c];
        tot[c] = row_block_sum(a, sh);
    }
    if (threadIdx.x == 0) {
        for (int c = 0; c < 3; c++) {
            const double num = tot[2 * c], den = tot[2 * c + 1];
            out[c] = first ? INFINITY : (den > 0.0 ? sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0));
        }
        out[3] = tot[6];
    }
}

template <int PREC>
cudaError_t launch(lbm_ctx *c, double *snap, int first, double *out, double *part)
{
    using St = lbm::Store<PREC>;
    residual_rows_kernel<PREC><<<c->ny, 256, 0, c->stream>>>(
        (const typename St::S *)c->buf.dist[c->cur], (const typename St::TauS *)c->buf.tau[c->cur],
        lbm::make_params<typename St::R>(c), snap, part, first);
    residual_rows_final<<<1, 256, 0, c->stream>>>(part, c->ny, first, out);
    return cudaGetLastError();
}

}  // namespace

extern "C" int lbm_residual_noalloc(lbm_ctx *c, double *d_snapshot, int first, double *d_result)
{
    if (!c || !d_snapshot || !d_result) return LBM_ERR_ARG;
    if (c->ny > LBM_NOALLOC_MAX_ROWS) return LBM_ERR_SIZE;
    if (c->opts.layout != 0) return LBM_ERR_UNSUPPORTED;   // two-buffer layout only
    if (c->row_lo != 0 || c->row_hi != c->ny) return LBM_ERR_UNSUPPORTED;   // whole cavities only
    if (cudaSetDevice(c->device) != cudaSuccess) return LBM_ERR_CUDA;
    double *part = nullptr;
    const int rc = scratch_address(c->device, &part);
    if (rc != LBM_OK) return rc;
    cudaError_t e;
    switch (c->opts.prec) {
    case LBM_F64: e = launch<LBM_F64>(c, d_snapshot, first ? 1 : 0, d_result, part); break;
    case LBM_F32: e = launch<LBM_F32>(c, d_snapshot, first ? 1 : 0, d_result, part); break;
    case LBM_BF16D: e = launch<LBM_BF16D>(c, d_snapshot, first ? 1 : 0, d_result, part); break;
    case LBM_F16D: e = launch<LBM_F16D>(c, d_snapshot, first ? 1 : 0, d_result, part); break;
    case LBM_F32D: e = launch<LBM_F32D>(c, d_snapshot, first ? 1 : 0, d_result, part); break;
    case LBM_F16S: e = launch<LBM_F16S>(c, d_snapshot, first ? 1 : 0, d_result, part); break;
    case LBM_BF16S: e = launch<LBM_BF16S>(c, d_snapshot, first ? 1 : 0, d_result, part); break;
    default: return LBM_ERR_ARG;
    }
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
