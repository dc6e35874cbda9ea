// lbm_debug.cu -- the padding canary and the rounding check of include/lbm_debug.h.
#include <cuda_runtime.h>

#include "lbm_debug.h"
#include "lbm_internal.h"
#include "lbm_round.cuh"

namespace {

// Count nonzero bytes of the padding (row bytes [row_bytes, pitch_bytes))
// of `rows` rows of pitch_bytes bytes starting at base.
__global__ void padding_count_kernel(const unsigned char *__restrict__ base, int64_t rows, int64_t pitch_bytes,
                                     int64_t row_bytes, unsigned long long *__restrict__ out)
{
    const int64_t pad = pitch_bytes - row_bytes;
    const int64_t total = rows * pad;
    unsigned long long cnt = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / pad, b = i - r * pad;
        cnt += base[r * pitch_bytes + row_bytes + b] != 0;
    }
    if (cnt) atomicAdd(out, cnt);
}

// The step kernels' pair conversion applied to given values and random bits.
__global__ void sr_pairs_kernel(int fmt, const float *__restrict__ x, const uint32_t *__restrict__ r,
                                uint32_t *__restrict__ out, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = fmt == 0 ? lbm::sr_half2(x[2 * i], x[2 * i + 1], r[i]) : lbm::sr_bf16x2(x[2 * i], x[2 * i + 1], r[i]);
}

}  // namespace

extern "C" int lbm_debug_padding_canary(lbm_ctx *c, unsigned long long *nonzero)
{
    if (!c || !nonzero) return LBM_ERR_ARG;
    *nonzero = 0;
    if (cudaSetDevice(c->device) != cudaSuccess) return LBM_ERR_CUDA;
    if (c->pitch == c->nx) return LBM_OK;
    unsigned long long *d = nullptr;
    if (cudaMalloc(&d, sizeof(*d)) != cudaSuccess) return LBM_ERR_OOM;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(*d), c->stream);
    const int nbuf = c->opts.layout == 1 ? 1 : 2;
    for (int b = 0; b < nbuf && e == cudaSuccess; b++) {
        const struct {
            const void *base;
            size_t es;
            int64_t planes;
        } parts[2] = {{c->buf.dist[b], c->dist_elem, 14}, {c->buf.tau[b], c->tau_elem, 1}};
        for (const auto &pt : parts) {
            if (!pt.base) continue;
            const int64_t rows = pt.planes * c->ny;
            padding_count_kernel<<<152 * 4, 256, 0, c->stream>>>((const unsigned char *)pt.base, rows,
                                                                 c->pitch * (int64_t)pt.es, c->nx * (int64_t)pt.es, d);
            e = cudaGetLastError();
            if (e != cudaSuccess) break;
        }
    }
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    *nonzero = h;
    return LBM_OK;
}

extern "C" int lbm_debug_sr_pairs(int device, int fmt, const float *x, const uint32_t *r, uint16_t *out,
                                  size_t n_pairs)
{
    if (!x || !r || !out || (fmt != 0 && fmt != 1)) return LBM_ERR_ARG;
    if (n_pairs == 0) return LBM_OK;
    if (cudaSetDevice(device) != cudaSuccess) return LBM_ERR_CUDA;
    float *dx = nullptr;
    uint32_t *dr = nullptr, *dout = nullptr;
    if (cudaMalloc(&dx, n_pairs * 2 * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&dr, n_pairs * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&dout, n_pairs * sizeof(uint32_t)) != cudaSuccess) {
        cudaFree(dx);
        cudaFree(dr);
        cudaFree(dout);
        return LBM_ERR_OOM;
    }
    cudaError_t e = cudaMemcpy(dx, x, n_pairs * 2 * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dr, r, n_pairs * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const size_t blocks = (n_pairs + 255) / 256;
        sr_pairs_kernel<<<(unsigned)(blocks < 152 * 8 ? blocks : 152 * 8), 256>>>(fmt, dx, dr, dout, n_pairs);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, n_pairs * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    cudaFree(dx);
    cudaFree(dr);
    cudaFree(dout);
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
