// lbm_debug.cu -- the padding canary of include/lbm_debug.h.
#include <cuda_runtime.h>

#include "lbm_debug.h"
#include "lbm_internal.h"

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
