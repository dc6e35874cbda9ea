// lbm_bench.cu -- FMA-throughput probes (include/lbm_bench.h): the measured
// ALU peaks that the FP64 step kernel's roofline and the FMA-pipe activity of
// the FP32 kernels are compared with.
#include <cuda_runtime.h>

#include "lbm.h"
#include "lbm_bench.h"

namespace {

constexpr int kChains = 8;     // independent accumulators per thread
constexpr int kIters = 2048;   // dependent FMAs per chain
constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) fma_kernel(T a, T b, T *out, int store)
{
    T acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) acc[c] = T(threadIdx.x + c);
#pragma unroll 16
    for (int i = 0; i < kIters; i++)
#pragma unroll
        for (int c = 0; c < kChains; c++) acc[c] = fma(acc[c], a, b);
    T s = acc[0];
#pragma unroll
    for (int c = 1; c < kChains; c++) s += acc[c];
    if (store) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains alive
}

__global__ void __launch_bounds__(kThreads) fma2_kernel(float2 a, float2 b, float2 *out, int store)
{
    float2 acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) acc[c] = make_float2(threadIdx.x + c, c);
#pragma unroll 16
    for (int i = 0; i < kIters; i++)
#pragma unroll
        for (int c = 0; c < kChains; c++) acc[c] = __ffma2_rn(acc[c], a, b);
    float2 s = acc[0];
#pragma unroll
    for (int c = 1; c < kChains; c++) s = __fadd2_rn(s, acc[c]);
    if (store) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int lbm_bench_fma_peak(int kind, int device, int reps, double *fma_per_s, double *inst_per_s)
{
    if (kind < 0 || kind > 2 || reps < 1 || !fma_per_s) return LBM_ERR_ARG;
    if (device >= 0 && cudaSetDevice(device) != cudaSuccess) return LBM_ERR_CUDA;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LBM_ERR_CUDA;
    const int blocks = sms * 8;   // 8 x 256 threads per SM: every scheduler busy
    void *out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * kThreads * 16) != cudaSuccess) return LBM_ERR_CUDA;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = LBM_OK;
    float ms = 0.f;
    auto launch = [&]() {
        if (kind == 0)
            fma_kernel<double><<<blocks, kThreads>>>(0.999999, 1e-7, (double *)out, 0);
        else if (kind == 1)
            fma_kernel<float><<<blocks, kThreads>>>(0.999999f, 1e-7f, (float *)out, 0);
        else
            fma2_kernel<<<blocks, kThreads>>>(make_float2(0.999999f, 0.999998f), make_float2(1e-7f, 2e-7f),
                                              (float2 *)out, 0);
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = LBM_ERR_CUDA;
    } else {
        launch();
        cudaEventRecord(e0);
        for (int r = 0; r < reps; r++) launch();
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f))
            rc = LBM_ERR_CUDA;
    }
    if (rc == LBM_OK) {
        const double inst = (double)blocks * kThreads * kChains * kIters * reps;
        const double secs = ms * 1e-3;
        *fma_per_s = inst * (kind == 2 ? 2.0 : 1.0) / secs;
        if (inst_per_s) *inst_per_s = inst / secs;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}
