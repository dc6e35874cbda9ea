// lbm_step_rows.cu -- the two-node step for the 16-bit storages with a
// per-warp asynchronous-copy pipeline over rows.
//
// With 16-bit storage a warp's loads for one row carry half the bytes of the
// FP32 form, so at the occupancy the arithmetic allows too few bytes are in
// flight to cover the DRAM latency (the register path reaches 0.75 of the
// copy bandwidth).  Here each warp owns a 64-node column segment over ROWS
// consecutive rows and keeps NST row stages in shared memory: every thread
// copies its pair word of each pulled plane (cp.async, 4 bytes, no register
// held while in flight), lanes 0 and 31 also the words holding the x-halo,
// two rows ahead of the one it computes.  The warp synchronises only with
// itself (cp.async.wait_group, __syncwarp); the x-shifted populations are
// read from the neighbours' words in shared memory, so no shuffles.  The
// arithmetic is the one of lbm_step.cuh (deviation form, packed FP32x2), and
// so are the results, bit for bit.  Warps that touch a side wall or the
// ragged end of a row, and the top and bottom rows, take the per-node path.
#include <stdint.h>

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_step.cuh"

namespace lbm {

constexpr int ROWS = 16;        // rows per block
constexpr int NST = 3;          // row stages per warp
constexpr int SEG_WORDS = 34;   // words per plane row: x-halo word, 32 pair words, x-halo word
constexpr int STAGE_WORDS = 14 * SEG_WORDS;

__device__ __forceinline__ void cp_async4(uint32_t *dst_smem, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Copy row y's pulled words for a warp's segment starting at wx into a stage
// (plane q from row y - e_y, as in the pull).  Word j of a plane row holds
// nodes wx - 2 + 2j and wx - 1 + 2j.
__device__ __forceinline__ void issue_row(const unsigned short *__restrict__ s, int64_t P, int64_t W, int y,
                                          int wx, int lane, uint32_t *stage)
{
    constexpr unsigned UP = (1u << 2) | (1u << 5) | (1u << 6) | (1u << 11);     // e_y = +1: row y - 1
    constexpr unsigned DOWN = (1u << 4) | (1u << 7) | (1u << 8) | (1u << 13);   // e_y = -1: row y + 1
#pragma unroll
    for (int q = 0; q < 14; ++q) {
        const int row = y + (int)((DOWN >> q) & 1u) - (int)((UP >> q) & 1u);
        const unsigned short *base = s + q * P + (int64_t)row * W + wx;
        uint32_t *dst = stage + q * SEG_WORDS;
        cp_async4(dst + 1 + lane, base + 2 * lane);
        if (lane == 0) cp_async4(dst, base - 2);
        if (lane == 31) cp_async4(dst + 33, base + 64);
    }
}

template <int PREC, int FIELD, int TAU>
__device__ __forceinline__ void compute_row(const uint32_t *__restrict__ st, typename Store<PREC>::S *__restrict__ dst,
                                            const float *__restrict__ tsrc, float *__restrict__ tdst,
                                            const Phys<F2> &p2, int64_t k, int lane)
{
    using St = Store<PREC>;
    // own pair word (nodes x0, x0 + 1) and the pairs shifted by -1 / +1 node
    auto own = [&](int q) { return St::dec2(st[q * SEG_WORDS + 1 + lane]); };
    auto left = [&](int q) {
        return St::dec2(__funnelshift_r(st[q * SEG_WORDS + lane], st[q * SEG_WORDS + 1 + lane], 16));
    };
    auto right = [&](int q) {
        return St::dec2(__funnelshift_r(st[q * SEG_WORDS + 1 + lane], st[q * SEG_WORDS + 2 + lane], 16));
    };
    F2 f[9], g[5];
    f[0] = own(0);
    f[1] = left(1);
    f[2] = own(2);
    f[3] = right(3);
    f[4] = own(4);
    f[5] = left(5);
    f[6] = right(6);
    f[7] = right(7);
    f[8] = left(8);
    g[0] = own(9);
    g[1] = left(10);
    g[2] = own(11);
    g[3] = right(12);
    g[4] = own(13);
    const F2 t0 =
        tau_start<TAU, F2, FIELD, 1>(p2, f, g, k, [&] { return F2(*reinterpret_cast<const float2 *>(tsrc + k)); });
    Macro<F2> m;
    const F2 tau = collide<F2, FIELD, 1>(p2, f, g, t0, m, k);
    uint32_t rng = rng_init(p2.seed, k);
    const int64_t P = p2.plane;
#pragma unroll
    for (int i = 0; i < 9; i++) St::sdv2(dst + i * P, k, f[i], float(rest_f(i)), rng);
#pragma unroll
    for (int i = 0; i < 5; i++) St::sdv2(dst + (9 + i) * P, k, g[i], float(rest_g(i)), rng);
    if constexpr (TAU == 0) *reinterpret_cast<float2 *>(tdst + k) = tau.v;
}

template <int PREC, int FIELD, int TAU>
__global__ void __launch_bounds__(128)
step_rows_kernel(const typename Store<PREC>::S *__restrict__ src, typename Store<PREC>::S *__restrict__ dst,
                 const float *__restrict__ tsrc, float *__restrict__ tdst, Phys<float> p, Phys<F2> p2)
{
    __shared__ uint32_t stages[4][NST][STAGE_WORDS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = blockIdx.x * 256 + 2 * threadIdx.x;
    const int wx = blockIdx.x * 256 + 64 * warp;
    const int y0 = blockIdx.y * ROWS;
    const int y1 = y0 + ROWS < p.ny ? y0 + ROWS : p.ny;
    if (!(wx > 0 && wx + 64 < p.nx)) {   // side walls, ragged row end: per node (uniform per warp)
        for (int y = y0; y < y1; ++y)
            for (int j = 0; j < 2; j++)
                if (x0 + j < p.nx) step_node<PREC, float, FIELD, TAU>(src, dst, tsrc, tdst, p, x0 + j, y);
        return;
    }
    const unsigned short *s = reinterpret_cast<const unsigned short *>(src);
    const int64_t P = p.plane, W = p.pitch;
    auto interior = [&](int y) { return y > 0 && y < p.ny - 1; };
    uint32_t(*stg)[STAGE_WORDS] = stages[warp];
    // prologue: rows y0 and y0 + 1 (one commit group per row, empty for rows
    // outside the block or on a wall, so that the group count stays uniform)
    for (int r = 0; r < 2; ++r) {
        const int y = y0 + r;
        if (y < y1 && interior(y)) issue_row(s, P, W, y, wx, lane, stg[r]);
        cp_async_commit();
    }
#pragma unroll 1
    for (int y = y0; y < y1; ++y) {
        const int i = y - y0;
        const int yn = y + 2;
        if (yn < y1 && interior(yn)) issue_row(s, P, W, yn, wx, lane, stg[(i + 2) % NST]);
        cp_async_commit();
        asm volatile("cp.async.wait_group 2;" ::: "memory");   // row y's group has landed
        __syncwarp();
        if (interior(y)) {
            compute_row<PREC, FIELD, TAU>(stg[i % NST], dst, tsrc, tdst, p2, (int64_t)y * W + x0, lane);
        } else {
            for (int j = 0; j < 2; j++) step_node<PREC, float, FIELD, TAU>(src, dst, tsrc, tdst, p, x0 + j, y);
        }
        __syncwarp();   // the stage is read before a later row is copied into it
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

template <int PREC>
static cudaError_t rows_launch(lbm_ctx *c, const void *src, void *dst, const void *tsrc, void *tdst)
{
    using St = Store<PREC>;
    const dim3 grid((c->nx + 255) / 256, (c->ny + ROWS - 1) / ROWS);
    const bool field = c->d_da != nullptr, tau = c->opts.tau_iters > 0;
    auto *kern = field ? (tau ? step_rows_kernel<PREC, 1, 1> : step_rows_kernel<PREC, 1, 0>)
                       : (tau ? step_rows_kernel<PREC, 0, 1> : step_rows_kernel<PREC, 0, 0>);
    kern<<<grid, 128, 0, c->stream>>>((const typename St::S *)src, (typename St::S *)dst, (const float *)tsrc,
                                      (float *)tdst, make_params<float>(c), make_params<F2>(c));
    return cudaGetLastError();
}

cudaError_t launch_step_rows(lbm_ctx *c, const void *src, void *dst, const void *tsrc, void *tdst)
{
    switch (c->opts.prec) {
    case LBM_BF16D: return rows_launch<LBM_BF16D>(c, src, dst, tsrc, tdst);
    case LBM_F16D: return rows_launch<LBM_F16D>(c, src, dst, tsrc, tdst);
    case LBM_F16S: return rows_launch<LBM_F16S>(c, src, dst, tsrc, tdst);
    case LBM_BF16S: return rows_launch<LBM_BF16S>(c, src, dst, tsrc, tdst);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm
