// lbm_tma.cu -- the fused pull-scheme step with its inputs staged in shared
// memory by bulk asynchronous copies (the Tensor Memory Accelerator's
// cp.async.bulk, completion tracked by an mbarrier), for the storages computed
// in FP32 (FP32, FP32-deviation, BF16- and FP16-deviation).
//
// Work unit: a tile of 256 nodes of one row.  A persistent grid walks the
// tiles; each block keeps 3 (FP32) or 4 (16-bit) tile stages in shared
// memory, and while its four consumer warps compute one tile a producer warp
// has the copy engine fetch the next ones, so the DRAM latency is hidden by
// the copy pipeline rather than by resident warps.  Per
// tile and population plane the block copies the row the plane is pulled
// from (y - e_y) over the tile's columns plus a 16-byte halo on each side;
// the lagged-tau variant also copies the tile's tau row.  The arithmetic is
// the one of the register path (lbm_step.cuh): two nodes per thread on the
// packed FP32x2 pipe, results stored straight to global memory.  Warps that
// touch a wall or the ragged end of a row, and the top and bottom rows, run
// the per-node path with the wall rules from global memory, as there.
//
// Every wait on an mbarrier is bounded; a block that gives up raises the
// context's error word (reported as LBM_ERR_TIMEOUT), waits a bounded time
// for its copies in flight, and returns.
#include <stdint.h>

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_step.cuh"

namespace lbm {

constexpr int TMA_TILE = 256;      // nodes per tile
constexpr uint32_t TMA_SPIN = 1u << 20;  // mbarrier polls before giving up

template <int PREC>
struct TmaGeom {
    using S = typename Store<PREC>::S;
    static constexpr int HALO = 16 / (int)sizeof(S);       // elements in 16 bytes
    static constexpr int W = TMA_TILE + 2 * HALO;          // elements per staged row
    static constexpr int ROW_BYTES = W * (int)sizeof(S);   // a multiple of 16
    // shared bytes of one stage: 14 population rows, then the tau row
    static constexpr int stage_bytes(int tau) { return 14 * ROW_BYTES + (tau ? 0 : TMA_TILE * 4); }
    // tiles in flight per block: 3 x 15.8 KB (FP32) or 4 x 8.6 KB (16-bit),
    // inside the 48 KB a block gets without opting in
    static constexpr int STAGES = sizeof(S) == 4 ? 3 : 4;
    // blocks per SM the shared memory allows; registers are capped to match
    static constexpr int MIN_BLOCKS = sizeof(S) == 4 ? 4 : 5;
};

// Row each plane is pulled from, relative to the tile's row: f_i(x) comes
// from x - e_i.  Order f0..f8, g0..g4.
__device__ __forceinline__ int pull_dy(int q)
{
    // e_y = +1 for f2, f5, f6, g2 (planes 2, 5, 6, 11), -1 for f4, f7, f8, g4
    // (planes 4, 7, 8, 13), 0 otherwise
    constexpr unsigned UP = (1u << 2) | (1u << 5) | (1u << 6) | (1u << 11);
    constexpr unsigned DOWN = (1u << 4) | (1u << 7) | (1u << 8) | (1u << 13);
    return (int)((DOWN >> q) & 1u) - (int)((UP >> q) & 1u);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    for (uint32_t i = 0; i < TMA_SPIN; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// Global -> shared bulk copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned), completing `bytes` transactions on bar.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Issue the copies of tile t into one stage (thread 0 only).  Top and bottom
// rows copy nothing: their nodes take the per-node path.
template <int PREC, int TAU>
__device__ __forceinline__ void tma_issue(const typename Store<PREC>::S *src, const float *tsrc,
                                          const Phys<float> &p, int tiles_x, int64_t t, unsigned char *stage,
                                          uint64_t *bar)
{
    using G = TmaGeom<PREC>;
    using S = typename Store<PREC>::S;
    const int y = (int)(t / tiles_x);
    const int x0 = (int)(t - (int64_t)y * tiles_x) * TMA_TILE;
    if (y < 1 || y > p.ny - 2) {
        mbar_arrive_expect_tx(bar, 0);
        return;
    }
    const int cs = x0 - G::HALO > 0 ? x0 - G::HALO : 0;
    const int ce = x0 + TMA_TILE + G::HALO < p.pitch ? x0 + TMA_TILE + G::HALO : (int)p.pitch;
    const uint32_t row_bytes = (uint32_t)(ce - cs) * (uint32_t)sizeof(S);
    const int t_end = x0 + TMA_TILE < p.pitch ? x0 + TMA_TILE : (int)p.pitch;
    const uint32_t tau_bytes = TAU ? 0u : (uint32_t)(t_end - x0) * 4u;
    mbar_arrive_expect_tx(bar, 14u * row_bytes + tau_bytes);
    const int off = cs - (x0 - G::HALO);   // 0, or HALO at the left end of a row
#pragma unroll 1
    for (int q = 0; q < 14; ++q) {
        const S *row = src + (int64_t)q * p.plane + (int64_t)(y + pull_dy(q)) * p.pitch + cs;
        bulk_g2s(stage + q * G::ROW_BYTES + off * (int)sizeof(S), row, row_bytes, bar);
    }
    if (!TAU) bulk_g2s(stage + 14 * G::ROW_BYTES, tsrc + (int64_t)y * p.pitch + x0, tau_bytes, bar);
}

// Fast-path body: the warp's 64 nodes and their neighbours are interior.
// j: staged index of the thread's first node.
template <int PREC, int FIELD, int TAU>
__device__ __forceinline__ void tma_tile_fast(const unsigned char *stage, typename Store<PREC>::S *__restrict__ dst,
                                              float *__restrict__ tdst, const Phys<F2> &p2, int64_t k, int j)
{
    using St = Store<PREC>;
    using G = TmaGeom<PREC>;
    using S = typename St::S;
    const S *r[14];
#pragma unroll
    for (int q = 0; q < 14; ++q) r[q] = reinterpret_cast<const S *>(stage + q * G::ROW_BYTES);
    auto pair_l = [&](int q, float rest) {   // nodes' left neighbours (x - 1, x)
        return F2(St::ldd(r[q], j - 1, rest), St::ldd(r[q], j, rest));
    };
    auto pair_r = [&](int q, float rest) {   // right neighbours (x + 1, x + 2)
        return F2(St::ldd(r[q], j + 1, rest), St::ldd(r[q], j + 2, rest));
    };
    F2 f[9], g[5];
    f[0] = St::ldd2(r[0], j, float(rest_f(0)));
    f[1] = pair_l(1, float(rest_f(1)));
    f[2] = St::ldd2(r[2], j, float(rest_f(2)));
    f[3] = pair_r(3, float(rest_f(3)));
    f[4] = St::ldd2(r[4], j, float(rest_f(4)));
    f[5] = pair_l(5, float(rest_f(5)));
    f[6] = pair_r(6, float(rest_f(6)));
    f[7] = pair_r(7, float(rest_f(7)));
    f[8] = pair_l(8, float(rest_f(8)));
    g[0] = St::ldd2(r[9], j, float(rest_g(0)));
    g[1] = pair_l(10, float(rest_g(1)));
    g[2] = St::ldd2(r[11], j, float(rest_g(2)));
    g[3] = pair_r(12, float(rest_g(3)));
    g[4] = St::ldd2(r[13], j, float(rest_g(4)));
    const float *trow = reinterpret_cast<const float *>(stage + 14 * G::ROW_BYTES);
    const F2 t0 = tau_start<TAU, F2, FIELD, 1>(p2, f, g, k, [&] {
        return F2(*reinterpret_cast<const float2 *>(trow + (j - G::HALO)));
    });
    Macro<F2> m;
    const F2 tau = collide<F2, FIELD, 1>(p2, f, g, t0, m, k);
    const int64_t P = p2.plane;
    uint32_t rng = rng_init(p2.seed, k);
#pragma unroll
    for (int i = 0; i < 9; i++) St::sdv2(dst + i * P, k, f[i], float(rest_f(i)), rng);
#pragma unroll
    for (int i = 0; i < 5; i++) St::sdv2(dst + (9 + i) * P, k, g[i], float(rest_g(i)), rng);
    if constexpr (TAU == 0) *reinterpret_cast<float2 *>(tdst + k) = tau.v;
}

// Block = 4 consumer warps (64 nodes of the tile each) + 1 producer warp
// whose lane 0 issues the copies, up to STAGES - 1 tiles ahead.  Stage s has
// two barriers: full[s] completes when the tile's bytes have landed; empty[s]
// when the 4 consumer warps are done reading it.
template <int PREC, int FIELD, int TAU>
__global__ void __launch_bounds__(160, TmaGeom<PREC>::MIN_BLOCKS)
step_tma_kernel(const typename Store<PREC>::S *__restrict__ src, typename Store<PREC>::S *__restrict__ dst,
                const float *__restrict__ tsrc, float *__restrict__ tdst, Phys<float> p, Phys<F2> p2, int tiles_x,
                int64_t ntiles, unsigned *err)
{
    using G = TmaGeom<PREC>;
    constexpr int NS = G::STAGES;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[NS], empty[NS];
    constexpr int SB = G::stage_bytes(TAU);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == 4) {   // producer
        if (lane != 0) return;
        uint32_t it = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
            const int s = it % NS;
            const uint32_t round = it / NS;
            if (round > 0 && !mbar_wait_bounded(&empty[s], (round - 1) & 1)) {
                ok = false;
                break;
            }
            tma_issue<PREC, TAU>(src, tsrc, p, tiles_x, t, smem + s * SB, &full[s]);
        }
        if (!ok) {   // let the copies already issued land before the block's shared memory goes
            atomicExch(err, 1u);
            for (uint32_t j = it > (uint32_t)NS ? it - NS : 0; j < it; ++j)
                mbar_wait_bounded(&full[j % NS], (j / NS) & 1);
        }
        return;
    }
    uint32_t it = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int s = it % NS;
        const bool ok = mbar_wait_bounded(&full[s], (it / NS) & 1);
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) atomicExch(err, 1u);
            return;
        }
        const int y = (int)(t / tiles_x);
        const int x0 = (int)(t - (int64_t)y * tiles_x) * TMA_TILE;
        const int xn = x0 + 2 * (int)threadIdx.x;
        const int wx = x0 + 64 * warp;
        const bool fast = y > 0 && y < p.ny - 1 && wx > 0 && wx + 64 < p.nx;
        if (fast) {
            tma_tile_fast<PREC, FIELD, TAU>(smem + s * SB, dst, tdst, p2, (int64_t)y * p.pitch + xn,
                                            2 * (int)threadIdx.x + G::HALO);
        } else {
            for (int jn = 0; jn < 2; jn++)
                if (xn + jn < p.nx) step_node<PREC, float, FIELD, TAU>(src, dst, tsrc, tdst, p, xn + jn, y);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

// ------------------------------------------------------------- launcher
template <int PREC, int FIELD, int TAU>
static cudaError_t tma_launch_t(lbm_ctx *c, const void *src, void *dst, const void *tsrc, void *tdst)
{
    using St = Store<PREC>;
    auto *kern = step_tma_kernel<PREC, FIELD, TAU>;
    const int sb = TmaGeom<PREC>::STAGES * TmaGeom<PREC>::stage_bytes(TAU);
    const int tiles_x = (c->nx + TMA_TILE - 1) / TMA_TILE;
    const int64_t ntiles = (int64_t)tiles_x * c->ny;
    int per_sm = 0, nsm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 160, sb);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)nsm * per_sm;
    if (grid > ntiles) grid = ntiles;
    kern<<<(unsigned)grid, 160, sb, c->stream>>>((const typename St::S *)src, (typename St::S *)dst,
                                                 (const float *)tsrc, (float *)tdst, make_params<float>(c),
                                                 make_params<F2>(c), tiles_x, ntiles, c->d_err);
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t tma_dispatch(lbm_ctx *c, const void *src, void *dst, const void *tsrc, void *tdst)
{
    const bool field = c->d_da != nullptr, tau = c->opts.tau_iters > 0;
    if (field)
        return tau ? tma_launch_t<PREC, 1, 1>(c, src, dst, tsrc, tdst) : tma_launch_t<PREC, 1, 0>(c, src, dst, tsrc, tdst);
    return tau ? tma_launch_t<PREC, 0, 1>(c, src, dst, tsrc, tdst) : tma_launch_t<PREC, 0, 0>(c, src, dst, tsrc, tdst);
}

cudaError_t launch_step_tma(lbm_ctx *c, const void *src, void *dst, const void *tsrc, void *tdst)
{
    switch (c->opts.prec) {
    case LBM_F32: return tma_dispatch<LBM_F32>(c, src, dst, tsrc, tdst);
    case LBM_F32D: return tma_dispatch<LBM_F32D>(c, src, dst, tsrc, tdst);
    case LBM_BF16D: return tma_dispatch<LBM_BF16D>(c, src, dst, tsrc, tdst);
    case LBM_F16D: return tma_dispatch<LBM_F16D>(c, src, dst, tsrc, tdst);
    case LBM_F16S: return tma_dispatch<LBM_F16S>(c, src, dst, tsrc, tdst);
    case LBM_BF16S: return tma_dispatch<LBM_BF16S>(c, src, dst, tsrc, tdst);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm
