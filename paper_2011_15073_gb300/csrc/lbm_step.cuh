// lbm_step.cuh -- bodies of the fused pull-scheme step: one node at a time
// (any precision), a tile of two nodes per thread (FP32 arithmetic), used by
// the single-cavity kernels and by the batched sweep, and a tile of four
// nodes per thread for the 16-bit storages.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// Pull, collide and store one node (wall rules included).  TAU 0: the
// collision starts from the stored lagged tau and stores its new tau; TAU 1:
// from the node-local implicit tau, and no tau is read or written.  For the
// FP32-arithmetic storages the arithmetic runs on deviations from the rest
// state (DEV form of pull, macro and collide), which keeps the small
// per-step changes of a nearly steady state out of the rounding of O(1)
// population values; FP64 runs on full values (dev_form).  `seed`: the
// stochastic rounding's seed of this step (step_seed; Phys::seed in a plain
// launch).
template <int PREC, class R, int FIELD = 2, int TAU = 0>
__device__ __forceinline__ void step_node(const typename Store<PREC>::S *__restrict__ src,
                                          typename Store<PREC>::S *__restrict__ dst,
                                          const typename Store<PREC>::TauS *__restrict__ tsrc,
                                          typename Store<PREC>::TauS *__restrict__ tdst, const Phys<R> &p, int x,
                                          int y, uint32_t seed)
{
    using St = Store<PREC>;
    const int64_t k = (int64_t)y * p.pitch + x;
    R f[9], g[5];
    constexpr int DEV = dev_form<PREC>();
    pull<PREC, R, false, DEV>(src, p, x, y, f, g);
    Macro<R> m;
    const R t0 = tau_start<TAU, R, FIELD, DEV>(p, f, g, k, [&] { return R(tsrc[k]); });
    const R tau = collide<R, FIELD, DEV>(p, f, g, t0, m, k);
    uint32_t rng = rng_init(seed, k);   // random bits of the stochastic-rounding storages
#pragma unroll
    for (int i = 0; i < 9; i++) stf<PREC>(dst, i * p.plane + k, f[i], R(rest_f(i)), rng);
#pragma unroll
    for (int i = 0; i < 5; i++) stf<PREC>(dst + 9 * p.plane, i * p.plane + k, g[i], R(rest_g(i)), rng);
    if constexpr (TAU == 0) tdst[k] = typename St::TauS(tau);
}

// One tile of a row: thread t of the block updates nodes xbase + 2t and
// xbase + 2t + 1 of row y.  A warp whose 64 nodes and their neighbours are
// all interior takes the fast path -- aligned pair loads and stores, the
// x-shifted populations exchanged by warp shuffles, both nodes' arithmetic
// on the packed FP32x2 pipe; any warp that touches a wall or the ragged end
// of a row updates its nodes one at a time with the wall rules.  The branch
// is uniform per warp.  (Handing the side-wall warps to the packed path, as
// step4_tile does, costs this tile 8-40 registers per thread in its
// single-cavity and batched kernels; at 64 nodes per warp the wall warps are
// a small share of a row.)  TAU and seed as for step_node.
template <int PREC, int FIELD = 2, int TAU = 0>
__device__ __forceinline__ void step2_tile(const typename Store<PREC>::S *__restrict__ src,
                                           typename Store<PREC>::S *__restrict__ dst,
                                           const float *__restrict__ tsrc, float *__restrict__ tdst,
                                           const Phys<float> &p, const Phys<F2> &p2, int xbase, int y,
                                           uint32_t seed)
{
    using St = Store<PREC>;
    using S = typename St::S;
    const int lane = threadIdx.x & 31;
    const int x0 = xbase + 2 * threadIdx.x;
    const int wx = xbase + 2 * (threadIdx.x & ~31);
    const bool fast = y > 0 && y < p.ny - 1 && wx > 0 && wx + 64 < p.nx;
    if (!fast) {
        for (int j = 0; j < 2; j++)
            if (x0 + j < p.nx) step_node<PREC, float, FIELD, TAU>(src, dst, tsrc, tdst, p, x0 + j, y, seed);
        return;
    }
    const int64_t P = p.plane, W = p.pitch;
    const int64_t k = (int64_t)y * W + x0;
    const S *fs = src;
    const S *gs = src + 9 * P;
    const bool l0 = lane == 0, l31 = lane == 31;
    F2 f[9], g[5];
    f[0] = St::ldd2(fs, k, float(rest_f(0)));
    f[1] = from_left(St::ldd2(fs + P, k, float(rest_f(1))), l0 ? St::ldd(fs + P, k - 1, float(rest_f(1))) : 0.f, lane);
    f[2] = St::ldd2(fs + 2 * P, k - W, float(rest_f(2)));
    f[3] = from_right(St::ldd2(fs + 3 * P, k, float(rest_f(3))), l31 ? St::ldd(fs + 3 * P, k + 2, float(rest_f(3))) : 0.f, lane);
    f[4] = St::ldd2(fs + 4 * P, k + W, float(rest_f(4)));
    f[5] = from_left(St::ldd2(fs + 5 * P, k - W, float(rest_f(5))),
                     l0 ? St::ldd(fs + 5 * P, k - W - 1, float(rest_f(5))) : 0.f, lane);
    f[6] = from_right(St::ldd2(fs + 6 * P, k - W, float(rest_f(6))),
                      l31 ? St::ldd(fs + 6 * P, k - W + 2, float(rest_f(6))) : 0.f, lane);
    f[7] = from_right(St::ldd2(fs + 7 * P, k + W, float(rest_f(7))),
                      l31 ? St::ldd(fs + 7 * P, k + W + 2, float(rest_f(7))) : 0.f, lane);
    f[8] = from_left(St::ldd2(fs + 8 * P, k + W, float(rest_f(8))),
                     l0 ? St::ldd(fs + 8 * P, k + W - 1, float(rest_f(8))) : 0.f, lane);
    g[0] = St::ldd2(gs, k, float(rest_g(0)));
    g[1] = from_left(St::ldd2(gs + P, k, float(rest_g(1))), l0 ? St::ldd(gs + P, k - 1, float(rest_g(1))) : 0.f, lane);
    g[2] = St::ldd2(gs + 2 * P, k - W, float(rest_g(2)));
    g[3] = from_right(St::ldd2(gs + 3 * P, k, float(rest_g(3))), l31 ? St::ldd(gs + 3 * P, k + 2, float(rest_g(3))) : 0.f, lane);
    g[4] = St::ldd2(gs + 4 * P, k + W, float(rest_g(4)));
    const F2 t0 = tau_start<TAU, F2, FIELD, 1>(p2, f, g, k, [&] { return F2(*reinterpret_cast<const float2 *>(tsrc + k)); });
    Macro<F2> m;
    const F2 tau = collide<F2, FIELD, 1>(p2, f, g, t0, m, k);
    uint32_t rng = rng_init(seed, k);
#pragma unroll
    for (int i = 0; i < 9; i++) St::sdv2(dst + i * P, k, f[i], float(rest_f(i)), rng);
#pragma unroll
    for (int i = 0; i < 5; i++) St::sdv2(dst + (9 + i) * P, k, g[i], float(rest_g(i)), rng);
    if constexpr (TAU == 0) *reinterpret_cast<float2 *>(tdst + k) = tau.v;
}

// One pair of nodes of a four-node tile: the 14 stored words of the pair
// (deviation form, already shifted to this pair's sources) -> the 14 words
// to store and the new tau.  The same arithmetic, and the same random bits
// (rng_init at the pair's first node), as step2_tile's pair.
template <int PREC, int FIELD, int TAU>
__device__ __forceinline__ F2 pair_words(const Phys<F2> &p2, const uint32_t (&in)[14], F2 tau_lag, int64_t k,
                                         uint32_t seed, uint32_t (&out)[14])
{
    using St = Store<PREC>;
    F2 f[9], g[5];
#pragma unroll
    for (int i = 0; i < 9; i++) f[i] = St::unpack2(in[i]);
#pragma unroll
    for (int i = 0; i < 5; i++) g[i] = St::unpack2(in[9 + i]);
    const F2 t0 = tau_start<TAU, F2, FIELD, 1>(p2, f, g, k, [&] { return tau_lag; });
    Macro<F2> m;
    const F2 tau = collide<F2, FIELD, 1>(p2, f, g, t0, m, k);
    uint32_t rng = rng_init(seed, k);
#pragma unroll
    for (int i = 0; i < 9; i++) out[i] = St::pack2(f[i], rng);
#pragma unroll
    for (int i = 0; i < 5; i++) out[9 + i] = St::pack2(g[i], rng);
    return tau;
}

// Four nodes per thread for the 16-bit storages: thread t of the block
// updates nodes xbase + 4t .. xbase + 4t + 3 of row y.  Each population row
// is one 8-byte load per thread (twice the bytes in flight per load of
// step2_tile, which the 16-bit storages need to keep HBM busy); the
// x-shifted sources are assembled from the raw 16-bit words by byte
// permutes and one warp shuffle (lane 0 / 31 load their halo word), the two
// pairs are collided one after the other, and each population row is
// stored as one 8-byte word.  The top and bottom rows and the warp at the
// ragged end of a row update their nodes one at a time with the wall rules.
// The first and last warp of a row take the packed path too (at 128 nodes
// per warp, updating them one node at a time cost 6 % of a 4096-wide row's
// nodes three times the instructions); the packed result of the wall node
// itself (x = 0 or nx - 1) used a value from beyond the wall -- the previous
// row's tail or the next row's head, inside the allocation -- so that one
// node is then updated again with the wall rules.  Results equal
// step2_tile's wherever both take the packed path.  seed_of() returns the
// step's seed (as for step_node) where it is used: a plain launch reads its
// parameter there rather than holding it in a register across the tile.
template <int PREC, int FIELD, int TAU, class SeedOf>
__device__ __forceinline__ void step4_tile(const typename Store<PREC>::S *__restrict__ src,
                                           typename Store<PREC>::S *__restrict__ dst,
                                           const float *__restrict__ tsrc, float *__restrict__ tdst,
                                           const Phys<float> &p, const Phys<F2> &p2, int xbase, int y,
                                           SeedOf seed_of)
{
    static_assert(is16<PREC>(), "four-node tiles are built for the 16-bit storages");
    using S = typename Store<PREC>::S;
    const int lane = threadIdx.x & 31;
    const int x0 = xbase + 4 * threadIdx.x;
    const int wx = xbase + 4 * (threadIdx.x & ~31);
    const bool fast = y > 0 && y < p.ny - 1 && wx + 128 <= p.nx;
    if (!fast) {
        for (int j = 0; j < 4; j++)
            if (x0 + j < p.nx) step_node<PREC, float, FIELD, TAU>(src, dst, tsrc, tdst, p, x0 + j, y, seed_of());
        return;
    }
    const int64_t P = p.plane, W = p.pitch;
    const int64_t k = (int64_t)y * W + x0;
    // Source row offset and x-direction of population q (f0..f8, g0..g4):
    // -1 from x - 1, +1 from x + 1.
    const int64_t row[14] = {0, 0, -W, 0, W, -W, -W, W, W, 0, 0, -W, 0, W};
    constexpr int side[14] = {0, -1, 0, 1, 0, -1, 1, 1, -1, 0, -1, 0, 1, 0};
    uint2 c[14];
    uint32_t halo[14];
#pragma unroll
    for (int q = 0; q < 14; q++) {
        const S *b = src + q * P + k + row[q];
        c[q] = *reinterpret_cast<const uint2 *>(b);
        halo[q] = 0;
        if (side[q] < 0 && lane == 0) halo[q] = *reinterpret_cast<const uint32_t *>(b - 2);   // [x0-2, x0-1]
        if (side[q] > 0 && lane == 31) halo[q] = *reinterpret_cast<const uint32_t *>(b + 4);  // [x0+4, x0+5]
    }
    float4 lag = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (TAU == 0) lag = *reinterpret_cast<const float4 *>(tsrc + k);
    // ra: sources of nodes x0, x0+1; rb: of x0+2, x0+3.  __byte_perm(a, b,
    // 0x5432) = (high half of a, low half of b): the pair one node earlier.
    uint32_t ra[14], rb[14];
#pragma unroll
    for (int q = 0; q < 14; q++) {
        if (side[q] < 0) {
            uint32_t prev = __shfl_up_sync(0xffffffffu, c[q].y, 1);
            if (lane == 0) prev = halo[q];
            ra[q] = __byte_perm(prev, c[q].x, 0x5432);
            rb[q] = __byte_perm(c[q].x, c[q].y, 0x5432);
        } else if (side[q] > 0) {
            uint32_t next = __shfl_down_sync(0xffffffffu, c[q].x, 1);
            if (lane == 31) next = halo[q];
            ra[q] = __byte_perm(c[q].x, c[q].y, 0x5432);
            rb[q] = __byte_perm(c[q].y, next, 0x5432);
        } else {
            ra[q] = c[q].x;
            rb[q] = c[q].y;
        }
    }
    uint32_t oa[14], ob[14];
    const F2 ta = pair_words<PREC, FIELD, TAU>(p2, ra, F2(lag.x, lag.y), k, seed_of(), oa);
    const F2 tb = pair_words<PREC, FIELD, TAU>(p2, rb, F2(lag.z, lag.w), k + 2, seed_of(), ob);
#pragma unroll
    for (int q = 0; q < 14; q++) *reinterpret_cast<uint2 *>(dst + q * P + k) = make_uint2(oa[q], ob[q]);
    if constexpr (TAU == 0) *reinterpret_cast<float4 *>(tdst + k) = make_float4(ta.v.x, ta.v.y, tb.v.x, tb.v.y);
    if (x0 == 0) step_node<PREC, float, FIELD, TAU>(src, dst, tsrc, tdst, p, 0, y, seed_of());
    if (x0 + 3 == p.nx - 1) step_node<PREC, float, FIELD, TAU>(src, dst, tsrc, tdst, p, p.nx - 1, y, seed_of());
}

}  // namespace lbm
