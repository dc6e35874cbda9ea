// lbm_step.cuh -- bodies of the fused pull-scheme step: one node at a time
// (any precision) and a tile of two nodes per thread (FP32 arithmetic), used
// by the single-cavity kernels and by the batched sweep.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// Pull, collide and store one node (wall rules included).  TAU 0: the
// collision starts from the stored lagged tau and stores its new tau; TAU 1:
// from the node-local implicit tau, and no tau is read or written.  For the
// FP32-arithmetic storages the arithmetic runs on deviations from the rest
// state (DEV form of pull, macro and collide), which keeps the small
// per-step changes of a nearly steady state out of the rounding of O(1)
// population values; FP64 runs on full values (dev_form).
template <int PREC, class R, int FIELD = 2, int TAU = 0>
__device__ __forceinline__ void step_node(const typename Store<PREC>::S *__restrict__ src,
                                          typename Store<PREC>::S *__restrict__ dst,
                                          const typename Store<PREC>::TauS *__restrict__ tsrc,
                                          typename Store<PREC>::TauS *__restrict__ tdst, const Phys<R> &p, int x,
                                          int y)
{
    using St = Store<PREC>;
    const int64_t k = (int64_t)y * p.pitch + x;
    R f[9], g[5];
    constexpr int DEV = dev_form<PREC>();
    pull<PREC, R, false, DEV>(src, p, x, y, f, g);
    Macro<R> m;
    const R t0 = tau_start<TAU, R, FIELD, DEV>(p, f, g, k, [&] { return R(tsrc[k]); });
    const R tau = collide<R, FIELD, DEV>(p, f, g, t0, m, k);
    uint32_t rng = rng_init(p.seed, k);   // random bits of the stochastic-rounding storages
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
// is uniform per warp.  TAU as for step_node.
template <int PREC, int FIELD = 2, int TAU = 0>
__device__ __forceinline__ void step2_tile(const typename Store<PREC>::S *__restrict__ src,
                                           typename Store<PREC>::S *__restrict__ dst,
                                           const float *__restrict__ tsrc, float *__restrict__ tdst,
                                           const Phys<float> &p, const Phys<F2> &p2, int xbase, int y)
{
    using St = Store<PREC>;
    using S = typename St::S;
    const int lane = threadIdx.x & 31;
    const int x0 = xbase + 2 * threadIdx.x;
    const int wx = xbase + 2 * (threadIdx.x & ~31);
    const bool fast = y > 0 && y < p.ny - 1 && wx > 0 && wx + 64 < p.nx;
    if (!fast) {
        for (int j = 0; j < 2; j++)
            if (x0 + j < p.nx) step_node<PREC, float, FIELD, TAU>(src, dst, tsrc, tdst, p, x0 + j, y);
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
    uint32_t rng = rng_init(p.seed, k);
#pragma unroll
    for (int i = 0; i < 9; i++) St::sdv2(dst + i * P, k, f[i], float(rest_f(i)), rng);
#pragma unroll
    for (int i = 0; i < 5; i++) St::sdv2(dst + (9 + i) * P, k, g[i], float(rest_g(i)), rng);
    if constexpr (TAU == 0) *reinterpret_cast<float2 *>(tdst + k) = tau.v;
}

}  // namespace lbm
