// lbm_aa.cu -- in-place (AA-pattern) streaming: one buffer instead of two.
//
// The single array A holds, per node x and direction i, one population; its
// meaning alternates between two forms:
//   form E (after an even step, and at start): A[opp(i)][x] = f*_i(x), the
//     post-collision population of node x moving along e_i;
//   form O (after an odd step): A[i][x] = f_i(x), the population that has
//     arrived at x and enters its next collision.
// Even step (O -> E): each node reads its own slots i, collides and writes
//   f*_i into its own slot opp(i).  No neighbour is touched.
// Odd step (E -> O): each node gathers f_i(x) = f*_i(x - e_i) from slot
//   opp(i) of node x - e_i (its own slot i across a wall, with the thermal
//   wall rules), collides and pushes f*_i(x) into slot i of node x + e_i;
//   a link that leaves the cavity writes the returning population into the
//   node's own slot opp(i) (bounce-back; anti-bounce-back -g* + 2 w T_w on
//   the isothermal walls).
// Every slot a step writes is one the same node read in that step, so the
// update is race-free in place.  The bytes moved per node update are the
// same as with two buffers; the footprint is halved.
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

// Push node (x, y)'s post-collision populations for the odd step.
template <int PREC, class R>
__device__ __forceinline__ void push(typename Store<PREC>::S *__restrict__ A, const Phys<R> &p, int x, int y,
                                     const R f[9], const R g[5])
{
    using St = Store<PREC>;
    const int64_t P = p.plane, W = p.pitch;
    const int64_t k = (int64_t)y * W + x;
    const bool xl = x > 0, xr = x < p.nx - 1, yb = y > 0, yt = y < p.ny - 1;
    uint32_t rng = rng_init(p.seed, k);   // random bits of the stochastic-rounding storages
    // target x + e_i: e1 (1,0) e2 (0,1) e3 (-1,0) e4 (0,-1) e5 (1,1) e6 (-1,1) e7 (-1,-1) e8 (1,-1)
    stf<PREC>(A, 0 * P + k, f[0], R(rest_f(0)), rng);
    if (xr) stf<PREC>(A, 1 * P + k + 1, f[1], R(rest_f(1)), rng); else stf<PREC>(A, 3 * P + k, f[1], R(rest_f(3)), rng);
    if (yt) stf<PREC>(A, 2 * P + k + W, f[2], R(rest_f(2)), rng); else stf<PREC>(A, 4 * P + k, f[2], R(rest_f(4)), rng);
    if (xl) stf<PREC>(A, 3 * P + k - 1, f[3], R(rest_f(3)), rng); else stf<PREC>(A, 1 * P + k, f[3], R(rest_f(1)), rng);
    if (yb) stf<PREC>(A, 4 * P + k - W, f[4], R(rest_f(4)), rng); else stf<PREC>(A, 2 * P + k, f[4], R(rest_f(2)), rng);
    if (xr && yt) stf<PREC>(A, 5 * P + k + W + 1, f[5], R(rest_f(5)), rng); else stf<PREC>(A, 7 * P + k, f[5], R(rest_f(7)), rng);
    if (xl && yt) stf<PREC>(A, 6 * P + k + W - 1, f[6], R(rest_f(6)), rng); else stf<PREC>(A, 8 * P + k, f[6], R(rest_f(8)), rng);
    if (xl && yb) stf<PREC>(A, 7 * P + k - W - 1, f[7], R(rest_f(7)), rng); else stf<PREC>(A, 5 * P + k, f[7], R(rest_f(5)), rng);
    if (xr && yb) stf<PREC>(A, 8 * P + k - W + 1, f[8], R(rest_f(8)), rng); else stf<PREC>(A, 6 * P + k, f[8], R(rest_f(6)), rng);
    typename Store<PREC>::S *G = A + 9 * P;
    stf<PREC>(G, 0 * P + k, g[0], R(rest_g(0)), rng);
    if (xr) stf<PREC>(G, 1 * P + k + 1, g[1], R(rest_g(1)), rng); else stf<PREC>(G, 3 * P + k, (dev_form<PREC>() ? p.abbd_cold : p.abb_cold) - g[1], R(rest_g(3)), rng);
    if (yt) stf<PREC>(G, 2 * P + k + W, g[2], R(rest_g(2)), rng); else stf<PREC>(G, 4 * P + k, g[2], R(rest_g(4)), rng);
    if (xl) stf<PREC>(G, 3 * P + k - 1, g[3], R(rest_g(3)), rng); else stf<PREC>(G, 1 * P + k, (dev_form<PREC>() ? p.abbd_hot : p.abb_hot) - g[3], R(rest_g(1)), rng);
    if (yb) stf<PREC>(G, 4 * P + k - W, g[4], R(rest_g(4)), rng); else stf<PREC>(G, 2 * P + k, g[4], R(rest_g(2)), rng);
}

// ------------------------------------------------------- one node / thread
template <int PREC, int TAU, int FIELD>
__global__ void __launch_bounds__(128)
aa_even_kernel(typename Store<PREC>::S *__restrict__ A, typename Store<PREC>::TauS *__restrict__ tau,
               Phys<typename Store<PREC>::R> p)
{
    using St = Store<PREC>;
    using R = typename St::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= p.nx) return;
    const int64_t P = p.plane, k = (int64_t)y * p.pitch + x;
    R f[9], g[5];
#pragma unroll
    for (int i = 0; i < 9; i++) f[i] = ldf<PREC>(A, i * P + k, R(rest_f(i)));
#pragma unroll
    for (int i = 0; i < 5; i++) g[i] = ldf<PREC>(A + 9 * P, i * P + k, R(rest_g(i)));
    Macro<R> m;
    constexpr int DEV = dev_form<PREC>();
    const R t = collide<R, FIELD, DEV>(p, f, g, tau_start<TAU, R, FIELD, DEV>(p, f, g, k, [&] { return R(tau[k]); }), m, k);
    uint32_t rng = rng_init(p.seed, k);
#pragma unroll
    for (int i = 0; i < 9; i++) stf<PREC>(A, opp(i) * P + k, f[i], R(rest_f(opp(i))), rng);
#pragma unroll
    for (int i = 0; i < 5; i++) stf<PREC>(A + 9 * P, opp(i) * P + k, g[i], R(rest_g(opp(i))), rng);
    if constexpr (TAU == 0) tau[k] = typename St::TauS(t);
}

template <int PREC, class R, int TAU, int FIELD>
__device__ __forceinline__ void odd_node(typename Store<PREC>::S *__restrict__ A,
                                         typename Store<PREC>::TauS *__restrict__ tau, const Phys<R> &p, int x,
                                         int y)
{
    const int64_t k = (int64_t)y * p.pitch + x;
    R f[9], g[5];
    constexpr int DEV = dev_form<PREC>();
    pull<PREC, R, true, DEV>(A, p, x, y, f, g);
    Macro<R> m;
    const R t = collide<R, FIELD, DEV>(p, f, g, tau_start<TAU, R, FIELD, DEV>(p, f, g, k, [&] { return R(tau[k]); }), m, k);
    push<PREC, R>(A, p, x, y, f, g);
    if constexpr (TAU == 0) tau[k] = typename Store<PREC>::TauS(t);
}

template <int PREC, int TAU, int FIELD>
__global__ void __launch_bounds__(128)
aa_odd_kernel(typename Store<PREC>::S *__restrict__ A, typename Store<PREC>::TauS *__restrict__ tau,
              Phys<typename Store<PREC>::R> p)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= p.nx) return;
    odd_node<PREC, typename Store<PREC>::R, TAU, FIELD>(A, tau, p, x, y);
}

// ------------------------------------------------------ two nodes / thread
template <int PREC, int TAU, int FIELD>
__global__ void __launch_bounds__(128)
aa_even2_kernel(typename Store<PREC>::S *__restrict__ A, float *__restrict__ tau, Phys<float> p, Phys<F2> p2)
{
    using St = Store<PREC>;
    const int x0 = (blockIdx.x * 128 + threadIdx.x) * 2, y = blockIdx.y;
    if (x0 >= p.nx) return;
    const int64_t P = p.plane, k = (int64_t)y * p.pitch + x0;
    if (x0 + 1 >= p.nx) {   // ragged end of the row: one node
        float f[9], g[5];
        for (int i = 0; i < 9; i++) f[i] = St::ldd(A, i * P + k, float(rest_f(i)));
        for (int i = 0; i < 5; i++) g[i] = St::ldd(A + 9 * P, i * P + k, float(rest_g(i)));
        Macro<float> m;
        const float t =
            collide<float, FIELD, 1>(p, f, g, tau_start<TAU, float, FIELD, 1>(p, f, g, k, [&] { return tau[k]; }), m, k);
        uint32_t rng = rng_init(p.seed, k);
        for (int i = 0; i < 9; i++) St::sdv(A, opp(i) * P + k, f[i], float(rest_f(opp(i))), rng);
        for (int i = 0; i < 5; i++) St::sdv(A + 9 * P, opp(i) * P + k, g[i], float(rest_g(opp(i))), rng);
        if constexpr (TAU == 0) tau[k] = t;
        return;
    }
    F2 f[9], g[5];
#pragma unroll
    for (int i = 0; i < 9; i++) f[i] = St::ldd2(A + i * P, k, float(rest_f(i)));
#pragma unroll
    for (int i = 0; i < 5; i++) g[i] = St::ldd2(A + (9 + i) * P, k, float(rest_g(i)));
    Macro<F2> m;
    const F2 t0 = tau_start<TAU, F2, FIELD, 1>(p2, f, g, k, [&] { return F2(*reinterpret_cast<const float2 *>(tau + k)); });
    const F2 t = collide<F2, FIELD, 1>(p2, f, g, t0, m, k);
    uint32_t rng = rng_init(p2.seed, k);
#pragma unroll
    for (int i = 0; i < 9; i++) St::sdv2(A + opp(i) * P, k, f[i], float(rest_f(opp(i))), rng);
#pragma unroll
    for (int i = 0; i < 5; i++) St::sdv2(A + (9 + opp(i)) * P, k, g[i], float(rest_g(opp(i))), rng);
    if constexpr (TAU == 0) *reinterpret_cast<float2 *>(tau + k) = t.v;
}

// Odd-step pushes of a pair (nodes x0, x0 + 1) one node to the right / left
// within one row of a plane; the aligned pair at x0 is assembled with a warp
// shuffle, and the lanes at the warp's ends store the element that belongs
// to the neighbouring warp's pair on their own.
template <int PREC>
__device__ __forceinline__ void push_right(typename Store<PREC>::S *base, int64_t kr, F2 v, float rest, int lane,
                                           uint32_t &rng)
{
    using St = Store<PREC>;
    const float prev = __shfl_up_sync(0xffffffffu, v.v.y, 1);
    if (lane != 0) St::sdv2(base, kr, F2(prev, v.v.x), rest, rng);
    else St::sdv(base, kr + 1, v.v.x, rest, rng);
    if (lane == 31) St::sdv(base, kr + 2, v.v.y, rest, rng);
}
template <int PREC>
__device__ __forceinline__ void push_left(typename Store<PREC>::S *base, int64_t kr, F2 v, float rest, int lane,
                                          uint32_t &rng)
{
    using St = Store<PREC>;
    const float next = __shfl_down_sync(0xffffffffu, v.v.x, 1);
    if (lane != 31) St::sdv2(base, kr, F2(v.v.y, next), rest, rng);
    else St::sdv(base, kr, v.v.y, rest, rng);
    if (lane == 0) St::sdv(base, kr - 1, v.v.x, rest, rng);
}

template <int PREC, int TAU, int FIELD>
__global__ void __launch_bounds__(128)
aa_odd2_kernel(typename Store<PREC>::S *__restrict__ A, float *__restrict__ tau, Phys<float> p, Phys<F2> p2)
{
    using St = Store<PREC>;
    using S = typename St::S;
    const int lane = threadIdx.x & 31;
    const int x0 = (blockIdx.x * 128 + threadIdx.x) * 2, y = blockIdx.y;
    const int wx = (blockIdx.x * 128 + (threadIdx.x & ~31)) * 2;
    const bool fast = y > 0 && y < p.ny - 1 && wx > 0 && wx + 64 < p.nx;
    if (!fast) {
        for (int j = 0; j < 2; j++)
            if (x0 + j < p.nx) odd_node<PREC, float, TAU, FIELD>(A, tau, p, x0 + j, y);
        return;
    }
    const int64_t P = p.plane, W = p.pitch;
    const int64_t k = (int64_t)y * W + x0;
    S *fs = A;
    S *gs = A + 9 * P;
    const bool l0 = lane == 0, l31 = lane == 31;
    // gather f_i(x) = f*_i(x - e_i), kept in slot opp(i) of node x - e_i
    F2 f[9], g[5];
    f[0] = St::ldd2(fs, k, float(rest_f(0)));
    f[1] = from_left(St::ldd2(fs + 3 * P, k, float(rest_f(3))), l0 ? St::ldd(fs + 3 * P, k - 1, float(rest_f(3))) : 0.f, lane);
    f[2] = St::ldd2(fs + 4 * P, k - W, float(rest_f(4)));
    f[3] = from_right(St::ldd2(fs + P, k, float(rest_f(1))), l31 ? St::ldd(fs + P, k + 2, float(rest_f(1))) : 0.f, lane);
    f[4] = St::ldd2(fs + 2 * P, k + W, float(rest_f(2)));
    f[5] = from_left(St::ldd2(fs + 7 * P, k - W, float(rest_f(7))),
                     l0 ? St::ldd(fs + 7 * P, k - W - 1, float(rest_f(7))) : 0.f, lane);
    f[6] = from_right(St::ldd2(fs + 8 * P, k - W, float(rest_f(8))),
                      l31 ? St::ldd(fs + 8 * P, k - W + 2, float(rest_f(8))) : 0.f, lane);
    f[7] = from_right(St::ldd2(fs + 5 * P, k + W, float(rest_f(5))),
                      l31 ? St::ldd(fs + 5 * P, k + W + 2, float(rest_f(5))) : 0.f, lane);
    f[8] = from_left(St::ldd2(fs + 6 * P, k + W, float(rest_f(6))),
                     l0 ? St::ldd(fs + 6 * P, k + W - 1, float(rest_f(6))) : 0.f, lane);
    g[0] = St::ldd2(gs, k, float(rest_g(0)));
    g[1] = from_left(St::ldd2(gs + 3 * P, k, float(rest_g(3))), l0 ? St::ldd(gs + 3 * P, k - 1, float(rest_g(3))) : 0.f, lane);
    g[2] = St::ldd2(gs + 4 * P, k - W, float(rest_g(4)));
    g[3] = from_right(St::ldd2(gs + P, k, float(rest_g(1))), l31 ? St::ldd(gs + P, k + 2, float(rest_g(1))) : 0.f, lane);
    g[4] = St::ldd2(gs + 2 * P, k + W, float(rest_g(2)));
    Macro<F2> m;
    const F2 t0 = tau_start<TAU, F2, FIELD, 1>(p2, f, g, k, [&] { return F2(*reinterpret_cast<const float2 *>(tau + k)); });
    const F2 t = collide<F2, FIELD, 1>(p2, f, g, t0, m, k);
    uint32_t rng = rng_init(p2.seed, k);
    // push f*_i(x) into slot i of node x + e_i
    St::sdv2(fs, k, f[0], float(rest_f(0)), rng);
    push_right<PREC>(fs + P, k, f[1], float(rest_f(1)), lane, rng);
    St::sdv2(fs + 2 * P, k + W, f[2], float(rest_f(2)), rng);
    push_left<PREC>(fs + 3 * P, k, f[3], float(rest_f(3)), lane, rng);
    St::sdv2(fs + 4 * P, k - W, f[4], float(rest_f(4)), rng);
    push_right<PREC>(fs + 5 * P, k + W, f[5], float(rest_f(5)), lane, rng);
    push_left<PREC>(fs + 6 * P, k + W, f[6], float(rest_f(6)), lane, rng);
    push_left<PREC>(fs + 7 * P, k - W, f[7], float(rest_f(7)), lane, rng);
    push_right<PREC>(fs + 8 * P, k - W, f[8], float(rest_f(8)), lane, rng);
    St::sdv2(gs, k, g[0], float(rest_g(0)), rng);
    push_right<PREC>(gs + P, k, g[1], float(rest_g(1)), lane, rng);
    St::sdv2(gs + 2 * P, k + W, g[2], float(rest_g(2)), rng);
    push_left<PREC>(gs + 3 * P, k, g[3], float(rest_g(3)), lane, rng);
    St::sdv2(gs + 4 * P, k - W, g[4], float(rest_g(4)), rng);
    if constexpr (TAU == 0) *reinterpret_cast<float2 *>(tau + k) = t.v;
}

// Odd step for a uniform permeability: lane l of each warp updates nodes
// wx + l and wx + 32 + l (wx: the warp's first of 64 nodes) as one packed
// pair.  Every population row is then read and written by coalesced
// 32-node accesses, shifted by one element for the x-moving populations,
// with no warp shuffles and no warp-end special cases -- which adjacent pairs
// need on both the gathers and the pushes of the odd step.  The per-node
// Darcy field keeps aa_odd2_kernel (its loads take adjacent pairs).
template <int PREC, int TAU>
__global__ void __launch_bounds__(128)
aa_odd_split_kernel(typename Store<PREC>::S *__restrict__ A, float *__restrict__ tau, Phys<float> p, Phys<F2> p2)
{
    using St = Store<PREC>;
    using S = typename St::S;
    const int lane = threadIdx.x & 31;
    const int wx = blockIdx.x * 256 + (threadIdx.x >> 5) * 64, y = blockIdx.y;
    const int xa = wx + lane;
    const bool fast = y > 0 && y < p.ny - 1 && wx > 0 && wx + 64 < p.nx;
    if (!fast) {
        if (xa < p.nx) odd_node<PREC, float, TAU, 0>(A, tau, p, xa, y);
        if (xa + 32 < p.nx) odd_node<PREC, float, TAU, 0>(A, tau, p, xa + 32, y);
        return;
    }
    const int64_t P = p.plane, W = p.pitch;
    const int64_t k = (int64_t)y * W + xa;   // node a; node b is k + 32
    S *fs = A;
    S *gs = A + 9 * P;
    auto gather = [&](const S *plane, int64_t off, double rest) {
        return F2(St::ldd(plane, k + off, float(rest)), St::ldd(plane, k + 32 + off, float(rest)));
    };
    // gather f_i(x) = f*_i(x - e_i), kept in slot opp(i) of node x - e_i
    F2 f[9], g[5];
    f[0] = gather(fs, 0, rest_f(0));
    f[1] = gather(fs + 3 * P, -1, rest_f(3));
    f[2] = gather(fs + 4 * P, -W, rest_f(4));
    f[3] = gather(fs + P, 1, rest_f(1));
    f[4] = gather(fs + 2 * P, W, rest_f(2));
    f[5] = gather(fs + 7 * P, -W - 1, rest_f(7));
    f[6] = gather(fs + 8 * P, -W + 1, rest_f(8));
    f[7] = gather(fs + 5 * P, W + 1, rest_f(5));
    f[8] = gather(fs + 6 * P, W - 1, rest_f(6));
    g[0] = gather(gs, 0, rest_g(0));
    g[1] = gather(gs + 3 * P, -1, rest_g(3));
    g[2] = gather(gs + 4 * P, -W, rest_g(4));
    g[3] = gather(gs + P, 1, rest_g(1));
    g[4] = gather(gs + 2 * P, W, rest_g(2));
    Macro<F2> m;
    const F2 t0 = tau_start<TAU, F2, 0, 1>(p2, f, g, k, [&] { return F2(tau[k], tau[k + 32]); });
    const F2 t = collide<F2, 0, 1>(p2, f, g, t0, m, k);
    uint32_t rng = rng_init(p2.seed, k);
    // push f*_i(x) into slot i of node x + e_i
    auto push = [&](S *plane, int64_t off, F2 v, double rest) {
        St::sdv(plane, k + off, v.v.x, float(rest), rng);
        St::sdv(plane, k + 32 + off, v.v.y, float(rest), rng);
    };
    push(fs, 0, f[0], rest_f(0));
    push(fs + P, 1, f[1], rest_f(1));
    push(fs + 2 * P, W, f[2], rest_f(2));
    push(fs + 3 * P, -1, f[3], rest_f(3));
    push(fs + 4 * P, -W, f[4], rest_f(4));
    push(fs + 5 * P, W + 1, f[5], rest_f(5));
    push(fs + 6 * P, W - 1, f[6], rest_f(6));
    push(fs + 7 * P, -W - 1, f[7], rest_f(7));
    push(fs + 8 * P, -W + 1, f[8], rest_f(8));
    push(gs, 0, g[0], rest_g(0));
    push(gs + P, 1, g[1], rest_g(1));
    push(gs + 2 * P, W, g[2], rest_g(2));
    push(gs + 3 * P, -1, g[3], rest_g(3));
    push(gs + 4 * P, -W, g[4], rest_g(4));
    if constexpr (TAU == 0) {
        tau[k] = t.v.x;
        tau[k + 32] = t.v.y;
    }
}

// Form O -> form E in place, without a collision: each interior link
// (x, x + e_i), i in {1, 2, 5, 6} (one of each opposite pair), swaps slot i of
// x + e_i with slot opp(i) of x; a thermal link that left through an
// isothermal wall turns its stored -g*_i + 2 w T_w back into g*_i.  Every slot
// belongs to exactly one such link.
template <int PREC>
__global__ void __launch_bounds__(128)
aa_normalize_kernel(typename Store<PREC>::S *__restrict__ A, Phys<typename Store<PREC>::R> p)
{
    using St = Store<PREC>;
    using R = typename St::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= p.nx) return;
    const int64_t P = p.plane, W = p.pitch, k = (int64_t)y * W + x;
    const bool xl = x > 0, xr = x < p.nx - 1, yt = y < p.ny - 1;
    // opposite directions have equal weights, so the stored representation
    // (value or deviation) moves between the two slots unchanged
    auto swap = [&](typename Store<PREC>::S *base, int i, int64_t kt, bool) {
        const typename Store<PREC>::S a = base[i * P + kt];
        base[i * P + kt] = base[opp(i) * P + k];
        base[opp(i) * P + k] = a;
    };
    if (xr) swap(A, 1, k + 1, true);
    if (yt) swap(A, 2, k + W, true);
    if (xr && yt) swap(A, 5, k + W + 1, true);
    if (xl && yt) swap(A, 6, k + W - 1, true);
    typename Store<PREC>::S *G = A + 9 * P;
    if (xr) swap(G, 1, k + 1, false);
    if (yt) swap(G, 2, k + W, false);
    uint32_t rng = rng_init(p.seed, k);
    if (!xl) St::sdv(G, 1 * P + k, p.abbd_hot - St::ldd(G, 1 * P + k, R(rest_g(1))), R(rest_g(1)), rng);
    if (!xr) St::sdv(G, 3 * P + k, p.abbd_cold - St::ldd(G, 3 * P + k, R(rest_g(3))), R(rest_g(3)), rng);
}

// ------------------------------------------------------------- launchers
template <int PREC, int TAU, int FIELD>
static void aa_launch(lbm_ctx *c)
{
    using St = Store<PREC>;
    auto *A = (typename St::S *)c->buf.dist[0];
    if constexpr (PREC == LBM_F64) {
        const dim3 grid((c->nx + 127) / 128, c->ny);
        if (c->aa_form_o)
            aa_even_kernel<PREC, TAU, FIELD><<<grid, 128, 0, c->stream>>>(A, (double *)c->buf.tau[0],
                                                                 make_params<double>(c));
        else
            aa_odd_kernel<PREC, TAU, FIELD><<<grid, 128, 0, c->stream>>>(A, (double *)c->buf.tau[0],
                                                                make_params<double>(c));
    } else {
        const dim3 grid((c->nx + 255) / 256, c->ny);
        if (c->aa_form_o)
            aa_even2_kernel<PREC, TAU, FIELD><<<grid, 128, 0, c->stream>>>(A, (float *)c->buf.tau[0],
                                                                  make_params<float>(c), make_params<F2>(c));
        else if constexpr (FIELD == 0)
            aa_odd_split_kernel<PREC, TAU><<<grid, 128, 0, c->stream>>>(A, (float *)c->buf.tau[0],
                                                               make_params<float>(c), make_params<F2>(c));
        else
            aa_odd2_kernel<PREC, TAU, FIELD><<<grid, 128, 0, c->stream>>>(A, (float *)c->buf.tau[0],
                                                                 make_params<float>(c), make_params<F2>(c));
    }
}

template <int PREC>
static cudaError_t aa_step_t(lbm_ctx *c)
{
    const bool field = c->d_da != nullptr;
    if (c->opts.tau_iters > 0)
        field ? aa_launch<PREC, 1, 1>(c) : aa_launch<PREC, 1, 0>(c);
    else
        field ? aa_launch<PREC, 0, 1>(c) : aa_launch<PREC, 0, 0>(c);
    c->aa_form_o = !c->aa_form_o;
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t aa_normalize_t(lbm_ctx *c)
{
    using St = Store<PREC>;
    if (!c->aa_form_o) return cudaSuccess;
    const dim3 grid((c->nx + 127) / 128, c->ny);
    aa_normalize_kernel<PREC><<<grid, 128, 0, c->stream>>>((typename St::S *)c->buf.dist[0],
                                                          make_params<typename St::R>(c));
    c->aa_form_o = false;
    return cudaGetLastError();
}

#define LBM_DISPATCH(fn, ...)                                      \
    switch (c->opts.prec) {                                        \
    case LBM_F64: return fn<LBM_F64>(__VA_ARGS__);                 \
    case LBM_F32: return fn<LBM_F32>(__VA_ARGS__);                 \
    case LBM_BF16D: return fn<LBM_BF16D>(__VA_ARGS__);             \
    case LBM_F16D: return fn<LBM_F16D>(__VA_ARGS__);               \
    case LBM_F32D: return fn<LBM_F32D>(__VA_ARGS__);               \
    case LBM_F16S: return fn<LBM_F16S>(__VA_ARGS__);               \
    case LBM_BF16S: return fn<LBM_BF16S>(__VA_ARGS__);             \
    default: return cudaErrorInvalidValue;                         \
    }

cudaError_t launch_aa_step(lbm_ctx *c) { LBM_DISPATCH(aa_step_t, c) }
cudaError_t launch_aa_normalize(lbm_ctx *c) { LBM_DISPATCH(aa_normalize_t, c) }

}  // namespace lbm
