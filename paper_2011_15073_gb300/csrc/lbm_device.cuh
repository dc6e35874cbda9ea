// lbm_device.cuh -- device-side physics of the fused MRT step (sm_103a).
//
// Closed-form moment transforms: the D2Q9 basis rows are mutually orthogonal,
// so M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4) and the
// D2Q5 N^-1 = N^T diag(1/5, 1/2, 1/2, 1/20, 1/4); every product below is
// written out with those integer coefficients instead of a matrix multiply.
// The strain-rate double sum of the power-law section collapses to the three
// non-equilibrium moments that carry second velocity moments (e, p_xx, p_xy).
//
// The node physics is written once over a value type V:
//   double -- FP64 arithmetic (IEEE division, square root and pow);
//   float  -- FP32 arithmetic with the approximate special-function unit
//             (rcp/sqrt/ex2/lg2 .approx, about 1-2 ulp);
//   F2     -- two nodes in one register pair, the arithmetic on the packed
//             FP32x2 pipe (fma/add/mul .f32x2) and the special functions
//             per lane as for float.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

#include "lbm_internal.h"
#include "lbm_round.cuh"

namespace lbm {

// ------------------------------------------------------------ packed FP32x2
struct F2 {
    float2 v;
    __host__ __device__ F2() {}
    __host__ __device__ F2(float a) : v(make_float2(a, a)) {}
    __host__ __device__ F2(double a) : v(make_float2((float)a, (float)a)) {}
    __host__ __device__ F2(int a) : v(make_float2((float)a, (float)a)) {}
    __host__ __device__ F2(float a, float b) : v(make_float2(a, b)) {}
    __host__ __device__ explicit F2(float2 w) : v(w) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b)
{
    return F2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v));  // exact: b * -1 is exact
}
__device__ __forceinline__ F2 operator-(F2 a) { return F2(__fmul2_rn(a.v, make_float2(-1.f, -1.f))); }

__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }

// Special functions.
__device__ __forceinline__ double vrcp(double x) { return 1.0 / x; }
__device__ __forceinline__ double vsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ double vpow(double x, double e) { return pow(x, e); }

__device__ __forceinline__ float vrcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float vsqrt(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float vexp2(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float vpow(float x, float e) { return vexp2(e * __log2f(x)); }

__device__ __forceinline__ F2 vrcp(F2 a) { return F2(vrcp(a.v.x), vrcp(a.v.y)); }
__device__ __forceinline__ F2 vsqrt(F2 a) { return F2(vsqrt(a.v.x), vsqrt(a.v.y)); }

// Per-case constants in the compute type V (built on the host from
// lbm_lattice by make_params below).
template <class V>
struct Phys {
    int nx, ny;
    int64_t pitch;   // elements between rows of a plane
    int64_t plane;   // elements between planes
    V nu_ref, gamma_scale, gamma1, gamma2, nm1, D_hi;
    int clamp_mode;
    V eps, half_eps, inv_eps;
    V half_eps_invK;   // eps / (4 K): c0 = 1/2 + half_eps_invK * nu
    V eps_invK;        // eps / K
    V c1;              // eps F_eps / (2 sqrt K)
    V eFe_isqK;        // eps F_eps / sqrt K
    V gbeta, Tm;
    V omegaT, s_e, s_p;
    V abb_hot, abb_cold;   // 2 w T_wall for the anti-bounce-back (w = 1/6)
    V abbd_hot, abbd_cold; // the same on deviations from w T_m: 2 w (T_wall - T_m)
    // Per-node Darcy numbers (lbm_set_darcy_field), or null for the uniform
    // permeability above: a plane of the compute type (float for the F2
    // paths), indexed like the state planes; K = Da L2.
    const void *da;
    V L2, eFe;                 // L^2 and eps F_eps
    // Node-local implicit relaxation time (tau_iters > 0): Newton steps per
    // collision, their start tau0 and 3 nu_ref.
    int tau_iters;
    V tau0, nu3;
    // Seed of the stochastic rounding of this launch (a new one every step).
    uint32_t seed;
};

// ------------------------------------------------------------ parameters
// The stochastic rounding's seeds: run_word() turns lbm_opts.seed into the
// run's stream word (0 keeps the default stream), step_seed() gives the seed
// of the step that starts at step count `steps` of that run -- on the host
// for plain launches, on the device for the batched sweep, so a case steps
// with the same random bits either way.
__host__ __device__ __forceinline__ uint32_t run_word(uint64_t s)
{
    return s ? mix32((uint32_t)s ^ mix32((uint32_t)(s >> 32) + 0x68e31da4u)) : 0u;
}
__host__ __device__ __forceinline__ uint32_t step_seed(uint64_t steps, uint32_t run)
{
    return mix32(0x9e3779b9u * (uint32_t)(steps + 1) ^ (uint32_t)(steps >> 32) ^ run);
}

template <class V>
inline Phys<V> make_params(const lbm_ctx *c)
{
    const lbm_lattice &L = c->lat;
    Phys<V> p;
    p.nx = c->nx;
    p.ny = c->ny;
    p.pitch = c->pitch;
    p.plane = c->plane;
    p.nu_ref = V(L.nu_ref);
    p.gamma_scale = V(L.gamma_scale);
    p.gamma1 = V(L.gamma1);
    p.gamma2 = V(L.gamma2);
    p.nm1 = V(L.n - 1.0);
    p.D_hi = V(pow(L.gamma2, L.n - 1.0));
    p.clamp_mode = L.clamp_mode;
    p.eps = V(L.eps);
    p.half_eps = V(0.5 * L.eps);
    p.inv_eps = V(1.0 / L.eps);
    p.half_eps_invK = V(L.eps / (4.0 * L.K));
    p.eps_invK = V(L.eps / L.K);
    p.c1 = V(L.eps * L.Feps / (2.0 * sqrt(L.K)));
    p.eFe_isqK = V(L.eps * L.Feps / sqrt(L.K));
    p.gbeta = V(L.gbeta);
    p.Tm = V(L.Tm);
    p.omegaT = V(1.0 / L.tauT);
    p.s_e = V(L.s_e);
    p.s_p = V(L.s_p);
    p.abb_hot = V(2.0 / 6.0 * L.T_hot);
    p.abb_cold = V(2.0 / 6.0 * L.T_cold);
    p.abbd_hot = V(2.0 / 6.0 * (L.T_hot - L.Tm));
    p.abbd_cold = V(2.0 / 6.0 * (L.T_cold - L.Tm));
    p.da = c->d_da;
    p.L2 = V(L.L * L.L);
    p.eFe = V(L.eps * L.Feps);
    p.tau_iters = c->opts.tau_iters;
    p.tau0 = V(L.tau0);
    p.nu3 = V(3.0 * L.nu_ref);
    p.seed = step_seed((uint64_t)c->steps, run_word(c->opts.seed));
    return p;
}

// Rest-state values used by the deviation storage forms.
__host__ __device__ constexpr double rest_f(int i)
{
    return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
}
__host__ __device__ constexpr double rest_g(int i)  // w_i T_m with T_m = 1/2
{
    return i == 0 ? 1.0 / 6.0 : 1.0 / 12.0;
}

// ---------------------------------------------------------------- storage
// ld/st move one node's value; ld2/st2 move the aligned pair (k, k+1) as F2.
// The 16-bit storages also convert a pair held as one 32-bit word (the lower
// node in the low half): unpack2 -> the two deviations, pack2 <- them (the
// stochastic-rounding ones draw their random bits from rng).  ldd2/sdv2 are
// written with them, so every path converts a pair the same way.
__device__ __forceinline__ __half2 as_h2(uint32_t u)
{
    __half2 h;
    memcpy(&h, &u, 4);
    return h;
}
__device__ __forceinline__ __nv_bfloat162 as_bf162(uint32_t u)
{
    __nv_bfloat162 h;
    memcpy(&h, &u, 4);
    return h;
}
template <class H2>
__device__ __forceinline__ uint32_t as_u32(H2 h)
{
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}

template <int PREC>
struct Store;

template <>
struct Store<LBM_F64> {
    using S = double;
    using R = double;
    using TauS = double;
    static __device__ __forceinline__ R ld(const S *p, int64_t k, R) { return p[k]; }
    static __device__ __forceinline__ void st(S *p, int64_t k, R v, R, uint32_t = 0) { p[k] = v; }
    static __device__ __forceinline__ R ldd(const S *p, int64_t k, R rest) { return p[k] - rest; }
    static __device__ __forceinline__ void sdv(S *p, int64_t k, R d, R rest, uint32_t &) { p[k] = d + rest; }
};
template <>
struct Store<LBM_F32> {
    using S = float;
    using R = float;
    using TauS = float;
    static __device__ __forceinline__ R ld(const S *p, int64_t k, R) { return p[k]; }
    static __device__ __forceinline__ void st(S *p, int64_t k, R v, R, uint32_t = 0) { p[k] = v; }
    static __device__ __forceinline__ R ldd(const S *p, int64_t k, R rest) { return p[k] - rest; }
    static __device__ __forceinline__ void sdv(S *p, int64_t k, R d, R rest, uint32_t &) { p[k] = d + rest; }
    static __device__ __forceinline__ F2 ldd2(const S *p, int64_t k, float rest)
    {
        return F2(*reinterpret_cast<const float2 *>(p + k)) - F2(rest);
    }
    static __device__ __forceinline__ void sdv2(S *p, int64_t k, F2 d, float rest, uint32_t &)
    {
        *reinterpret_cast<float2 *>(p + k) = (d + F2(rest)).v;
    }
    static __device__ __forceinline__ F2 ld2(const S *p, int64_t k, float)
    {
        return F2(*reinterpret_cast<const float2 *>(p + k));
    }
    static __device__ __forceinline__ void st2(S *p, int64_t k, F2 v, float, uint32_t = 0)
    {
        *reinterpret_cast<float2 *>(p + k) = v.v;
    }
};
template <>
struct Store<LBM_F32D> {
    using S = float;
    using R = float;
    using TauS = float;
    static __device__ __forceinline__ R ld(const S *p, int64_t k, R rest) { return rest + p[k]; }
    static __device__ __forceinline__ void st(S *p, int64_t k, R v, R rest, uint32_t = 0) { p[k] = v - rest; }
    static __device__ __forceinline__ F2 ld2(const S *p, int64_t k, float rest)
    {
        return F2(*reinterpret_cast<const float2 *>(p + k)) + F2(rest);
    }
    static __device__ __forceinline__ void st2(S *p, int64_t k, F2 v, float rest, uint32_t = 0)
    {
        *reinterpret_cast<float2 *>(p + k) = (v - F2(rest)).v;
    }
    static __device__ __forceinline__ R ldd(const S *p, int64_t k, R) { return p[k]; }
    static __device__ __forceinline__ void sdv(S *p, int64_t k, R d, R, uint32_t &) { p[k] = d; }
    static __device__ __forceinline__ F2 ldd2(const S *p, int64_t k, float)
    {
        return F2(*reinterpret_cast<const float2 *>(p + k));
    }
    static __device__ __forceinline__ void sdv2(S *p, int64_t k, F2 d, float, uint32_t &)
    {
        *reinterpret_cast<float2 *>(p + k) = d.v;
    }
};
template <>
struct Store<LBM_BF16D> {
    using S = __nv_bfloat16;
    using R = float;
    using TauS = float;
    static __device__ __forceinline__ R ld(const S *p, int64_t k, R rest)
    {
        return rest + __bfloat162float(p[k]);
    }
    static __device__ __forceinline__ void st(S *p, int64_t k, R v, R rest, uint32_t = 0)
    {
        p[k] = __float2bfloat16_rn(v - rest);
    }
    static __device__ __forceinline__ F2 ld2(const S *p, int64_t k, float rest)
    {
        const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(p + k);
        return F2(__bfloat1622float2(h)) + F2(rest);
    }
    static __device__ __forceinline__ void st2(S *p, int64_t k, F2 v, float rest, uint32_t = 0)
    {
        *reinterpret_cast<__nv_bfloat162 *>(p + k) = __float22bfloat162_rn((v - F2(rest)).v);
    }
    static __device__ __forceinline__ R ldd(const S *p, int64_t k, R) { return __bfloat162float(p[k]); }
    static __device__ __forceinline__ void sdv(S *p, int64_t k, R d, R, uint32_t &) { p[k] = __float2bfloat16_rn(d); }
    static __device__ __forceinline__ F2 unpack2(uint32_t u) { return F2(__bfloat1622float2(as_bf162(u))); }
    static __device__ __forceinline__ uint32_t pack2(F2 d, uint32_t &) { return as_u32(__float22bfloat162_rn(d.v)); }
    static __device__ __forceinline__ F2 ldd2(const S *p, int64_t k, float)
    {
        return unpack2(*reinterpret_cast<const uint32_t *>(p + k));
    }
    static __device__ __forceinline__ void sdv2(S *p, int64_t k, F2 d, float, uint32_t &rng)
    {
        *reinterpret_cast<uint32_t *>(p + k) = pack2(d, rng);
    }
};
template <>
struct Store<LBM_F16D> {
    using S = __half;
    using R = float;
    using TauS = float;
    static __device__ __forceinline__ R ld(const S *p, int64_t k, R rest)
    {
        return rest + __half2float(p[k]);
    }
    static __device__ __forceinline__ void st(S *p, int64_t k, R v, R rest, uint32_t = 0)
    {
        p[k] = __float2half_rn(v - rest);
    }
    static __device__ __forceinline__ F2 ld2(const S *p, int64_t k, float rest)
    {
        const __half2 h = *reinterpret_cast<const __half2 *>(p + k);
        return F2(__half22float2(h)) + F2(rest);
    }
    static __device__ __forceinline__ void st2(S *p, int64_t k, F2 v, float rest, uint32_t = 0)
    {
        *reinterpret_cast<__half2 *>(p + k) = __float22half2_rn((v - F2(rest)).v);
    }
    static __device__ __forceinline__ R ldd(const S *p, int64_t k, R) { return __half2float(p[k]); }
    static __device__ __forceinline__ void sdv(S *p, int64_t k, R d, R, uint32_t &) { p[k] = __float2half_rn(d); }
    static __device__ __forceinline__ F2 unpack2(uint32_t u) { return F2(__half22float2(as_h2(u))); }
    static __device__ __forceinline__ uint32_t pack2(F2 d, uint32_t &) { return as_u32(__float22half2_rn(d.v)); }
    static __device__ __forceinline__ F2 ldd2(const S *p, int64_t k, float)
    {
        return unpack2(*reinterpret_cast<const uint32_t *>(p + k));
    }
    static __device__ __forceinline__ void sdv2(S *p, int64_t k, F2 d, float, uint32_t &rng)
    {
        *reinterpret_cast<uint32_t *>(p + k) = pack2(d, rng);
    }
};

// FP16 / BF16 deviation storage with stochastic rounding (lbm_round.cuh).
// The FP16 form stores the deviation scaled by 2^15, which moves deviations
// down to 2e-9 into the normal range of FP16 (and keeps |d| < 2 finite): a
// custom 16-bit format with the exponent range shifted to where the
// deviations live (below 2e-9, FP16's subnormals keep a spacing of 2^-39 in
// deviation units).  The rounding is the conversion's own stochastic mode
// (sr_half2, sr_bf16x2: one instruction per stored pair).  The kernels'
// random bits: rng_init() hashes the step's seed and the node once,
// then rng_next() advances a Weyl sequence by one add per stored pair (each
// draw is uniform because the start is; the pairs of one node share it).
// Import uses the element's address for its random bits.
constexpr float F16S_SCALE = 32768.0f, F16S_ISCALE = 1.0f / 32768.0f;
template <>
struct Store<LBM_F16S> {
    using S = __half;
    using R = float;
    using TauS = float;
    static __device__ __forceinline__ R ldd(const S *p, int64_t k, R) { return __half2float(p[k]) * F16S_ISCALE; }
    static __device__ __forceinline__ R ld(const S *p, int64_t k, R rest) { return rest + ldd(p, k, rest); }
    static __device__ __forceinline__ void st(S *p, int64_t k, R v, R rest, uint32_t seed = 0)
    {
        p[k] = sr_half((v - rest) * F16S_SCALE, sr_bits(seed, p + k));
    }
    static __device__ __forceinline__ F2 unpack2(uint32_t u) { return F2(__half22float2(as_h2(u))) * F2(F16S_ISCALE); }
    static __device__ __forceinline__ uint32_t pack2(F2 d, uint32_t &rng)
    {
        rng = rng_next(rng);
        const F2 ds = d * F2(F16S_SCALE);
        return sr_half2(ds.v.x, ds.v.y, rng);
    }
    static __device__ __forceinline__ F2 ldd2(const S *p, int64_t k, float)
    {
        return unpack2(*reinterpret_cast<const uint32_t *>(p + k));
    }
    static __device__ __forceinline__ F2 ld2(const S *p, int64_t k, float rest) { return ldd2(p, k, rest) + F2(rest); }
    static __device__ __forceinline__ void st2(S *p, int64_t k, F2 v, float rest, uint32_t seed = 0)
    {
        const F2 d = (v - F2(rest)) * F2(F16S_SCALE);
        *reinterpret_cast<uint32_t *>(p + k) = sr_half2(d.v.x, d.v.y, sr_bits(seed, p + k));
    }
    static __device__ __forceinline__ void sdv(S *p, int64_t k, R d, R, uint32_t &rng)
    {
        rng = rng_next(rng);
        p[k] = sr_half(d * F16S_SCALE, rng);
    }
    static __device__ __forceinline__ void sdv2(S *p, int64_t k, F2 d, float, uint32_t &rng)
    {
        *reinterpret_cast<uint32_t *>(p + k) = pack2(d, rng);
    }
};
template <>
struct Store<LBM_BF16S> {
    using S = __nv_bfloat16;
    using R = float;
    using TauS = float;
    static __device__ __forceinline__ R ld(const S *p, int64_t k, R rest)
    {
        return rest + __bfloat162float(p[k]);
    }
    static __device__ __forceinline__ void st(S *p, int64_t k, R v, R rest, uint32_t seed = 0)
    {
        p[k] = sr_bf16(v - rest, sr_bits(seed, p + k));
    }
    static __device__ __forceinline__ F2 ld2(const S *p, int64_t k, float rest)
    {
        const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(p + k);
        return F2(__bfloat1622float2(h)) + F2(rest);
    }
    static __device__ __forceinline__ void st2(S *p, int64_t k, F2 v, float rest, uint32_t seed = 0)
    {
        const F2 d = v - F2(rest);
        *reinterpret_cast<uint32_t *>(p + k) = sr_bf16x2(d.v.x, d.v.y, sr_bits(seed, p + k));
    }
    static __device__ __forceinline__ R ldd(const S *p, int64_t k, R) { return __bfloat162float(p[k]); }
    static __device__ __forceinline__ void sdv(S *p, int64_t k, R d, R, uint32_t &rng)
    {
        rng = rng_next(rng);
        p[k] = sr_bf16(d, rng);
    }
    static __device__ __forceinline__ F2 unpack2(uint32_t u) { return F2(__bfloat1622float2(as_bf162(u))); }
    static __device__ __forceinline__ uint32_t pack2(F2 d, uint32_t &rng)
    {
        rng = rng_next(rng);
        return sr_bf16x2(d.v.x, d.v.y, rng);
    }
    static __device__ __forceinline__ F2 ldd2(const S *p, int64_t k, float)
    {
        return unpack2(*reinterpret_cast<const uint32_t *>(p + k));
    }
    static __device__ __forceinline__ void sdv2(S *p, int64_t k, F2 d, float, uint32_t &rng)
    {
        *reinterpret_cast<uint32_t *>(p + k) = pack2(d, rng);
    }
};

// Which form the step kernels run in: deviations from the rest state for the
// storages computed in FP32 (DEV 1), full values for FP64 (its rounding is far
// below the per-step changes of a steady state, and the rest-value
// subtraction and addition would cost FP64-pipe instructions).  ldf / stf
// load and store a population in that form.
template <int PREC>
constexpr int dev_form()
{
    return PREC == LBM_F64 ? 0 : 1;
}
// The 16-bit storages (two nodes' values per 32-bit word).
template <int PREC>
constexpr bool is16()
{
    return PREC == LBM_BF16D || PREC == LBM_F16D || PREC == LBM_F16S || PREC == LBM_BF16S;
}
template <int PREC, class R>
__device__ __forceinline__ R ldf(const typename Store<PREC>::S *p, int64_t k, R rest)
{
    if constexpr (dev_form<PREC>())
        return Store<PREC>::ldd(p, k, rest);
    else
        return Store<PREC>::ld(p, k, rest);
}
template <int PREC, class R>
__device__ __forceinline__ void stf(typename Store<PREC>::S *p, int64_t k, R v, R rest, uint32_t &rng)
{
    if constexpr (dev_form<PREC>())
        Store<PREC>::sdv(p, k, v, rest, rng);
    else
        Store<PREC>::st(p, k, v, rest);
}

// ----------------------------------------------------------- pull streaming
// Opposite directions: 1<->3, 2<->4, 5<->7, 6<->8 (D2Q5 uses the first five).
__host__ __device__ constexpr int opp(int i)
{
    return i == 0 ? 0 : (i <= 4 ? (i + 1) % 4 + 1 : (i - 3) % 4 + 5);
}

// Streamed populations of node (x, y): f_i(x) = f*_i(x - e_i) when the source
// node exists, otherwise the link crossed a wall halfway between the node and
// the wall and the population comes back reversed from the node itself
// (bounce-back for the flow; anti-bounce-back -g* + 2 w T_w on the isothermal
// left/right walls and bounce-back on the adiabatic top/bottom walls for the
// heat).  Velocity order: e0 (0,0), e1 (1,0), e2 (0,1), e3 (-1,0), e4 (0,-1),
// e5 (1,1), e6 (-1,1), e7 (-1,-1), e8 (1,-1).
// REV = true reads a state whose post-collision population f*_i(x) is kept
// in plane opp(i) (the in-place AA layout after an even step).
// DEV = 1 returns deviations from the rest state (f_i - w_i, g_i - w_i T_m);
// the bounce-back rules keep their form (opposite weights are equal), the
// anti-bounce-back becomes -g* + 2 w (T_w - T_m).
template <int PREC, class R, bool REV = false, int DEV = 0>
__device__ __forceinline__ void pull(const typename Store<PREC>::S *__restrict__ src,
                                     const Phys<R> &p, int x, int y, R f[9], R g[5])
{
    using St = Store<PREC>;
    const int64_t P = p.plane, W = p.pitch;
    const int64_t k = (int64_t)y * W + x;
    const bool xl = x > 0, xr = x < p.nx - 1, yb = y > 0, yt = y < p.ny - 1;
#define PL(i) ((REV ? opp(i) : (i)) * P)
#define LD(base, idx, rest) (DEV ? St::ldd(base, idx, rest) : St::ld(base, idx, rest))
    f[0] = LD(src, PL(0) + k, R(rest_f(0)));
    f[1] = xl ? LD(src, PL(1) + k - 1, R(rest_f(1))) : LD(src, PL(3) + k, R(rest_f(3)));
    f[2] = yb ? LD(src, PL(2) + k - W, R(rest_f(2))) : LD(src, PL(4) + k, R(rest_f(4)));
    f[3] = xr ? LD(src, PL(3) + k + 1, R(rest_f(3))) : LD(src, PL(1) + k, R(rest_f(1)));
    f[4] = yt ? LD(src, PL(4) + k + W, R(rest_f(4))) : LD(src, PL(2) + k, R(rest_f(2)));
    f[5] = (xl && yb) ? LD(src, PL(5) + k - W - 1, R(rest_f(5))) : LD(src, PL(7) + k, R(rest_f(7)));
    f[6] = (xr && yb) ? LD(src, PL(6) + k - W + 1, R(rest_f(6))) : LD(src, PL(8) + k, R(rest_f(8)));
    f[7] = (xr && yt) ? LD(src, PL(7) + k + W + 1, R(rest_f(7))) : LD(src, PL(5) + k, R(rest_f(5)));
    f[8] = (xl && yt) ? LD(src, PL(8) + k + W - 1, R(rest_f(8))) : LD(src, PL(6) + k, R(rest_f(6)));
    const typename Store<PREC>::S *gs = src + 9 * P;
    const R ah = DEV ? p.abbd_hot : p.abb_hot, ac = DEV ? p.abbd_cold : p.abb_cold;
    g[0] = LD(gs, PL(0) + k, R(rest_g(0)));
    g[1] = xl ? LD(gs, PL(1) + k - 1, R(rest_g(1))) : ah - LD(gs, PL(3) + k, R(rest_g(3)));
    g[2] = yb ? LD(gs, PL(2) + k - W, R(rest_g(2))) : LD(gs, PL(4) + k, R(rest_g(4)));
    g[3] = xr ? LD(gs, PL(3) + k + 1, R(rest_g(3))) : ac - LD(gs, PL(1) + k, R(rest_g(1)));
    g[4] = yt ? LD(gs, PL(4) + k + W, R(rest_g(4))) : LD(gs, PL(2) + k, R(rest_g(2)));
#undef LD
#undef PL
}

// Pairs of nodes along x for the two-nodes-per-thread paths.  A value taken
// from x - 1 is the previous lane's upper element (lane 0 supplies its own
// halo value); one taken from x + 1 is the next lane's lower element.
__device__ __forceinline__ F2 from_left(F2 a, float halo, int lane)
{
    float l = __shfl_up_sync(0xffffffffu, a.v.y, 1);
    if (lane == 0) l = halo;
    return F2(l, a.v.x);
}
__device__ __forceinline__ F2 from_right(F2 a, float halo, int lane)
{
    float r = __shfl_down_sync(0xffffffffu, a.v.x, 1);
    if (lane == 31) r = halo;
    return F2(a.v.y, r);
}

// ------------------------------------------------------ macroscopic moments
template <class V>
struct Macro {
    V rho, irho, T, ux, uy, Fx, Fy, nu_prev;
    V nu;        // apparent viscosity chosen by the collision (set by collide)
    V drho, dT;  // rho - 1 and T - T_m (accurate in the deviation form)
};

// Porous coefficients of node k when a per-node Darcy field is set:
// K = Da L^2, eps/(4K), eps/K, eps F_eps/(2 sqrt K), eps F_eps/sqrt K.
__device__ __forceinline__ double load_da(const Phys<double> &p, int64_t k) { return ((const double *)p.da)[k]; }
__device__ __forceinline__ float load_da(const Phys<float> &p, int64_t k) { return ((const float *)p.da)[k]; }
__device__ __forceinline__ F2 load_da(const Phys<F2> &p, int64_t k)
{
    return F2(*reinterpret_cast<const float2 *>((const float *)p.da + k));
}
template <class V>
struct Porous {
    V heK, eK, c1, eFsK;
};
// FIELD: 0 the uniform permeability, 1 the per-node field, 2 decide at run
// time from p.da (kernels that know which one they run pass 0 or 1, so the
// other path costs them no registers).
template <class V, int FIELD = 2>
__device__ __forceinline__ Porous<V> porous_at(const Phys<V> &p, int64_t k)
{
    Porous<V> q;
    if (FIELD == 0 || (FIELD == 2 && !p.da)) {
        q.heK = p.half_eps_invK;
        q.eK = p.eps_invK;
        q.c1 = p.c1;
        q.eFsK = p.eFe_isqK;
        return q;
    }
    const V iK = vrcp(load_da(p, k) * p.L2);
    const V isK = vsqrt(iK);
    q.heK = V(0.25) * p.eps * iK;
    q.eK = p.eps * iK;
    q.c1 = V(0.5) * p.eFe * isK;
    q.eFsK = p.eFe * isK;
    return q;
}

// Density and temperature (Eqs. macro_fluid_density and the D2Q5 zeroth
// moment), the half-force velocity of Eq. (velo) with buoyancy
// G = g beta (T - T_m) along +y, and the porous velocity solve
// u = v / (c0 + sqrt(c0^2 + c1 |v|)), c0 = (1 + eps nu / (2K)) / 2, with the
// apparent viscosity of the lagged relaxation time; then the total force
// F = -eps nu u / K - eps F_eps |u| u / sqrt K + eps G.
// DEV = 1: f and g are deviations from the rest state (f_i - w_i,
// g_i - w_i T_m), so the zeroth moments are rho - 1 and T - T_m; every other
// moment used is the same linear form of the deviations.
template <class V, int FIELD = 2, int DEV = 0>
__device__ __forceinline__ Macro<V> macro(const Phys<V> &p, const V f[9], const V g[5], V tau_prev, int64_t k)
{
    Macro<V> m;
    const Porous<V> q = porous_at<V, FIELD>(p, k);
    const V sax = (f[1] + f[2]) + (f[3] + f[4]);
    const V sdg = (f[5] + f[6]) + (f[7] + f[8]);
    const V r0 = f[0] + sax + sdg;
    m.rho = DEV ? r0 + V(1) : r0;
    m.drho = DEV ? r0 : r0 - V(1);
    const V jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    const V jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    const V t0 = g[0] + (g[1] + g[2]) + (g[3] + g[4]);
    m.T = DEV ? t0 + p.Tm : t0;
    m.dT = DEV ? t0 : t0 - p.Tm;
    const V Gy = p.gbeta * m.dT;
    m.irho = vrcp(m.rho);
    const V vx = jx * m.irho;
    const V vy = vfma(p.half_eps, Gy, jy * m.irho);
    m.nu_prev = (tau_prev - V(0.5)) * V(1.0 / 3.0);
    const V c0 = vfma(q.heK, m.nu_prev, V(0.5));
    const V vmag = vsqrt(vfma(vx, vx, vy * vy));
    const V iden = vrcp(c0 + vsqrt(vfma(c0, c0, q.c1 * vmag)));
    m.ux = vx * iden;
    m.uy = vy * iden;
    const V umag = vmag * iden;  // |u| = |v| / den
    const V drag = -vfma(q.eK, m.nu_prev, q.eFsK * umag);
    m.Fx = drag * m.ux;
    m.Fy = vfma(drag, m.uy, p.eps * Gy);
    return m;
}

// Apparent-viscosity factor of Eq. (MPL) for the non-dimensional shear rate.
template <class R>
__device__ __forceinline__ R apparent_s(int mode, R gs, R g1, R g2, R nm1, R Dhi)
{
    if (mode == 0) return gs < g1 ? R(1) : (gs <= g2 ? vpow(gs, nm1) : Dhi);
    const R gc = gs < g1 ? g1 : (gs > g2 ? g2 : gs);
    return vpow(gc, nm1);
}
template <class V>
__device__ __forceinline__ V apparent(const Phys<V> &p, V gs)
{
    return apparent_s(p.clamp_mode, gs, p.gamma1, p.gamma2, p.nm1, p.D_hi);
}
template <>
__device__ __forceinline__ F2 apparent(const Phys<F2> &p, F2 gs)
{
    return F2(apparent_s(p.clamp_mode, gs.v.x, p.gamma1.v.x, p.gamma2.v.x, p.nm1.v.x, p.D_hi.v.x),
              apparent_s(p.clamp_mode, gs.v.y, p.gamma1.v.x, p.gamma2.v.x, p.nm1.v.x, p.D_hi.v.x));
}

// ------------------------------------------- node-local implicit tau
// The relaxation time a collision starts from, solved at the node from its
// own streamed populations instead of read from a stored (lagged) value: the
// root of tau = Phi(tau) = 3 nu_ref D(gamma*(tau)) + 1/2 (Eq. MPL), where
// gamma(tau) is the strain rate macro() and collide() compute when started
// from tau (viscosity of the velocity solve, s7 = s8 = 1/tau).  p.tau_iters
// Newton steps on ln tau from the rest-state tau0:
//   tau <- tau (Phi / tau)^(1/J),  J = 1 + (n - 1) R (Phi - 1/2) / Phi
// where gamma1 < gamma* < gamma2 (D has slope) and J = 1 elsewhere, with
// R = (B^2 + C^2) / (A^2 + B^2 + C^2) = d ln|gamma| / d ln(1/tau) at fixed
// velocity.  J lies between n and 1, so every step is defined.
template <class R>
__device__ __forceinline__ R tau_newton_s(R tau, R gs, R bc, R ss, R g1, R g2, R nm1, R Dhi, int mode, R nu3)
{
    const R phi = vfma(nu3, apparent_s(mode, gs, g1, g2, nm1, Dhi), R(0.5));
    if (!(gs > g1 && gs < g2)) return phi;
    const R J = vfma(nm1 * (bc * vrcp(ss)), (phi - R(0.5)) * vrcp(phi), R(1));
    return tau * vpow(phi * vrcp(tau), vrcp(J));
}
template <class V>
__device__ __forceinline__ V tau_newton(const Phys<V> &p, V tau, V gs, V bc, V ss)
{
    return tau_newton_s(tau, gs, bc, ss, p.gamma1, p.gamma2, p.nm1, p.D_hi, p.clamp_mode, p.nu3);
}
template <>
__device__ __forceinline__ F2 tau_newton(const Phys<F2> &p, F2 tau, F2 gs, F2 bc, F2 ss)
{
    const float g1 = p.gamma1.v.x, g2 = p.gamma2.v.x, nm1 = p.nm1.v.x, Dhi = p.D_hi.v.x, nu3 = p.nu3.v.x;
    return F2(tau_newton_s(tau.v.x, gs.v.x, bc.v.x, ss.v.x, g1, g2, nm1, Dhi, p.clamp_mode, nu3),
              tau_newton_s(tau.v.y, gs.v.y, bc.v.y, ss.v.y, g1, g2, nm1, Dhi, p.clamp_mode, nu3));
}

template <class V, int FIELD = 2, int DEV = 0>
__device__ __forceinline__ V implicit_tau(const Phys<V> &p, const V f[9], const V g[5], int64_t k)
{
    const Porous<V> q = porous_at<V, FIELD>(p, k);
    // moments that do not depend on tau (as in macro() and collide(); DEV as
    // there)
    const V sax = (f[1] + f[2]) + (f[3] + f[4]);
    const V sdg = (f[5] + f[6]) + (f[7] + f[8]);
    const V r0 = f[0] + sax + sdg;
    const V rho = DEV ? r0 + V(1) : r0;
    const V jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    const V jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    const V t0 = g[0] + (g[1] + g[2]) + (g[3] + g[4]);
    const V dT = DEV ? t0 : t0 - p.Tm;
    const V irho = vrcp(rho);
    const V vx = jx * irho;
    const V vy = vfma(p.half_eps, p.gbeta * dT, jy * irho);
    const V c1v = q.c1 * vsqrt(vfma(vx, vx, vy * vy));
    const V e = vfma(V(2), sdg, vfma(V(-4), f[0], -sax));
    const V pxx = (f[1] + f[3]) - (f[2] + f[4]);
    const V pxy = (f[5] + f[7]) - (f[6] + f[8]);
    const V rie = rho * p.inv_eps;
    const V gsc = V(3) * irho * p.gamma_scale;
    V tau = p.tau0;
#pragma unroll 1
    for (int it = 0; it < p.tau_iters; ++it) {
        const V nu = (tau - V(0.5)) * V(1.0 / 3.0);
        const V c0 = vfma(q.heK, nu, V(0.5));
        const V iden = vrcp(c0 + vsqrt(vfma(c0, c0, c1v)));
        const V ux = vx * iden, uy = vy * iden;
        const V u2e3 = V(3) * vfma(ux, ux, uy * uy) * p.inv_eps;
        const V e_eq = vfma(rho, u2e3, V(-2) * (DEV ? r0 : rho));
        const V w = vrcp(tau);
        const V A = V(1.4 / 6.0) * (e - e_eq);
        const V B = V(0.5) * w * (pxx - rie * vfma(ux, ux, -(uy * uy)));
        const V C = w * (pxy - rie * (ux * uy));
        const V bc = vfma(B, B, C * C);
        const V ss = vfma(A, A, bc);
        tau = tau_newton(p, tau, gsc * vsqrt(ss), bc, ss);
    }
    return tau;
}

// tau the collision of a node starts from: TAU 0 the stored lagged value
// (loaded only then), TAU 1 the implicit solve.
template <int TAU, class V, int FIELD, int DEV = 0, class Load>
__device__ __forceinline__ V tau_start(const Phys<V> &p, const V f[9], const V g[5], int64_t k, Load load)
{
    if constexpr (TAU == 1)
        return implicit_tau<V, FIELD, DEV>(p, f, g, k);
    else
        return load();
}

// Full node update in place: f, g become the post-collision populations.
// Returns the new relaxation time; m receives the macroscopic moments and the
// apparent lattice viscosity of this collision.  k is the node's offset in a
// plane (used only to read a per-node Darcy field).
template <class V, int FIELD = 2, int DEV = 0>
__device__ __forceinline__ V collide(const Phys<V> &p, V f[9], V g[5], V tau_prev, Macro<V> &m, int64_t k)
{
    m = macro<V, FIELD, DEV>(p, f, g, tau_prev, k);
    const V rho = m.rho, ux = m.ux, uy = m.uy;
    // raw moments (DEV: e + 2 and eps - 1, their rest values removed)
    const V sax = (f[1] + f[2]) + (f[3] + f[4]);
    const V sdg = (f[5] + f[6]) + (f[7] + f[8]);
    const V e = vfma(V(2), sdg, vfma(V(-4), f[0], -sax));
    const V ep = vfma(V(4), f[0], vfma(V(-2), sax, sdg));
    const V qx = vfma(V(-2), f[1] - f[3], (f[5] - f[6]) + (f[8] - f[7]));
    const V qy = vfma(V(-2), f[2] - f[4], (f[5] + f[6]) - (f[7] + f[8]));
    const V pxx = (f[1] + f[3]) - (f[2] + f[4]);
    const V pxy = (f[5] + f[7]) - (f[6] + f[8]);
    // equilibria
    const V rie = rho * p.inv_eps;
    const V u2e3 = V(3) * vfma(ux, ux, uy * uy) * p.inv_eps;
    // DEV: e_eq + 2 = rho u2e3 - 2 (rho - 1), eps_eq - 1 = (rho - 1) - rho u2e3
    const V r0 = DEV ? m.drho : rho;
    const V e_eq = vfma(rho, u2e3, V(-2) * r0);
    const V ep_eq = r0 - rho * u2e3;
    const V pxx_eq = rie * vfma(ux, ux, -(uy * uy));
    const V pxy_eq = rie * (ux * uy);
    // strain rate from the non-equilibrium moments with the lagged tau:
    // gamma_xx,yy = -3/(2 rho) (s1 e_neq / 6 +- w pxx_neq / 2),
    // gamma_xy = -3/(2 rho) w pxy_neq, |gamma| = sqrt(2 gamma:gamma)
    //          = (3 / rho) sqrt(A^2 + B^2 + C^2)
    const V wp = vrcp(tau_prev);
    const V A = V(1.4 / 6.0) * (e - e_eq);
    const V B = V(0.5) * wp * (pxx - pxx_eq);
    const V C = wp * (pxy - pxy_eq);
    const V gam = V(3) * m.irho * vsqrt(vfma(A, A, vfma(B, B, C * C)));
    const V nu = p.nu_ref * apparent<V>(p, gam * p.gamma_scale);
    const V tau = vfma(V(3), nu, V(0.5));
    const V w = vrcp(tau);
    m.nu = nu;
    // forcing moments (M applied to the velocity-space porous force term)
    const V Fe = V(6) * rie * vfma(ux, m.Fx, uy * m.Fy);
    const V Fxx = V(2) * rie * vfma(ux, m.Fx, -(uy * m.Fy));
    const V Fxy = rie * vfma(ux, m.Fy, uy * m.Fx);
    // post-collision moments, m* = m - S (m - m_eq) + (I - S/2) F
    const V es = vfma(V(0.3), Fe, vfma(V(-1.4), e - e_eq, e));
    const V eps_s = vfma(V(-0.3), Fe, vfma(V(-1.4), ep - ep_eq, ep));
    const V jxs = rho * vfma(V(0.5), m.Fx, ux);
    const V jys = rho * vfma(V(0.5), m.Fy, uy);
    const V qxs = vfma(V(-0.4) * rho, m.Fx, vfma(V(-1.2), vfma(rho, ux, qx), qx));
    const V qys = vfma(V(-0.4) * rho, m.Fy, vfma(V(-1.2), vfma(rho, uy, qy), qy));
    const V hw = vfma(V(-0.5), w, V(1));
    const V pxxs = vfma(hw, Fxx, vfma(-w, pxx - pxx_eq, pxx));
    const V pxys = vfma(hw, Fxy, vfma(-w, pxy - pxy_eq, pxy));
    // f* = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4) m*
    const V a0 = r0 * V(1.0 / 9.0), a1 = es * V(1.0 / 36.0), a2 = eps_s * V(1.0 / 36.0);
    const V a3 = jxs * V(1.0 / 6.0), a4 = qxs * V(1.0 / 12.0);
    const V a5 = jys * V(1.0 / 6.0), a6 = qys * V(1.0 / 12.0);
    const V a7 = pxxs * V(0.25), a8 = pxys * V(0.25);
    const V b_ax = vfma(V(-2), a2, a0 - a1);  // common part of f1..f4
    const V b_dg = vfma(V(2), a1, a0 + a2);   // common part of f5..f8
    const V xa = vfma(V(-2), a4, a3), ya = vfma(V(-2), a6, a5);
    const V xd = a3 + a4, yd = a5 + a6;
    f[0] = vfma(V(4), a2 - a1, a0);
    f[1] = b_ax + xa + a7;
    f[2] = b_ax + ya - a7;
    f[3] = b_ax - xa + a7;
    f[4] = b_ax - ya - a7;
    f[5] = b_dg + xd + yd + a8;
    f[6] = b_dg - xd + yd - a8;
    f[7] = b_dg - xd - yd + a8;
    f[8] = b_dg + xd - yd - a8;
    // thermal MRT: n = N g, n* = n - S_T (n - n_eq), n_eq = (T, T u, -2T/3, 0)
    // (DEV: n_0 and n_3 without their rest values T_m and -2 T_m / 3)
    const V T = m.T, T0 = DEV ? m.dT : m.T;
    const V n1 = g[1] - g[3], n2 = g[2] - g[4];
    const V n3 = vfma(V(-4), g[0], (g[1] + g[2]) + (g[3] + g[4]));
    const V n4 = (g[1] + g[3]) - (g[2] + g[4]);
    const V n1s = vfma(-p.omegaT, vfma(-T, ux, n1), n1);
    const V n2s = vfma(-p.omegaT, vfma(-T, uy, n2), n2);
    const V n3s = vfma(-p.s_e, vfma(V(2.0 / 3.0), T0, n3), n3);
    const V n4s = vfma(-p.s_p, n4, n4);
    // g* = N^T diag(1/5, 1/2, 1/2, 1/20, 1/4) n*
    const V t0 = T0 * V(0.2), t3 = n3s * V(0.05), t4 = n4s * V(0.25);
    const V h1 = n1s * V(0.5), h2 = n2s * V(0.5);
    const V t03 = t0 + t3;
    g[0] = vfma(V(-0.2), n3s, t0);
    g[1] = t03 + h1 + t4;
    g[2] = t03 + h2 - t4;
    g[3] = t03 - h1 + t4;
    g[4] = t03 - h2 - t4;
    return tau;
}

}  // namespace lbm
