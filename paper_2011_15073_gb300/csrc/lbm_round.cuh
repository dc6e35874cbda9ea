// lbm_round.cuh -- stochastic rounding of FP32 values to the 16-bit storage
// formats, and the counter-based hash that supplies its random bits.
//
// Round-to-nearest storage loses every update smaller than half a unit in
// the last place, and near a steady state the per-step change of a
// population is far below that for 16-bit formats, so the stored state
// stalls away from the steady state of the scheme.  Stochastic rounding
// rounds x to the representable neighbour above or below with probability
// proportional to its distance from the other one, so the stored value is x
// in expectation and small updates survive on average.
//
// Everything here is __host__ __device__ so that the host unit test can
// check it exhaustively.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <string.h>

namespace lbm {

// 32-bit integer hash "lowbias32" (C. Wellons, "Prospecting for Hash
// Functions", 2018): xorshift-multiply rounds with the published constants.
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Random bits for the value stored at element address a in step seed s.
__host__ __device__ __forceinline__ uint32_t sr_bits(uint32_t seed, const void *a)
{
    const uint64_t u = (uint64_t)(uintptr_t)a;
    return mix32(seed ^ (uint32_t)(u >> 1) ^ (uint32_t)(u >> 33) * 0x9e3779b9u);
}

__host__ __device__ __forceinline__ uint32_t f2u(float x)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(x);
#else
    uint32_t u;
    memcpy(&u, &x, 4);
    return u;
#endif
}
__host__ __device__ __forceinline__ float u2f(uint32_t u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float x;
    memcpy(&x, &u, 4);
    return x;
#endif
}

// Start of a thread's random bits for the node at plane offset k in the
// launch with seed `seed`, and the next draw: a Weyl sequence (golden-ratio
// increment), one add per draw.  Every draw is uniform over 32 bits because
// the hashed start is; draws of one node are correlated with each other,
// which leaves each rounding unbiased.
__host__ __device__ __forceinline__ uint32_t rng_init(uint32_t seed, int64_t k)
{
    return mix32(seed ^ (uint32_t)k ^ (uint32_t)((uint64_t)k >> 32) * 0x9e3779b9u);
}
__host__ __device__ __forceinline__ uint32_t rng_next(uint32_t r) { return r + 0x9e3779b9u; }

// FP32 -> FP16 with stochastic rounding, r16 = 16 random bits.
// * Half normals (|x| >= 2^-14): the FP32 bits below the half's last place
//   are the low 13 mantissa bits; adding a uniform integer in [0, 2^13) to
//   the FP32 bit pattern and truncating toward zero rounds the magnitude up
//   with probability (distance to the lower neighbour) / (spacing).  A carry
//   into the exponent lands on the next binade's first value, which is the
//   upper neighbour there, so binade ends are handled too.
// * Half subnormals (|x| < 2^-14): the spacing is the constant 2^-24, so
//   |x| / 2^-24 = q (exact in FP32) is rounded to floor(q) or floor(q) + 1 by
//   comparing its fraction with a uniform number in [0, 1) of 16-bit
//   resolution.
__host__ __device__ __forceinline__ __half sr_half(float x, uint32_t r16)
{
    uint32_t b = f2u(x);
    const int e = (int)((b >> 23) & 0xffu);
    if (e < 113) {
        const float q = u2f(b & 0x7fffffffu) * 16777216.0f;   // |x| / 2^-24 < 1024, exact
        const float fl = floorf(q);
        const float u = (float)(r16 & 0xffffu) * (1.0f / 65536.0f);
        const float m = (fl + (u < q - fl ? 1.0f : 0.0f)) * 5.9604644775390625e-8f;
        return __float2half_rz((b >> 31) ? -m : m);
    }
    b += (r16 & 0xffffu) >> 3;
    return __float2half_rz(u2f(b));
}

// The half-normal branch alone, for the scaled FP16 storage whose values
// sit in the normal range: one integer add and one conversion.  Magnitudes
// below 2^-14 (FP16's smallest normal) are then truncated toward zero on the
// subnormal grid instead of rounded stochastically: the result is still one
// of the two neighbours, biased toward zero by less than one spacing, 2^-24.
__host__ __device__ __forceinline__ __half sr_half_normal(float x, uint32_t r16)
{
    return __float2half_rz(u2f(f2u(x) + ((r16 & 0xffffu) >> 3)));
}

// Two values at once, as packed 16-bit pairs (x in the low half): the same
// dithers as sr_half_normal(x, r & 0xffff), sr_half_normal(y, r >> 16) and
// sr_bf16 likewise, with one packed truncating conversion.
__device__ __forceinline__ uint32_t sr_half2_normal(float x, float y, uint32_t r)
{
    const float xd = u2f(f2u(x) + ((r & 0xffffu) >> 3)), yd = u2f(f2u(y) + (r >> 19));
    uint32_t out;
    asm("cvt.rz.f16x2.f32 %0, %1, %2;" : "=r"(out) : "f"(yd), "f"(xd));
    return out;
}
__device__ __forceinline__ uint32_t sr_bf16x2(float x, float y, uint32_t r)
{
    const float xd = u2f(f2u(x) + (r & 0xffffu)), yd = u2f(f2u(y) + (r >> 16));
    uint32_t out;
    asm("cvt.rz.bf16x2.f32 %0, %1, %2;" : "=r"(out) : "f"(yd), "f"(xd));
    return out;
}

// FP32 -> BF16 with stochastic rounding: BF16 keeps the top 16 bits of the
// FP32 pattern, so the dither is the 16 random bits themselves (FP32
// subnormals are not stored: |deviation| >= 2^-126 or 0 in practice).
__host__ __device__ __forceinline__ __nv_bfloat16 sr_bf16(float x, uint32_t r16)
{
    const uint32_t b = f2u(x) + (r16 & 0xffffu);
    return __float2bfloat16_rz(u2f(b));
}

}  // namespace lbm
