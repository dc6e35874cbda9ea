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
// The hash and the random-bit sequence are __host__ __device__, so that a
// host test can check the hash; the conversions are device instructions,
// checked on the GPU over every value of their random bits.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

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

// FP32 -> 16-bit with stochastic rounding, done by the conversion
// instruction itself: cvt with the .rs rounding mode (PTX ISA 8.7, sm_100
// family) turns each FP32 value of a pair into the 16-bit neighbour below or
// above it in magnitude, the one above with probability (distance to the one
// below) / (their spacing).  The value in the word's high half draws on the
// high 16 bits of r, the low half on the low 16 bits.  Measured on GB300
// over every value of those bits: BF16 rounds up iff the 16 dropped bits
// plus the 16 random bits carry, so the result is x in expectation exactly;
// FP16 uses the low 13 of its 16 bits against the 13 mantissa bits a normal
// FP16 drops (exact in expectation too), and for FP16 subnormals, which drop
// more bits, it compares the top 13 of them, a bias toward zero under 2^-13
// of a spacing.  One instruction per pair replaces the integer dither and
// truncating conversion of a software version.
__device__ __forceinline__ uint32_t sr_half2(float lo, float hi, uint32_t r)
{
    uint32_t out;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(out) : "f"(hi), "f"(lo), "r"(r));
    return out;
}
__device__ __forceinline__ uint32_t sr_bf16x2(float lo, float hi, uint32_t r)
{
    uint32_t out;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(out) : "f"(hi), "f"(lo), "r"(r));
    return out;
}
// One value (the low half of a pair; the low half of r decides).
__device__ __forceinline__ __half sr_half(float x, uint32_t r)
{
    return __ushort_as_half((unsigned short)(sr_half2(x, 0.0f, r) & 0xffffu));
}
__device__ __forceinline__ __nv_bfloat16 sr_bf16(float x, uint32_t r)
{
    return __ushort_as_bfloat16((unsigned short)(sr_bf16x2(x, 0.0f, r) & 0xffffu));
}

}  // namespace lbm
