// Host check of the stochastic rounding in lbm_round.cuh (compiled with nvcc
// for the host only; no GPU).  For each test value x and every one of the
// 65536 values of the 16 random bits:
//   * the result is one of the two representable neighbours of x (x itself
//     when x is representable);
//   * the mean over all 65536 draws equals x to within 2^-12 of the spacing
//     (the dither's resolution), i.e. the rounding is unbiased.
// Also: the hash is a bijection on 32 bits (no collision over 2^22 inputs).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "lbm_round.cuh"

using namespace lbm;

static float half_next_away(__half h)
{
    unsigned short b;
    memcpy(&b, &h, 2);
    b = (unsigned short)(b + 1);   // magnitude bits + 1 (sign-magnitude)
    __half n;
    memcpy(&n, &b, 2);
    return __half2float(n);
}
static float bf16_next_away(__nv_bfloat16 h)
{
    unsigned short b;
    memcpy(&b, &h, 2);
    b = (unsigned short)(b + 1);
    __nv_bfloat16 n;
    memcpy(&n, &b, 2);
    return __bfloat162float(n);
}

// kind 0: sr_half, 1: sr_bf16, 2: sr_half_normal (unbiased only for
// |x| >= 2^-14; below, biased toward zero by less than one spacing)
static int check_kind(float x, int kind)
{
    const bool half = kind != 1;
    const float lo = half ? __half2float(__float2half_rz(x)) : __bfloat162float(__float2bfloat16_rz(x));
    const float hi = half ? half_next_away(__float2half_rz(x)) : bf16_next_away(__float2bfloat16_rz(x));
    double sum = 0.0;
    for (uint32_t r = 0; r < 65536u; ++r) {
        const float v = kind == 0 ? __half2float(sr_half(x, r))
                                  : kind == 1 ? __bfloat162float(sr_bf16(x, r)) : __half2float(sr_half_normal(x, r));
        if (lo == x ? v != x : (v != lo && v != hi)) {
            printf("FAIL bracket %s x=%.9g r=%u v=%.9g lo=%.9g hi=%.9g\n", half ? "half" : "bf16", x, r, v, lo, hi);
            return 1;
        }
        sum += v;
    }
    const double mean = sum / 65536.0;
    const bool sub = kind == 2 && fabs(x) < 6.103515625e-05;
    const double tol = fabs((double)hi - (double)lo) * (sub ? 1.0 : 1.0 / 4096.0);
    if (fabs(mean - (double)x) > tol) {
        printf("FAIL mean %s x=%.9g mean=%.12g tol=%.3g\n", half ? "half" : "bf16", x, mean, tol);
        return 1;
    }
    return 0;
}

static int check(float x, bool half) { return half ? check_kind(x, 0) + check_kind(x, 2) : check_kind(x, 1); }

int main()
{
    int bad = 0, n = 0;
    const float special[] = {0.0f, 5.9604644775390625e-8f, 2.98e-8f, 8.9e-8f, 1.0e-7f, 6.1035156e-5f,
                             6.0e-5f, 6.2e-5f, 1.0f, 0.5f, 0.0123f, 3.0e-6f, 1.5e-9f};
    for (float s : special)
        for (int sign = 0; sign < 2; ++sign) {
            const float x = sign ? -s : s;
            bad += check(x, true) + check(x, false);
            n += 2;
        }
    uint64_t st = 2011;
    for (int i = 0; i < 3000; ++i) {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        const double u = (double)(st >> 11) * (1.0 / 9007199254740992.0);
        const float x = (float)((i & 1 ? -1.0 : 1.0) * pow(10.0, -10.0 + 10.0 * u));
        bad += check(x, true) + check(x, false);
        n += 2;
    }
    // the hash is invertible: no two of 2^22 consecutive inputs collide
    const uint32_t N = 1u << 22;
    unsigned char *seen = (unsigned char *)calloc(1u << 29, 1);   // one bit per 32-bit value
    if (!seen) return 2;
    for (uint32_t i = 0; i < N; ++i) {
        const uint32_t h = mix32(0x12345u + i);
        if (seen[h >> 3] & (1u << (h & 7))) {
            printf("FAIL hash collision at %u\n", i);
            ++bad;
            break;
        }
        seen[h >> 3] |= (unsigned char)(1u << (h & 7));
    }
    free(seen);
    printf("%s %d values checked\n", bad ? "FAILED" : "OK", n);
    return bad ? 1 : 0;
}
