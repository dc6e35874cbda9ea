// Host check of the counter-based hash that supplies the stochastic
// rounding's random bits (lbm_round.cuh; compiled with nvcc for the host
// only, no GPU): lowbias32 is a bijection on 32 bits, so no two of 2^22
// consecutive inputs collide, and the hashed starts of a row of nodes are
// uniform in their top 16 bits (chi-square over 256 bins).  The conversions
// themselves are device instructions, checked on the GPU.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "lbm_round.cuh"

using namespace lbm;

int main()
{
    int bad = 0;
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
    // rng_init over 2^20 consecutive nodes: top byte of the 16 bits a half-word uses
    static double cnt[256];
    const int M = 1 << 20;
    for (int k = 0; k < M; ++k) cnt[rng_init(7u, k) >> 24] += 1.0;
    double chi = 0.0;
    for (int b = 0; b < 256; ++b) chi += (cnt[b] - M / 256.0) * (cnt[b] - M / 256.0) / (M / 256.0);
    if (chi > 400.0) {   // 255 degrees of freedom: mean 255, sd 22.6
        printf("FAIL chi-square %.1f\n", chi);
        ++bad;
    }
    printf("%s hash bijective over 2^22 inputs, chi-square %.1f\n", bad ? "FAILED" : "OK", chi);
    return bad ? 1 : 0;
}
