/*
 * lbm_debug.h -- checks of the library's own machinery, for tests (the paper
 * has no counterpart): its memory discipline and the stochastic rounding of
 * its 16-bit storages.  Not part of the method.
 *
 * Same conventions as lbm.h: 0 on success, a negative LBM_* code otherwise.
 */
#ifndef LBM_DEBUG_H
#define LBM_DEBUG_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Canary of the state buffers.  Every plane row is padded to a multiple of
 * 64 elements, the buffers are zero-filled when the context is created, and
 * no kernel may write a padding element (x >= nx).  *nonzero receives the
 * number of nonzero bytes in the padding of every distribution and relaxation
 * time plane of both buffers: 0 unless a kernel wrote outside the rows.
 * Grids whose width is a multiple of 64 have no padding (always 0).
 * Synchronous.  Errors: LBM_ERR_ARG (NULL), LBM_ERR_OOM, LBM_ERR_CUDA. */
int lbm_debug_padding_canary(lbm_ctx *ctx, unsigned long long *nonzero);

/* The stochastic rounding the 16-bit storages store with, one pair of values
 * per 32-bit word as the step kernels store it.  fmt 0: FP16, 1: BF16.  For
 * i < n_pairs, x[2i] (low half) and x[2i+1] (high half) are converted with the
 * 32 random bits r[i]; out[2i], out[2i+1] receive the 16-bit codes.  The
 * values are converted as given (the FP16 storage's 2^15 scale is applied by
 * the caller).  Host buffers (x: 2 n_pairs floats, r: n_pairs words, out:
 * 2 n_pairs codes), owned by the caller; runs on `device` and returns when
 * the codes are in out.  n_pairs = 0 does nothing.
 * Errors: LBM_ERR_ARG (NULL buffer, fmt not 0 or 1), LBM_ERR_OOM,
 * LBM_ERR_CUDA. */
int lbm_debug_sr_pairs(int device, int fmt, const float *x, const uint32_t *r, uint16_t *out, size_t n_pairs);

#ifdef __cplusplus
}
#endif
#endif
