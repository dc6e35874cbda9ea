/*
 * lbm_debug.h -- a check of the library's own memory discipline, for tests
 * (the paper has no counterpart).  Not part of the method.
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

#ifdef __cplusplus
}
#endif
#endif
