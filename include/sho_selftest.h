/*
 * sho_selftest.h -- self-test of the tensor-core operand layouts (part of libsho.so).
 *
 * The paper has no counterpart: this entry point lets the test suite check, in isolation, that the
 * shared-memory operand layouts and descriptors the tcgen05 kernels build give the textbook product.
 */
#ifndef SHO_SELFTEST_H
#define SHO_SELFTEST_H

#include "sho.h"

#ifdef __cplusplus
extern "C" {
#endif

/* One fifth-generation tensor-core MMA on the current device, D = A B^T with M = 128, N = 32 and
 * K = 8 (bf16 == 0: TF32 operands) or K = 16 (bf16 != 0: BF16 operands), FP32 accumulation:
 *   A  host [128][K] floats (rounded to the operand type), B  host [32][K] floats, D  host [128][32] out.
 * The operands go through the same K-major shared-memory layout, descriptors and tensor-memory read-back
 * as the expansion kernel.  Synchronous; allocates and frees its own device buffers.  Returns SHO_OK,
 * SHO_ERR_ARG for a null pointer, SHO_ERR_OOM / SHO_ERR_CUDA, or SHO_ERR_TIMEOUT when the MMA's
 * completion barrier did not arrive within its bound. */
int sho_selftest_umma(int bf16, const float* A, const float* B, float* D);

/* The digit-pair MMA schedule of the FP64-accurate expansion on the tensor cores: six TF32 digit slices
 * of A [128][8] and of B [32][8], every pair (i, j) with i + j <= 8 (i, j = 1..6) accumulated into level
 * accumulator min(i + j, 5) - 2, M = 128, N = 32, K = 8:
 *   A  host [6][128][8] floats (slice i - 1 of A), B  host [6][32][8] floats, D  host [4][128][32] out.
 * The operands go through the same shared-memory layout (states 4..7 in a second chunk), descriptors
 * and tensor-memory read-back as the expansion kernel; with digit values that are integers of at most
 * 128 times 2^(-8 i) the first three accumulators are exact sums.  Synchronous; allocates and frees its
 * own device buffers.  Returns as sho_selftest_umma. */
int sho_selftest_ozaki(const float* A, const float* B, float* D);

#ifdef __cplusplus
}
#endif

#endif /* SHO_SELFTEST_H */
