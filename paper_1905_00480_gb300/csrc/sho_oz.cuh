// sho_oz.cuh -- device helpers of the exact digit slicing (Ozaki scheme) shared by the tensor-core
// FP64-accurate projection and expansion.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace sho {

// float 2^e for e in [-126, 127]
__device__ __forceinline__ float oz_pow2(int e) { return __uint_as_float((uint32_t)(e + 127) << 23); }

// Knuth's TwoSum: s + e = a + b exactly.
__device__ __forceinline__ void oz_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Round r to the grid 2^(k - 23) with the constant 1.5 * 2^k (|r| <= 2^(k-1)): the digit, and r less it.
__device__ __forceinline__ float oz_digit(float& r, float sigma) {
  const float d = __fsub_rn(__fadd_rn(r, sigma), sigma);
  r = __fsub_rn(r, d);
  return d;
}

}  // namespace sho
