// sho_ff.cuh -- float-float ("double-FP32") arithmetic for the FP64-accurate form on the FP32 pipe.
//
// A double v is carried as an unevaluated pair (hi, lo) of floats with v ~= hi + lo to about 48
// significant bits.  Products use the error-free FMA product (Dekker's TwoProduct as restated with a
// fused multiply-add): p = a*b, e = fma(a, b, -p) gives a*b = p + e exactly.  Sums use Knuth's
// error-free TwoSum.  A dot product accumulated this way (Ogita, Rump & Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005, Algorithm Dot2 extended to pair inputs) is as accurate as if
// computed in twice the working precision: relative errors of order 2^-48, far inside the 1e-12 bar
// of the FP64 form, while every instruction runs on the FP32 pipe (61x the FP64 rate on GB300).
#pragma once

#include <cuda_runtime.h>

namespace sho {

struct ff {
  float hi, lo;
};

// Split a double into hi + lo without FP64 instructions: hi takes the sign, exponent and the top 23
// mantissa bits (truncation), lo the next bits of the remainder (rounded once to float).  Magnitudes
// outside the float normal range (below 2^-126 or at/above 2^128) are flushed to zero; the FP64-accurate
// form documents that its inputs must lie inside that range.
//   hi: bits 29..60 of the double hold the low 9 exponent bits and the top 23 mantissa bits; subtracting
//       384 from that 9-bit field modulo 2^32 rebases the exponent from 1023 to 127 for every exponent in
//       range (the result's field, e - 896, fits in 8 bits), then the sign is or-ed in.
//   lo: the low 29 mantissa bits converted to float times 2^(e - 1075), a signed power of two taken from
//       hi's exponent field minus 52; zero when that would leave the normal range (|v| < 2^-74).
__device__ __forceinline__ ff ff_from_double(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned int lw = (unsigned int)b, hw = (unsigned int)(b >> 32);
  const unsigned int ax = hw & 0x7fffffffu;
  const bool ok = ax - 0x38100000u < 0x47f00000u - 0x38100000u;  // biased exponent in [897, 1150]
  const unsigned int hib = ((unsigned int)(b >> 29) - 0xc0000000u) | (hw & 0x80000000u);
  const unsigned int sb = (hib - 0x1a000000u) & 0xff800000u;       // sign | (e - 948) << 23
  ff r;
  r.hi = ok ? __uint_as_float(hib) : 0.0f;
  r.lo = (ok && ax >= 0x3b500000u) ? __uint2float_rn(lw & 0x1fffffffu) * __uint_as_float(sb) : 0.0f;
  return r;
}

// True for a value the split above cannot carry: outside [2^-126, 2^128) in magnitude (values too small
// or too large for a float exponent, inf and NaN) and not zero.  Integer instructions on the high word
// that ff_from_double also tests; a double whose high word is zero apart from the sign (|v| < 2^-1042)
// counts as zero.
__device__ __forceinline__ bool ff_out_of_range(double v) {
  const unsigned int ax = (unsigned int)((unsigned long long)__double_as_longlong(v) >> 32) & 0x7fffffffu;
  return (ax - 0x38100000u >= 0x47f00000u - 0x38100000u) && ax != 0u;
}

// Split a double into hi + lo with FP64 arithmetic (for values computed once per table entry).
__device__ __forceinline__ ff ff_from_double_exact(double v) {
  ff r;
  r.hi = __double2float_rn(v);
  r.lo = __double2float_rn(v - (double)r.hi);
  return r;
}

// Exact float -> double widening with integer instructions (no FP64-pipe conversion); zeros and
// subnormal floats map to 0.
__device__ __forceinline__ double f2d_int(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xffu;
  if (e == 0u) return 0.0;
  const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                  ((unsigned long long)(e - 127u + 1023u) << 52) |
                                  ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

// s + c as a double: two exact widenings and one FP64 add.
__device__ __forceinline__ double ff_to_double(float s, float c) { return f2d_int(s) + f2d_int(c); }

// Accumulate a*b (pairs) into the running dot product (s, c):  s + c += (a.hi + a.lo)(b.hi + b.lo),
// dropping only a.lo*b.lo.  s carries the error-free sum of the leading products, c the errors and
// the cross terms.  With p = fl(a.hi b.hi) and TwoSum(s, p) = (t, (s - (t - bb)) + (p - bb)), the
// product's exact low part a.hi b.hi - p and TwoSum's exact term p - bb are taken together as one
// fused a.hi b.hi - bb (rounded once, as their sum would be), so a step is 10 FP32 instructions.
// p must be the rounded product: __fmul_rn keeps the compiler from fusing it into s + a.hi b.hi,
// which would break TwoSum's exactness (errors near 1e-8 instead of 1e-15).
__device__ __forceinline__ void ff_dot_step(float& s, float& c, const ff a, const ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float t = s + p;                     // TwoSum(s, p)
  const float bb = t - s;
  float q = fmaf(a.hi, b.hi, -bb);           // (a.hi b.hi - p) + (p - bb)
  q = fmaf(a.hi, b.lo, q);
  q = fmaf(a.lo, b.hi, q);
  const float r = s - (t - bb);              // TwoSum's other exact term
  s = t;
  c += q + r;
}

// Renormalise a pair so that |lo| <= ulp(hi)/2 (Fast2Sum; valid because |c| <= |s| here).
__device__ __forceinline__ ff ff_norm(float s, float c) {
  const float t = s + c;
  ff r;
  r.hi = t;
  r.lo = c - (t - s);
  return r;
}

// v times the unit complex number ph = (re.hi, re.lo, im.hi, im.lo) for complex data held by lane pairs,
// the real part in the even lane and the imaginary part in the odd one (every lane of the warp calls it):
// even lane re c - im s, odd lane im c + re s, as two float-float products and a TwoSum (the products may
// cancel, so no ordering of the pair is assumed).
__device__ __forceinline__ ff ff_rotate(ff v, const float4 ph, int lane) {
  const ff u{__shfl_xor_sync(0xffffffffu, v.hi, 1), __shfl_xor_sync(0xffffffffu, v.lo, 1)};
  const float sg = (lane & 1) ? 1.0f : -1.0f;
  float s = 0.0f, c = 0.0f;
  ff_dot_step(s, c, v, ff{ph.x, ph.y});
  ff_dot_step(s, c, u, ff{sg * ph.z, sg * ph.w});
  const float t = s + c;
  const float bb = t - s;
  return ff{t, (s - (t - bb)) + (c - bb)};
}

// True when ph is exactly 1 (no turn needed).
__device__ __forceinline__ bool ff_is_one(const float4 ph) {
  return ph.x == 1.0f && ph.y == 0.0f && ph.z == 0.0f && ph.w == 0.0f;
}

}  // namespace sho
