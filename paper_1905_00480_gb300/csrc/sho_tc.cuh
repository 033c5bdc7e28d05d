// sho_tc.cuh -- tensor-core fragments for the reduced-precision x-pass.
//
// The x-pass of one grid row is the small GEMM  T1[b][n] = sum_x psi[x][b] phi_n(x)  (projection) or
// psi[x][b] += sum_n T1[b][n] phi_n(x)  (expansion), bands on the M side.  Warp-level mma.sync tiles
// (m16n8k8 TF32, m16n8k16 BF16/FP16, FP32 accumulation) are used with operands taken straight from
// registers.  Precision forms (Markidis et al. 2018; Ootomo & Yokota 2022 for the split forms):
//   TF32        a*b with both rounded to TF32 (cvt.rna)
//   3XTF32      a_hi*b_hi + a_hi*b_lo + a_lo*b_hi, x_hi = tf32(x), x_lo = tf32(x - x_hi)
//   BF16        a*b with both rounded to BF16
//   SPLIT_FP16  a_hi*b_hi + 2^-11 (a_hi*b_lo' + a_lo'*b_hi), x_hi = fp16(x), x_lo' = fp16((x - x_hi) 2^11);
//               the scaled low parts keep their precision away from the FP16 subnormal range.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "sho_device.cuh"

namespace sho {

enum class TcMode : int { TF32 = 0, X3TF32 = 1, BF16 = 2, SPLIT16 = 3 };

__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_bits(x);
  lo = tf32_bits(x - __uint_as_float(hi));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo_k, float hi_k) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo_k, hi_k);  // .x = lo_k (lower half), .y = hi_k
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t pack_f16(float lo_k, float hi_k) {
  __half2 v = __floats2half2_rn(lo_k, hi_k);
  return *reinterpret_cast<uint32_t*>(&v);
}

// x = hi + 2^-11 lo' with hi = fp16(x), lo' = fp16((x - hi) * 2^11)
__device__ __forceinline__ void f16_split(float x, float& hi, float& lo_scaled) {
  hi = __half2float(__float2half_rn(x));
  lo_scaled = (x - hi) * 2048.0f;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_f16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// K extent of one MMA step for a mode: 8 (TF32 forms) or 16 (16-bit forms).
template <TcMode M>
struct TcK {
  static constexpr int K = (M == TcMode::TF32 || M == TcMode::X3TF32) ? 8 : 16;
};

// B operand of one MMA step, converted once (it depends only on the atom, not on the grid row).
template <TcMode M>
struct BFrag {
  uint32_t hi[2];
  uint32_t lo[2];  // used by the split forms
};

// Build the B fragment from this lane's FP32 B elements (fragment order, see tc_product).
template <TcMode M>
__device__ __forceinline__ BFrag<M> make_bfrag(const float* b) {
  BFrag<M> f;
  if constexpr (M == TcMode::TF32) {
    f.hi[0] = tf32_bits(b[0]);
    f.hi[1] = tf32_bits(b[1]);
    f.lo[0] = f.lo[1] = 0u;
  } else if constexpr (M == TcMode::X3TF32) {
    tf32_split(b[0], f.hi[0], f.lo[0]);
    tf32_split(b[1], f.hi[1], f.lo[1]);
  } else if constexpr (M == TcMode::BF16) {
    f.hi[0] = pack_bf16(b[0], b[1]);
    f.hi[1] = pack_bf16(b[2], b[3]);
    f.lo[0] = f.lo[1] = 0u;
  } else {
    float bh[4], bl[4];
#pragma unroll
    for (int i = 0; i < 4; i++) f16_split(b[i], bh[i], bl[i]);
    f.hi[0] = pack_f16(bh[0], bh[1]);
    f.hi[1] = pack_f16(bh[2], bh[3]);
    f.lo[0] = pack_f16(bl[0], bl[1]);
    f.lo[1] = pack_f16(bl[2], bl[3]);
  }
  return f;
}

// One warp-tile product  D[16 x 8] += A[16 x K] B[K x 8]  in the given precision form.  `a` holds the
// four (TF32) or eight (16-bit) FP32 A elements of this lane in fragment order; for the split forms
// dlo collects the correction products (scaled by tc_lo_scale when combined).
//   TF32 order    a: (g,t) (g+8,t) (g,t+4) (g+8,t+4)                        b: (t,g) (t+4,g)
//   16-bit order  a: (g,2t) (g,2t+1) (g+8,2t) (g+8,2t+1) (g,2t+8) (g,2t+9) (g+8,2t+8) (g+8,2t+9)
//                 b: (2t,g) (2t+1,g) (2t+8,g) (2t+9,g)
template <TcMode M>
__device__ __forceinline__ void tc_product(float (&d)[4], float (&dlo)[4], const float* a, const BFrag<M>& b) {
  if constexpr (M == TcMode::TF32) {
    const uint32_t af[4] = {tf32_bits(a[0]), tf32_bits(a[1]), tf32_bits(a[2]), tf32_bits(a[3])};
    mma_tf32(d, af, b.hi[0], b.hi[1]);
  } else if constexpr (M == TcMode::X3TF32) {
    uint32_t ah[4], al[4];
#pragma unroll
    for (int i = 0; i < 4; i++) tf32_split(a[i], ah[i], al[i]);
    mma_tf32(dlo, al, b.hi[0], b.hi[1]);
    mma_tf32(dlo, ah, b.lo[0], b.lo[1]);
    mma_tf32(d, ah, b.hi[0], b.hi[1]);
  } else if constexpr (M == TcMode::BF16) {
    const uint32_t af[4] = {pack_bf16(a[0], a[1]), pack_bf16(a[2], a[3]), pack_bf16(a[4], a[5]),
                            pack_bf16(a[6], a[7])};
    mma_bf16(d, af, b.hi[0], b.hi[1]);
  } else {
    float ah[8], al[8];
#pragma unroll
    for (int i = 0; i < 8; i++) f16_split(a[i], ah[i], al[i]);
    const uint32_t afh[4] = {pack_f16(ah[0], ah[1]), pack_f16(ah[2], ah[3]), pack_f16(ah[4], ah[5]),
                             pack_f16(ah[6], ah[7])};
    const uint32_t afl[4] = {pack_f16(al[0], al[1]), pack_f16(al[2], al[3]), pack_f16(al[4], al[5]),
                             pack_f16(al[6], al[7])};
    mma_f16(dlo, afl, b.hi[0], b.hi[1]);
    mma_f16(dlo, afh, b.lo[0], b.lo[1]);
    mma_f16(d, afh, b.hi[0], b.hi[1]);
  }
}

// A operand of one MMA step converted to the mode's operand type (hi and, for the split forms, lo
// parts), for reuse across several B tiles of the same rows.
template <TcMode M>
struct AFrag {
  uint32_t hi[4];
  uint32_t lo[4];  // used by the split forms
};

// Same conversions as tc_product applies to its A elements (fragment order as there).
template <TcMode M>
__device__ __forceinline__ AFrag<M> make_afrag(const float* a) {
  AFrag<M> f;
  if constexpr (M == TcMode::TF32) {
#pragma unroll
    for (int i = 0; i < 4; i++) {
      f.hi[i] = tf32_bits(a[i]);
      f.lo[i] = 0u;
    }
  } else if constexpr (M == TcMode::X3TF32) {
#pragma unroll
    for (int i = 0; i < 4; i++) tf32_split(a[i], f.hi[i], f.lo[i]);
  } else if constexpr (M == TcMode::BF16) {
#pragma unroll
    for (int i = 0; i < 4; i++) {
      f.hi[i] = pack_bf16(a[2 * i], a[2 * i + 1]);
      f.lo[i] = 0u;
    }
  } else {
    float ah[8], al[8];
#pragma unroll
    for (int i = 0; i < 8; i++) f16_split(a[i], ah[i], al[i]);
#pragma unroll
    for (int i = 0; i < 4; i++) {
      f.hi[i] = pack_f16(ah[2 * i], ah[2 * i + 1]);
      f.lo[i] = pack_f16(al[2 * i], al[2 * i + 1]);
    }
  }
  return f;
}

// tc_product with the A operand already converted (make_afrag); the same MMAs in the same order.
template <TcMode M>
__device__ __forceinline__ void tc_product_pre(float (&d)[4], float (&dlo)[4], const AFrag<M>& a,
                                               const BFrag<M>& b) {
  if constexpr (M == TcMode::TF32) {
    mma_tf32(d, a.hi, b.hi[0], b.hi[1]);
  } else if constexpr (M == TcMode::X3TF32) {
    mma_tf32(dlo, a.lo, b.hi[0], b.hi[1]);
    mma_tf32(dlo, a.hi, b.lo[0], b.lo[1]);
    mma_tf32(d, a.hi, b.hi[0], b.hi[1]);
  } else if constexpr (M == TcMode::BF16) {
    mma_bf16(d, a.hi, b.hi[0], b.hi[1]);
  } else {
    mma_f16(dlo, a.lo, b.hi[0], b.hi[1]);
    mma_f16(dlo, a.hi, b.lo[0], b.lo[1]);
    mma_f16(d, a.hi, b.hi[0], b.hi[1]);
  }
}

// Scale applied to the correction accumulator before it is added to the main one.
template <TcMode M>
__device__ __forceinline__ float tc_lo_scale() {
  return M == TcMode::SPLIT16 ? (1.0f / 2048.0f) : 1.0f;
}

// Number of A / B elements per lane per MMA step.
template <TcMode M>
struct TcFrag {
  static constexpr int NA = (M == TcMode::TF32 || M == TcMode::X3TF32) ? 4 : 8;
  static constexpr int NB = (M == TcMode::TF32 || M == TcMode::X3TF32) ? 2 : 4;
};

// Row (m) and column (k) of A element i of this lane (g = lane / 4, t = lane % 4).
template <TcMode M>
__device__ __forceinline__ void a_coord(int i, int g, int t, int& m, int& k) {
  if constexpr (TcFrag<M>::NA == 4) {
    m = g + ((i & 1) ? 8 : 0);
    k = t + ((i & 2) ? 4 : 0);
  } else {
    m = g + ((i & 2) ? 8 : 0);
    k = 2 * t + (i & 1) + ((i & 4) ? 8 : 0);
  }
}

// Row (k) and column (n) of B element i of this lane.
template <TcMode M>
__device__ __forceinline__ void b_coord(int i, int g, int t, int& k, int& n) {
  n = g;
  if constexpr (TcFrag<M>::NB == 2) {
    k = t + (i ? 4 : 0);
  } else {
    k = 2 * t + (i & 1) + ((i & 2) ? 8 : 0);
  }
}

}  // namespace sho
