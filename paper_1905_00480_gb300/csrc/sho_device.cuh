// sho_device.cuh -- device helpers shared by the SHO kernels: on-the-fly 1D function tables,
// storage-type conversion and compile-time basis indexing.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "sho_internal.h"

namespace sho {

// Device checks: true when 0 <= i < n; otherwise sets kStatusBounds in *flag and returns false, and the
// caller skips the access.  Compiled to `true` in the unchecked kernels.
template <bool CHK>
__device__ __forceinline__ bool dc_ok(long long i, long long n, int* flag) {
  if constexpr (!CHK) {
    return true;
  } else {
    if ((unsigned long long)i < (unsigned long long)n) return true;
    atomicOr(flag, kStatusBounds);
    return false;
  }
}

// ---------------------------------------------------------------------------------------------
// Compile-time basis bookkeeping for numax NU (eq. SHO-basis / SHO_basis_size, Sec. 2.5).
//   pairs (nx, ny) with nx + ny <= NU: ny outer, nx inner
//   states (nx, ny, nz) with nx + ny + nz <= NU: nz outer, ny middle, nx inner
template <int NU>
struct Basis {
  static constexpr int NP = NU + 1;                               // 1D functions per axis
  static constexpr int P = (NU + 1) * (NU + 2) / 2;               // (nx, ny) pairs
  static constexpr int N = (NU + 1) * (NU + 2) * (NU + 3) / 6;    // 3D states
  // index of pair (nx, ny)
  __host__ __device__ static constexpr int pair(int nx, int ny) { return ny * (NU + 1) - ny * (ny - 1) / 2 + nx; }
  // index of state (nx, ny, nz)
  __host__ __device__ static constexpr int state(int nx, int ny, int nz) {
    int k = 0;
    for (int z = 0; z < nz; z++) k += (NU - z + 1) * (NU - z + 2) / 2;
    for (int y = 0; y < ny; y++) k += NU - nz - y + 1;
    return k + nx;
  }
};

// Runtime state index (nx, ny, nz) within the basis of numax nu (same order as Basis<NU>::state).
__host__ __device__ inline int state_index(int nu, int nx, int ny, int nz) {
  int k = 0;
  for (int z = 0; z < nz; z++) k += (nu - z + 1) * (nu - z + 2) / 2;
  for (int y = 0; y < ny; y++) k += nu - nz - y + 1;
  return k + nx;
}

// ---------------------------------------------------------------------------------------------
// Storage conversions.
__device__ __forceinline__ double to_real(double v, double) { return v; }
__device__ __forceinline__ double to_real(float v, double) { return (double)v; }
__device__ __forceinline__ float to_real(float v, float) { return v; }
__device__ __forceinline__ float to_real(double v, float) { return (float)v; }
__device__ __forceinline__ float to_real(__nv_bfloat16 v, float) { return __bfloat162float(v); }
__device__ __forceinline__ double to_real(__nv_bfloat16 v, double) { return (double)__bfloat162float(v); }

template <typename T>
__device__ __forceinline__ T from_real(double v);
template <>
__device__ __forceinline__ double from_real<double>(double v) { return v; }
template <>
__device__ __forceinline__ float from_real<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_real<__nv_bfloat16>(double v) { return __float2bfloat16_rn((float)v); }
__device__ __forceinline__ double store_cast(double v, double*) { return v; }
__device__ __forceinline__ float store_cast(float v, float*) { return v; }
__device__ __forceinline__ float store_cast(double v, float*) { return (float)v; }
__device__ __forceinline__ __nv_bfloat16 store_cast(float v, __nv_bfloat16*) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ double store_cast(float v, double*) { return (double)v; }

// ---------------------------------------------------------------------------------------------
// Cube geometry along one axis: grid index of cube point i, or -1 when dropped (not periodic).
__device__ __forceinline__ int cube_index(int o, int i, int n, int periodic) {
  int j = o + i;
  if (periodic) {
    j %= n;  // C remainder keeps the sign of j; fold negatives into [0, n)
    if (j < 0) j += n;
    return j;
  }
  return (j >= 0 && j < n) ? j : -1;
}

// Offset of cube point i from the atom, u = (o + i) h - X, rounded exactly as written
// (no contraction into an FMA), so that both cube conventions agree bit for bit.
__device__ __forceinline__ double cube_offset(int o, int i, double h, double X) {
  return __dsub_rn(__dmul_rn((double)(o + i), h), X);
}

// Spherical support (projection spheres of radius R, Sec. 6): is the cube point with offsets (ux, uy, uz)
// inside, (ux^2 + uy^2) + uz^2 <= R^2, each product and sum rounded to FP64 in that order?
__device__ __forceinline__ bool sphere_inside(double ux, double uy, double uz, double r2max) {
  return __dadd_rn(__dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy)), __dmul_rn(uz, uz)) <= r2max;
}

// Bit i set: cube point i of cube row (iy, iz) of atom `at` is in its support (all C bits without a
// sphere).  The points inside form one contiguous run of the row.  Warp-collective (full warp): lane l
// decides points l and l + 32.
__device__ __forceinline__ unsigned long long row_support(const GridDev& g, const AtomDev& at, int iy, int iz,
                                                          int lane) {
  const int C = g.cube;
  const unsigned long long all = C >= 64 ? ~0ull : ((1ull << C) - 1ull);
  if (!(g.r2max > 0.0)) return all;
  const double uy = cube_offset(at.o[1], iy, g.h, at.X[1]);
  const double uz = cube_offset(at.o[2], iz, g.h, at.X[2]);
  const bool in0 = lane < C && sphere_inside(cube_offset(at.o[0], lane, g.h, at.X[0]), uy, uz, g.r2max);
  const bool in1 = lane + 32 < C && sphere_inside(cube_offset(at.o[0], lane + 32, g.h, at.X[0]), uy, uz, g.r2max);
  return (unsigned long long)__ballot_sync(0xffffffffu, in0) |
         ((unsigned long long)__ballot_sync(0xffffffffu, in1) << 32);
}

// First and one-past-last set bit of a support mask (lo = hi = 0 when empty).
__device__ __forceinline__ void support_run(unsigned long long m, int& lo, int& hi) {
  lo = m ? __ffsll((long long)m) - 1 : 0;
  hi = m ? 64 - __clzll((long long)m) : 0;
}

// Normalised 1D oscillator functions phi_0 .. phi_nmax at offset u (FP64):
//   phi_0 = (sigma sqrt(pi))^(-1/2) exp(-xi^2/2),  xi = u / sigma
//   phi_1 = sqrt(2) xi phi_0
//   phi_{n+1} = sqrt(2/(n+1)) xi phi_n - sqrt(n/(n+1)) phi_{n-1}
// This is the Hermite recursion of Sec. 3.7 (h_{n+1} = x h_n - (n/2) h_{n-1}) carried by the
// normalised functions, so no factorials or powers of two are formed.  out[n * stride].
template <typename T>
__device__ __forceinline__ void phi_column(double u, double sigma, int nmax, T* out, int stride) {
  const double xi = u / sigma;
  const double inv_norm0 = 1.0 / sqrt(sigma * 1.7724538509055160273);  // sqrt(pi)
  double pm = 0.0;
  double p = inv_norm0 * exp(-0.5 * xi * xi);
  out[0] = (T)p;
  for (int n = 0; n < nmax; n++) {
    const double a = sqrt(2.0 / (double)(n + 1));
    const double b = sqrt((double)n / (double)(n + 1));
    const double pn = a * xi * p - b * pm;
    pm = p;
    p = pn;
    out[(n + 1) * stride] = (T)p;
  }
}

}  // namespace sho
