// sho_usu.cu -- stored-projector baseline (the conventional scheme the paper compares with, "USU" in
// Sec. 6, in double and float as its Tables 1 and 2): the projector values Psi_k(u_i) of every atom are
// sampled once onto its cube and stored in device memory, [A][C^3][N] of the compute type; projection
// and expansion then stream them from memory instead of generating the 1D functions on the fly.  Same cube convention, same band-major psi, same
// deterministic decomposition as the SHO kernels (cluster-reduced z-slabs; row gather), so the two
// differ only in where the projector values come from.
#include <cooperative_groups.h>

#include "sho_device.cuh"

namespace cg = cooperative_groups;

namespace sho {

// --------------------------------------------------------------------------------- build
template <typename T, int NU>
__global__ void __launch_bounds__(128) k_usu_build(GridDev g, const AtomDev* __restrict__ atoms, int nproj,
                                                   T* __restrict__ proj) {
  using BS = Basis<NU>;
  constexpr int NP = BS::NP;
  const int C = g.cube;
  const long long c3 = (long long)C * C * C;
  const int a = blockIdx.y;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c3) return;
  const AtomDev at = atoms[a];
  const int ix = (int)(i % C), iy = (int)((i / C) % C), iz = (int)(i / ((long long)C * C));
  double fx[NP], fy[NP], fz[NP];
  phi_column(cube_offset(at.o[0], ix, g.h, at.X[0]), at.sigma, NU, fx, 1);
  phi_column(cube_offset(at.o[1], iy, g.h, at.X[1]), at.sigma, NU, fy, 1);
  phi_column(cube_offset(at.o[2], iz, g.h, at.X[2]), at.sigma, NU, fz, 1);
  T* out = proj + ((long long)a * c3 + i) * nproj;
  // spherical support: stored values outside the atom's projection sphere are zero
  const bool in = !(g.r2max > 0.0) ||
                  sphere_inside(cube_offset(at.o[0], ix, g.h, at.X[0]), cube_offset(at.o[1], iy, g.h, at.X[1]),
                                cube_offset(at.o[2], iz, g.h, at.X[2]), g.r2max);
  int k = 0;
#pragma unroll
  for (int nz = 0; nz < NP; nz++)
#pragma unroll
    for (int ny = 0; ny + nz <= NU; ny++)
#pragma unroll
      for (int nx = 0; nx + ny + nz <= NU; nx++) {
        if (k < nproj) out[k] = in ? (T)(fx[nx] * fy[ny] * fz[nz]) : (T)0;
        k++;
      }
}

// --------------------------------------------------------------------------------- project
// BPL consecutive bands per lane (1 in double; 2 or 4 in float, where the stored values -- one load per
// grid point and state, shared by the warp -- would otherwise outnumber the FMAs they feed).
template <typename T, int BPL>
__device__ __forceinline__ void usu_load(const T* p, bool full, int valid, T (&v)[BPL]) {
  if (BPL == 4 && full) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x;
    v[1] = q.y;
    v[2 % BPL] = q.z;
    v[3 % BPL] = q.w;
  } else if (BPL == 2 && full) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    v[0] = q.x;
    v[1 % BPL] = q.y;
  } else {
#pragma unroll
    for (int j = 0; j < BPL; j++) v[j] = j < valid ? p[j] : (T)0;
  }
}

template <typename T, int N, int BPL>
__global__ void __launch_bounds__(kWarp) k_usu_project(GridDev g, const T* __restrict__ psi,
                                                       const AtomDev* __restrict__ atoms,
                                                       const T* __restrict__ proj, int zsplit,
                                                       T* __restrict__ coeff) {
  __shared__ T acc[N * kWarp * BPL];
  const int C = g.cube;
  const int lane = threadIdx.x;
  const int a = blockIdx.z;
  const int B = g.nbands;
  const int b = (blockIdx.y * kWarp + lane) * BPL;  // first band of this lane
  const int valid = min(BPL, B - b);               // bands of this lane inside [0, B)
  const bool full = valid == BPL;
  const AtomDev at = atoms[a];
  const long long c3 = (long long)C * C * C;
  const T* pa = proj + (long long)a * c3 * N;
  const int oxm = g.periodic ? ((at.o[0] % g.n[0]) + g.n[0]) % g.n[0] : at.o[0];
  T r[N][BPL];
#pragma unroll
  for (int k = 0; k < N; k++)
#pragma unroll
    for (int j = 0; j < BPL; j++) r[k][j] = (T)0;
  const int chunk = (C + zsplit - 1) / zsplit;
  const int iz0 = blockIdx.x * chunk, iz1 = min(C, iz0 + chunk);
  for (int iz = iz0; iz < iz1; iz++) {
    const int jz = cube_index(at.o[2], iz, g.n[2], g.periodic);
    if (jz < 0) continue;
    for (int iy = 0; iy < C; iy++) {
      const int jy = cube_index(at.o[1], iy, g.n[1], g.periodic);
      if (jy < 0) continue;
      const T* row = psi + ((long long)jz * g.n[1] + jy) * g.n[0] * B + b;
      // cube points of this row inside the grid (all when periodic, one contiguous run otherwise) and
      // inside the projection sphere (a contiguous run too; the stored values outside it are zero)
      int slo = 0, shi = C;
      if (g.r2max > 0.0) support_run(row_support(g, at, iy, iz, lane), slo, shi);
      const int ix0 = max(slo, g.periodic ? 0 : max(0, -at.o[0]));
      const int ix1 = min(shi, g.periodic ? C : min(C, g.n[0] - at.o[0]));
#pragma unroll 4
      for (int ix = ix0; ix < ix1; ix++) {
        int jx = oxm + ix;  // periodic: oxm in [0, Nx) and ix < C <= Nx, so one wrap at most
        if (g.periodic && jx >= g.n[0]) jx -= g.n[0];
        T v[BPL];
        if (valid > 0) usu_load<T, BPL>(row + (long long)jx * B, full, valid, v);
        else
#pragma unroll
          for (int j = 0; j < BPL; j++) v[j] = (T)0;
        const T* p = pa + (((long long)iz * C + iy) * C + ix) * N;
#pragma unroll
        for (int k = 0; k < N; k++) {
          const T w = __ldg(p + k);
#pragma unroll
          for (int j = 0; j < BPL; j++) r[k][j] = fma(w, v[j], r[k][j]);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < N; k++)
#pragma unroll
    for (int j = 0; j < BPL; j++) acc[(k * kWarp + lane) * BPL + j] = r[k][j];
  cg::cluster_group cl = cg::this_cluster();
  cl.sync();
  const int rank = (int)cl.block_rank();
  const T h3 = (T)(g.h * g.h * g.h);
  for (int k = rank; k < N; k += zsplit)
#pragma unroll
    for (int j = 0; j < BPL; j++) {
      T s = (T)0;
      for (int q = 0; q < zsplit; q++) s += cl.map_shared_rank(acc, q)[(k * kWarp + lane) * BPL + j];
      if (j < valid) coeff[((long long)a * N + k) * B + b + j] = s * h3;
    }
  cl.sync();
}

// --------------------------------------------------------------------------------- add (row gather)
template <typename T, int N, int BPL>
__global__ void __launch_bounds__(kWarp) k_usu_add(GridDev g, const AtomDev* __restrict__ atoms,
                                                   const int* __restrict__ plane_ptr,
                                                   const int* __restrict__ plane_atoms,
                                                   const T* __restrict__ proj,
                                                   const T* __restrict__ coeff, T* __restrict__ psi) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* acc = reinterpret_cast<T*>(smem_raw);  // [Nx][32 * BPL]
  const int C = g.cube;
  const int Nx = g.n[0], Ny = g.n[1];
  const int lane = threadIdx.x;
  const int r = blockIdx.x;
  const int z = r / Ny, y = r - z * Ny;
  const int B = g.nbands;
  const int b = (blockIdx.y * kWarp + lane) * BPL;
  const int valid = min(BPL, B - b);
  const int q0 = plane_ptr[z], q1 = plane_ptr[z + 1];
  bool any = false;
  for (int q = q0; q < q1 && !any; q++) {
    int iy = y - atoms[plane_atoms[q]].o[1];
    if (g.periodic) {
      iy %= Ny;
      if (iy < 0) iy += Ny;
    }
    any = (iy >= 0 && iy < C);
  }
  if (!any) return;
  T* row = psi + (long long)r * Nx * B + b;
  for (int jx = 0; jx < Nx; jx++)
#pragma unroll
    for (int j = 0; j < BPL; j++) acc[(jx * kWarp + lane) * BPL + j] = j < valid ? row[(long long)jx * B + j] : (T)0;
  const long long c3 = (long long)C * C * C;
  for (int q = q0; q < q1; q++) {
    const int a = plane_atoms[q];
    const AtomDev at = atoms[a];
    int iy = y - at.o[1], iz = z - at.o[2];
    if (g.periodic) {
      iy %= Ny;
      if (iy < 0) iy += Ny;
      iz %= g.n[2];
      if (iz < 0) iz += g.n[2];
    }
    if (iy < 0 || iy >= C) continue;
    T cr[N][BPL];
    const T* ca = coeff + (long long)a * N * B + b;
#pragma unroll
    for (int k = 0; k < N; k++)
#pragma unroll
      for (int j = 0; j < BPL; j++) cr[k][j] = j < valid ? ca[(long long)k * B + j] : (T)0;
    const T* pa = proj + ((long long)a * c3 + ((long long)iz * C + iy) * C) * N;
    int slo = 0, shi = C;  // projection-sphere run of the row (stored values outside it are zero)
    if (g.r2max > 0.0) support_run(row_support(g, at, iy, iz, lane), slo, shi);
    const int ix0 = max(slo, g.periodic ? 0 : max(0, -at.o[0])), ix1 = min(shi, g.periodic ? C : min(C, Nx - at.o[0]));
    const int oxm = g.periodic ? ((at.o[0] % Nx) + Nx) % Nx : at.o[0];
#pragma unroll 4
    for (int ix = ix0; ix < ix1; ix++) {
      int jx = oxm + ix;  // periodic: one wrap at most
      if (g.periodic && jx >= Nx) jx -= Nx;
      const T* p = pa + (long long)ix * N;
      T sv[BPL];
#pragma unroll
      for (int j = 0; j < BPL; j++) sv[j] = (T)0;
#pragma unroll
      for (int k = 0; k < N; k++) {
        const T w = __ldg(p + k);
#pragma unroll
        for (int j = 0; j < BPL; j++) sv[j] = fma(cr[k][j], w, sv[j]);
      }
#pragma unroll
      for (int j = 0; j < BPL; j++) acc[(jx * kWarp + lane) * BPL + j] += sv[j];
    }
  }
  for (int jx = 0; jx < Nx; jx++)
#pragma unroll
    for (int j = 0; j < BPL; j++)
      if (j < valid) row[(long long)jx * B + j] = acc[(jx * kWarp + lane) * BPL + j];
}

template <typename T, int NU>
static cudaError_t usu_build_nu(const UsuLaunch& p) {
  const long long c3 = (long long)p.g.cube * p.g.cube * p.g.cube;
  k_usu_build<T, NU><<<dim3((unsigned)((c3 + 127) / 128), p.natoms), 128, 0, p.stream>>>(p.g, p.atoms, p.nproj,
                                                                                        static_cast<T*>(p.proj));
  return cudaGetLastError();
}

template <typename T, int N, int BPL>
static cudaError_t usu_run_nb(int op, const UsuLaunch& p) {
  const int nbt = (p.g.nbands + kWarp * BPL - 1) / (kWarp * BPL);
  if (op == 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p.zsplit, nbt, p.natoms);
    cfg.blockDim = dim3(kWarp, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = p.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = p.zsplit;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_usu_project<T, N, BPL>, p.g, static_cast<const T*>(p.psi_in), p.atoms,
                              static_cast<const T*>(p.proj), p.zsplit, static_cast<T*>(p.coeff_out));
  }
  auto kern = k_usu_add<T, N, BPL>;
  const size_t smem = (size_t)p.g.n[0] * kWarp * BPL * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<dim3(p.g.n[1] * p.g.n[2], nbt), kWarp, smem, p.stream>>>(p.g, p.atoms, p.plane_ptr, p.plane_atoms,
                                                                  static_cast<const T*>(p.proj),
                                                                  static_cast<const T*>(p.coeff_in),
                                                                  static_cast<T*>(p.psi_out));
  return cudaGetLastError();
}

// Bands per lane: 1 in double; in float 4 (up to 20 stored values per point) or 2, when the band rows
// are aligned for vector loads (nbands a multiple of BPL, 16-byte aligned psi) and, for the expansion,
// the row buffer [Nx][32 BPL] fits in shared memory.
template <typename T, int N>
static cudaError_t usu_run_n(int op, const UsuLaunch& p) {
  if constexpr (sizeof(T) == 4) {
    const void* ps = op == 1 ? p.psi_in : (const void*)p.psi_out;
    const bool aligned = ((uintptr_t)ps & 15u) == 0;
    const int want = N <= 20 ? 4 : 2;
    const size_t row_limit = 200 * 1024;
    auto fits = [&](int bpl) {
      return p.g.nbands % bpl == 0 && aligned &&
             (op == 1 || (size_t)p.g.n[0] * kWarp * bpl * sizeof(T) <= row_limit);
    };
    if constexpr (N <= 20) {
      if (want == 4 && fits(4)) return usu_run_nb<T, N, 4>(op, p);
    }
    if (fits(2)) return usu_run_nb<T, N, 2>(op, p);
  }
  return usu_run_nb<T, N, 1>(op, p);
}

template <typename T>
static cudaError_t launch_usu_t(int op, const UsuLaunch& p) {
  if (op == 0) {
    switch (p.numax) {
      case 0: return usu_build_nu<T, 0>(p);
      case 1: return usu_build_nu<T, 1>(p);
      case 2: return usu_build_nu<T, 2>(p);
      case 3: return usu_build_nu<T, 3>(p);
      case 4: return usu_build_nu<T, 4>(p);
      case 5: return usu_build_nu<T, 5>(p);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (p.nproj) {
    case 1: return usu_run_n<T, 1>(op, p);
    case 4: return usu_run_n<T, 4>(op, p);
    case 10: return usu_run_n<T, 10>(op, p);
    case 18: return usu_run_n<T, 18>(op, p);
    case 20: return usu_run_n<T, 20>(op, p);
    case 35: return usu_run_n<T, 35>(op, p);
    case 56: return usu_run_n<T, 56>(op, p);
    default: return cudaErrorInvalidValue;
  }
}

// Stored-projector counts with compiled kernels: the SHO basis sizes of numax 0..5 and 18 (the
// s, s*, p, p*, d, d* set of a transition metal, Sec. 6).
bool usu_supported_nproj(int n) {
  return n == 1 || n == 4 || n == 10 || n == 18 || n == 20 || n == 35 || n == 56;
}

cudaError_t launch_usu(int op, const UsuLaunch& p) {
  return p.dtype == SHO_F32 ? launch_usu_t<float>(op, p) : launch_usu_t<double>(op, p);
}

}  // namespace sho
