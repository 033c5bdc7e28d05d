// sho_project.cu -- SHO projection on CUDA cores (FP64 and FP32 forms).
//
//   coeff[a][k][b] = h^3 sum_{cube points} Psi_k(u) psi[j][b]        (Sec. 3.2 step 1, Sec. 3.5)
//
// evaluated as the separable three-pass contraction of eq. TuckerTensor (Sec. 3.4):
//   x-pass  T1[z][y][nx][b]      = sum_x psi[z][y][x][b] phi_nx(x)             C^3 (numax+1) FMAs
//   y-pass  T2[z][(nx,ny)][b]    = sum_y T1 phi_ny(y),  nx + ny <= numax       C^2 P FMAs
//   z-pass  C[(nx,ny,nz)][b]    += sum_z T2 phi_nz(z),  nx + ny + nz <= numax  C N FMAs
// with the 1D functions generated in shared memory from the Hermite recursion (Sec. 3.7), so no
// projector data is read from memory.
//
// Work decomposition: one warp per (atom, 32-band tile, slab of cube z-planes); lane = band, so
// every psi load of a warp is 32 consecutive bands of one grid point (coalesced).  The z-slabs of one
// (atom, band tile) form a thread-block cluster; their partial coefficients are summed in a fixed
// order through distributed shared memory, so the result is deterministic and needs no global
// scratch memory.
#include <cooperative_groups.h>

#include "sho_device.cuh"

namespace cg = cooperative_groups;

namespace sho {

template <int NU>
struct ProjectSmem {
  static constexpr int NP = NU + 1;
  static constexpr int NPX = (NP + 1) & ~1;  // x table row padded to an even count (16-byte rows)
  template <typename TC>
  static size_t bytes(int cube) {
    size_t t = (size_t)cube * NPX * sizeof(TC) + 2 * (size_t)NP * cube * sizeof(TC);
    t = (t + 15) & ~(size_t)15;
    t += (size_t)cube * sizeof(long long);
    t = (t + 15) & ~(size_t)15;
    t += (size_t)Basis<NU>::N * kWarp * sizeof(TC);
    return t;
  }
};

// SPH: spherical support (one support mask per cube row); compiled separately so that the cube form keeps
// its plain inner loop.
// CHK: device checks of every psi and coefficient index (sho_set_device_checks), a separate instantiation.
template <int NU, typename TP, typename TC, bool SPH = false, bool CHK = false>
__global__ void __launch_bounds__(kWarp) k_project(GridDev g, const TP* __restrict__ psi,
                                                   const AtomDev* __restrict__ atoms, int zsplit,
                                                   TC* __restrict__ coeff, DevCheck dc) {
  using BS = Basis<NU>;
  constexpr int NP = BS::NP, P = BS::P, N = BS::N;
  constexpr int NPX = ProjectSmem<NU>::NPX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int C = g.cube;
  TC* phx = reinterpret_cast<TC*>(smem_raw);       // [C][NPX]  x functions, state index fastest
  TC* phy = phx + (size_t)C * NPX;                  // [NP][C]
  TC* phz = phy + (size_t)NP * C;                   // [NP][C]
  size_t off_bytes = ((size_t)C * NPX + 2 * (size_t)NP * C) * sizeof(TC);
  off_bytes = (off_bytes + 15) & ~(size_t)15;
  long long* xoff = reinterpret_cast<long long*>(smem_raw + off_bytes);  // [C] psi offset of x point
  off_bytes += (size_t)C * sizeof(long long);
  off_bytes = (off_bytes + 15) & ~(size_t)15;
  TC* acc = reinterpret_cast<TC*>(smem_raw + off_bytes);                 // [N][32] partial coefficients

  const int lane = threadIdx.x;
  const int a = blockIdx.z;
  const int B = g.nbands;
  const int b = blockIdx.y * kWarp + lane;
  const bool bok = b < B;
  const AtomDev at = atoms[a];

  // 1D function tables for the three axes (a1): one lane per cube point.
  for (int i = lane; i < C; i += kWarp) {
    phi_column(cube_offset(at.o[0], i, g.h, at.X[0]), at.sigma, NU, phx + (size_t)i * NPX, 1);
    phi_column(cube_offset(at.o[1], i, g.h, at.X[1]), at.sigma, NU, phy + i, C);
    phi_column(cube_offset(at.o[2], i, g.h, at.X[2]), at.sigma, NU, phz + i, C);
    const int jx = cube_index(at.o[0], i, g.n[0], g.periodic);
    xoff[i] = jx < 0 ? -1ll : (long long)jx * B;
  }
  for (int i = lane; i < N * kWarp; i += kWarp) acc[i] = (TC)0;
  __syncwarp();

  const int chunk = (C + zsplit - 1) / zsplit;
  const int iz0 = blockIdx.x * chunk;
  const int iz1 = min(C, iz0 + chunk);
  const long long rowlen = (long long)g.n[0] * B;

  for (int iz = iz0; iz < iz1; iz++) {
    const int jz = cube_index(at.o[2], iz, g.n[2], g.periodic);
    if (jz < 0) continue;
    TC t2[P];
#pragma unroll
    for (int p = 0; p < P; p++) t2[p] = (TC)0;
    for (int iy = 0; iy < C; iy++) {
      const int jy = cube_index(at.o[1], iy, g.n[1], g.periodic);
      if (jy < 0) continue;
      unsigned long long sup = ~0ull;
      if constexpr (SPH) {
        sup = row_support(g, at, iy, iz, lane);  // spherical support of the row
        if (sup == 0) continue;
      }
      const long long row0 = ((long long)jz * g.n[1] + jy) * rowlen + b;  // psi index of this row's x = 0
      const TP* row = psi + row0;
      // x-pass (a3)
      TC t1[NP];
#pragma unroll
      for (int n = 0; n < NP; n++) t1[n] = (TC)0;
      for (int ix = 0; ix < C; ix += 8) {
        if constexpr (SPH) {
          if (((sup >> ix) & 0xffull) == 0) continue;
        }
        TC v[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
          const long long o = xoff[ix + u];
          v[u] = (o >= 0 && bok && (!SPH || ((sup >> (ix + u)) & 1ull)) && dc_ok<CHK>(row0 + o, dc.psi_n, dc.flag))
                     ? to_real(row[o], (TC)0)
                     : (TC)0;
        }
#pragma unroll
        for (int u = 0; u < 8; u++) {
          const TC* f = phx + (size_t)(ix + u) * NPX;
#pragma unroll
          for (int n = 0; n < NP; n++) t1[n] = fma(v[u], f[n], t1[n]);
        }
      }
      // y-pass (a4)
#pragma unroll
      for (int ny = 0; ny < NP; ny++) {
        const TC w = phy[ny * C + iy];
#pragma unroll
        for (int nx = 0; nx + ny <= NU; nx++) t2[BS::pair(nx, ny)] = fma(t1[nx], w, t2[BS::pair(nx, ny)]);
      }
    }
    // z-pass (a5), accumulated over the slab's planes in shared memory
    int k = 0;
#pragma unroll
    for (int nz = 0; nz < NP; nz++) {
      const TC w = phz[nz * C + iz];
#pragma unroll
      for (int ny = 0; ny + nz <= NU; ny++) {
#pragma unroll
        for (int nx = 0; nx + ny + nz <= NU; nx++) {
          acc[k * kWarp + lane] = fma(t2[BS::pair(nx, ny)], w, acc[k * kWarp + lane]);
          k++;
        }
      }
    }
  }

  // Sum the slabs of the cluster in rank order (deterministic) and apply the h^3 weight.
  cg::cluster_group cl = cg::this_cluster();
  cl.sync();
  const int rank = (int)cl.block_rank();
  const TC h3 = (TC)(g.h * g.h * g.h);
  for (int k = rank; k < N; k += zsplit) {
    TC s = (TC)0;
    for (int r = 0; r < zsplit; r++) {
      const TC* rem = cl.map_shared_rank(acc, r);
      s += rem[k * kWarp + lane];
    }
    const long long ci = ((long long)a * N + k) * B + b;
    if (bok && dc_ok<CHK>(ci, dc.coeff_n, dc.flag)) coeff[ci] = s * h3;
  }
  cl.sync();
}

template <int NU, typename TP, typename TC, bool SPH = false, bool CHK = false>
static cudaError_t launch_project_t(const ProjectLaunch& p) {
  if constexpr (!CHK) {
    if (p.chk.flag) return launch_project_t<NU, TP, TC, SPH, true>(p);
  }
  const int C = p.g.cube;
  const size_t smem = ProjectSmem<NU>::template bytes<TC>(C);
  auto kern = k_project<NU, TP, TC, SPH, CHK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.zsplit, (p.g.nbands + kWarp - 1) / kWarp, p.natoms);
  cfg.blockDim = dim3(kWarp, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = p.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = p.zsplit;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, p.g, static_cast<const TP*>(p.psi), p.atoms, p.zsplit,
                            static_cast<TC*>(p.coeff), p.chk);
}

template <int NU>
static cudaError_t launch_project_nu(const ProjectLaunch& p) {
  if (p.coeff_dtype == SHO_F64) {
    if (p.psi_dtype == SHO_F64)
      return p.g.r2max > 0.0 ? launch_project_t<NU, double, double, true>(p) : launch_project_t<NU, double, double>(p);
    return cudaErrorInvalidValue;
  }
  if (p.g.r2max > 0.0) return cudaErrorInvalidValue;  // spherical support: FP64 forms only
  if (p.psi_dtype == SHO_F32) return launch_project_t<NU, float, float>(p);
  if (p.psi_dtype == SHO_BF16) return launch_project_t<NU, __nv_bfloat16, float>(p);
  return cudaErrorInvalidValue;
}

cudaError_t launch_project(const ProjectLaunch& p) {
  switch (p.numax) {
    case 0: return launch_project_nu<0>(p);
    case 1: return launch_project_nu<1>(p);
    case 2: return launch_project_nu<2>(p);
    case 3: return launch_project_nu<3>(p);
    case 4: return launch_project_nu<4>(p);
    case 5: return launch_project_nu<5>(p);
    case 6: return launch_project_nu<6>(p);
    case 7: return launch_project_nu<7>(p);
    case 8: return launch_project_nu<8>(p);
    case 9: return launch_project_nu<9>(p);
    case 10: return launch_project_nu<10>(p);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sho
