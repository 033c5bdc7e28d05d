// sho_tc.cu -- reduced-precision forms with the x-pass on tensor cores (TF32, 3xTF32, BF16, split-FP16).
//
// Same decomposition, cube convention and determinism as the CUDA-core kernels (sho_project.cu,
// sho_expand.cu); only the x-pass (C^3 (numax+1) of the C^3 (numax+1) + C^2 P + C N FMAs per atom-band)
// moves to warp-level MMA tiles with FP32 accumulation:
//   projection  T1[b][n] = sum_x psi[x][b] phi_n(x):  M = 16 bands, N = 8 states, K = x points;
//               the four accumulator fragments of a 32-band warp are transposed through shared memory
//               into the lane-per-band layout of the y- and z-passes (FP32 CUDA cores).
//   expansion   psi[x][b] += sum_n T1[b][n] phi_n(x):  M = 16 bands, N = 8 x points, K = states, the
//               grid-row accumulator in shared memory is the MMA's C operand.
// numax <= 7 (eight states per axis fill one N = 8 tile).  The 1D tables are generated in FP64 and
// rounded once to FP32 before the operand conversion.
#include <cooperative_groups.h>

#include "sho_tc.cuh"

namespace cg = cooperative_groups;

namespace sho {

constexpr int kT1Stride = 36;  // transpose buffer row stride: conflict-free fragment scatter

// ------------------------------------------------------------------------------- projection
template <int NU, typename TP, TcMode MODE>
__global__ void __launch_bounds__(kWarp) k_project_tc(GridDev g, const TP* __restrict__ psi,
                                                      const AtomDev* __restrict__ atoms, int zsplit,
                                                      float* __restrict__ coeff) {
  static_assert(NU <= 7, "one N = 8 tile");
  using BS = Basis<NU>;
  constexpr int NP = BS::NP, P = BS::P, N = BS::N;
  constexpr int K = TcK<MODE>::K;
  constexpr int NA = TcFrag<MODE>::NA, NB = TcFrag<MODE>::NB;
  constexpr int MAXSTEP = kMaxCube / K;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int C = g.cube;
  float* phx = reinterpret_cast<float*>(smem_raw);   // [NP][C]
  float* phy = phx + NP * C;                          // [NP][C]
  float* phz = phy + NP * C;                          // [NP][C]
  float* t1s = phz + NP * C;                          // [8][kT1Stride]
  float* acc = t1s + 8 * kT1Stride;                   // [N][32]
  long long* xoff = reinterpret_cast<long long*>(acc + N * kWarp);  // [C]

  const int lane = threadIdx.x, gq = lane >> 2, tq = lane & 3;
  const int a = blockIdx.z;
  const int B = g.nbands;
  const int b0 = blockIdx.y * kWarp;
  const bool bok = b0 + lane < B;
  const AtomDev at = atoms[a];

  for (int i = lane; i < C; i += kWarp) {
    phi_column(cube_offset(at.o[0], i, g.h, at.X[0]), at.sigma, NU, phx + i, C);
    phi_column(cube_offset(at.o[1], i, g.h, at.X[1]), at.sigma, NU, phy + i, C);
    phi_column(cube_offset(at.o[2], i, g.h, at.X[2]), at.sigma, NU, phz + i, C);
    const int jx = cube_index(at.o[0], i, g.n[0], g.periodic);
    xoff[i] = jx < 0 ? -1ll : (long long)jx * B;
  }
  for (int i = lane; i < N * kWarp; i += kWarp) acc[i] = 0.0f;
  __syncwarp();

  // B fragments (phi_n(x), K = x, N = n) for every K step of the cube row: fixed per atom.
  const int nsteps = C / K;
  BFrag<MODE> bf[MAXSTEP];
#pragma unroll
  for (int s = 0; s < MAXSTEP; s++) {
    if (s < nsteps) {
      float bv[NB];
#pragma unroll
      for (int i = 0; i < NB; i++) {
        int k, n;
        b_coord<MODE>(i, gq, tq, k, n);
        bv[i] = (n <= NU) ? phx[n * C + s * K + k] : 0.0f;
      }
      bf[s] = make_bfrag<MODE>(bv);
    }
  }

  const int chunk = (C + zsplit - 1) / zsplit;
  const int iz0 = blockIdx.x * chunk, iz1 = min(C, iz0 + chunk);
  const long long rowlen = (long long)g.n[0] * B;
  const float lo_scale = tc_lo_scale<MODE>();

  for (int iz = iz0; iz < iz1; iz++) {
    const int jz = cube_index(at.o[2], iz, g.n[2], g.periodic);
    if (jz < 0) continue;
    float t2[P];
#pragma unroll
    for (int p = 0; p < P; p++) t2[p] = 0.0f;
    for (int iy = 0; iy < C; iy++) {
      const int jy = cube_index(at.o[1], iy, g.n[1], g.periodic);
      if (jy < 0) continue;
      const TP* row = psi + ((long long)jz * g.n[1] + jy) * rowlen + b0;
      // x-pass (a3) on tensor cores: two 16-band tiles
      float d[2][4], dl[2][4];
#pragma unroll
      for (int m = 0; m < 2; m++)
#pragma unroll
        for (int j = 0; j < 4; j++) d[m][j] = dl[m][j] = 0.0f;
#pragma unroll
      for (int s = 0; s < MAXSTEP; s++) {
        if (s < nsteps) {
#pragma unroll
          for (int m = 0; m < 2; m++) {
            float av[NA];
#pragma unroll
            for (int i = 0; i < NA; i++) {
              int mm, k;
              a_coord<MODE>(i, gq, tq, mm, k);
              const long long o = xoff[s * K + k];
              const int band = 16 * m + mm;
              av[i] = (o >= 0 && b0 + band < B) ? to_real(row[o + band], 0.0f) : 0.0f;
            }
            tc_product<MODE>(d[m], dl[m], av, bf[s]);
          }
        }
      }
      // accumulator fragments -> t1s[n][band]
#pragma unroll
      for (int m = 0; m < 2; m++) {
        t1s[(2 * tq) * kT1Stride + 16 * m + gq] = d[m][0] + lo_scale * dl[m][0];
        t1s[(2 * tq + 1) * kT1Stride + 16 * m + gq] = d[m][1] + lo_scale * dl[m][1];
        t1s[(2 * tq) * kT1Stride + 16 * m + gq + 8] = d[m][2] + lo_scale * dl[m][2];
        t1s[(2 * tq + 1) * kT1Stride + 16 * m + gq + 8] = d[m][3] + lo_scale * dl[m][3];
      }
      __syncwarp();
      float t1[NP];
#pragma unroll
      for (int n = 0; n < NP; n++) t1[n] = t1s[n * kT1Stride + lane];
      __syncwarp();
      // y-pass (a4) on CUDA cores
#pragma unroll
      for (int ny = 0; ny < NP; ny++) {
        const float w = phy[ny * C + iy];
#pragma unroll
        for (int nx = 0; nx + ny <= NU; nx++) t2[BS::pair(nx, ny)] = fmaf(t1[nx], w, t2[BS::pair(nx, ny)]);
      }
    }
    // z-pass (a5)
    int k = 0;
#pragma unroll
    for (int nz = 0; nz < NP; nz++) {
      const float w = phz[nz * C + iz];
#pragma unroll
      for (int ny = 0; ny + nz <= NU; ny++)
#pragma unroll
        for (int nx = 0; nx + ny + nz <= NU; nx++) {
          acc[k * kWarp + lane] = fmaf(t2[BS::pair(nx, ny)], w, acc[k * kWarp + lane]);
          k++;
        }
    }
  }

  cg::cluster_group cl = cg::this_cluster();
  cl.sync();
  const int rank = (int)cl.block_rank();
  const float h3 = (float)(g.h * g.h * g.h);
  for (int k = rank; k < N; k += zsplit) {
    float sum = 0.0f;
    for (int r = 0; r < zsplit; r++) sum += cl.map_shared_rank(acc, r)[k * kWarp + lane];
    if (bok) coeff[((long long)a * N + k) * B + b0 + lane] = sum * h3;
  }
  cl.sync();
}

// ------------------------------------------------------------------------------- expansion rows
constexpr int kAccStride = 36;  // row accumulator stride (bands) for conflict-free C fragments

template <int NU, typename TP, TcMode MODE>
__global__ void __launch_bounds__(kWarp) k_expand_rows_tc(GridDev g, const AtomDev* __restrict__ atoms,
                                                          const int* __restrict__ plane_ptr,
                                                          const int* __restrict__ plane_atoms,
                                                          const float* __restrict__ tables,
                                                          const float* __restrict__ t2, TP* __restrict__ psi) {
  static_assert(NU <= 7, "one K tile of states");
  using BS = Basis<NU>;
  constexpr int NP = BS::NP, P = BS::P;
  constexpr int NA = TcFrag<MODE>::NA, NB = TcFrag<MODE>::NB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* t1s = reinterpret_cast<float*>(smem_raw);   // [16][kT1Stride]  (K up to 16, rows >= NP zero)
  float* acc = t1s + 16 * kT1Stride;                  // [Nx][kAccStride]
  const int C = g.cube;
  const int Nx = g.n[0], Ny = g.n[1];
  const int lane = threadIdx.x, gq = lane >> 2, tq = lane & 3;
  const int r = blockIdx.x;
  const int z = r / Ny, y = r - z * Ny;
  const int B = g.nbands;
  const int b0 = blockIdx.y * kWarp;
  const bool bok = b0 + lane < B;
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

  for (int i = lane; i < 16 * kT1Stride; i += kWarp) t1s[i] = 0.0f;
  TP* row = psi + (long long)r * Nx * B + b0;
  for (int jx = 0; jx < Nx; jx++) acc[jx * kAccStride + lane] = bok ? to_real(row[(long long)jx * B + lane], 0.0f) : 0.0f;
  __syncwarp();
  const float lo_scale = tc_lo_scale<MODE>();

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
    const float* tx = tables + (long long)a * 2 * NP * C;
    const float* ty = tx + NP * C;
    // y-pass (CUDA cores, lane = band)
    const float* t2a = t2 + ((long long)a * C + iz) * P * B + b0 + lane;
    float t1[NP];
#pragma unroll
    for (int n = 0; n < NP; n++) t1[n] = 0.0f;
#pragma unroll
    for (int ny = 0; ny < NP; ny++) {
      const float w = ty[ny * C + iy];
#pragma unroll
      for (int nx = 0; nx + ny <= NU; nx++)
        t1[nx] = fmaf(bok ? t2a[(long long)BS::pair(nx, ny) * B] : 0.0f, w, t1[nx]);
    }
#pragma unroll
    for (int n = 0; n < NP; n++) t1s[n * kT1Stride + lane] = t1[n];
    __syncwarp();
    // A fragments (T1, M = bands, K = states) of the two 16-band tiles
    float av[2][NA];
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
      for (int i = 0; i < NA; i++) {
        int mm, k;
        a_coord<MODE>(i, gq, tq, mm, k);
        av[m][i] = t1s[k * kT1Stride + 16 * m + mm];
      }
    __syncwarp();
    // x-pass: N tiles of 8 cube points, C operand = row accumulator
    for (int x0 = 0; x0 < C; x0 += 8) {
      float bv[NB];
#pragma unroll
      for (int i = 0; i < NB; i++) {
        int k, n;
        b_coord<MODE>(i, gq, tq, k, n);
        bv[i] = (k <= NU) ? tx[k * C + x0 + n] : 0.0f;
      }
      const BFrag<MODE> bfr = make_bfrag<MODE>(bv);
      const int ja = cube_index(at.o[0], x0 + 2 * tq, Nx, g.periodic);
      const int jb = cube_index(at.o[0], x0 + 2 * tq + 1, Nx, g.periodic);
#pragma unroll
      for (int m = 0; m < 2; m++) {
        const int bl = 16 * m + gq;
        float d[4], dl[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        d[0] = ja >= 0 ? acc[ja * kAccStride + bl] : 0.0f;
        d[1] = jb >= 0 ? acc[jb * kAccStride + bl] : 0.0f;
        d[2] = ja >= 0 ? acc[ja * kAccStride + bl + 8] : 0.0f;
        d[3] = jb >= 0 ? acc[jb * kAccStride + bl + 8] : 0.0f;
        tc_product<MODE>(d, dl, av[m], bfr);
        if (ja >= 0) {
          acc[ja * kAccStride + bl] = d[0] + lo_scale * dl[0];
          acc[ja * kAccStride + bl + 8] = d[2] + lo_scale * dl[2];
        }
        if (jb >= 0) {
          acc[jb * kAccStride + bl] = d[1] + lo_scale * dl[1];
          acc[jb * kAccStride + bl + 8] = d[3] + lo_scale * dl[3];
        }
      }
      __syncwarp();
    }
  }
  __syncwarp();
  if (bok)
    for (int jx = 0; jx < Nx; jx++) row[(long long)jx * B + lane] = store_cast(acc[jx * kAccStride + lane], (TP*)nullptr);
}

// ------------------------------------------------------------------------------- launchers
template <int NU, typename TP, TcMode MODE>
static cudaError_t project_tc_t(const ProjectLaunch& p) {
  constexpr int N = Basis<NU>::N;
  const int C = p.g.cube;
  const size_t smem = (3 * (size_t)(NU + 1) * C + 8 * kT1Stride + (size_t)N * kWarp) * sizeof(float) +
                      (size_t)C * sizeof(long long) + 16;
  auto kern = k_project_tc<NU, TP, MODE>;
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
                            static_cast<float*>(p.coeff));
}

template <int NU, typename TP, TcMode MODE>
static cudaError_t expand_tc_t(const ExpandLaunch& p) {
  const int nbt = (p.g.nbands + kWarp - 1) / kWarp;
  cudaError_t e = launch_expand_zpass_f32(p);
  if (e != cudaSuccess) return e;
  auto kern = k_expand_rows_tc<NU, TP, MODE>;
  const size_t smem = (16 * (size_t)kT1Stride + (size_t)p.g.n[0] * kAccStride) * sizeof(float);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<dim3(p.g.n[1] * p.g.n[2], nbt), kWarp, smem, p.stream>>>(
      p.g, p.atoms, p.plane_ptr, p.plane_atoms, static_cast<const float*>(p.tables), static_cast<const float*>(p.t2),
      static_cast<TP*>(p.psi));
  return cudaGetLastError();
}

template <int NU, TcMode MODE>
static cudaError_t tc_dispatch_dtype(int op, const ProjectLaunch* pp, const ExpandLaunch* pe) {
  const sho_dtype dt = op == 0 ? pp->psi_dtype : pe->psi_dtype;
  if (dt == SHO_F32) return op == 0 ? project_tc_t<NU, float, MODE>(*pp) : expand_tc_t<NU, float, MODE>(*pe);
  if (dt == SHO_BF16)
    return op == 0 ? project_tc_t<NU, __nv_bfloat16, MODE>(*pp) : expand_tc_t<NU, __nv_bfloat16, MODE>(*pe);
  return cudaErrorInvalidValue;
}

template <int NU>
static cudaError_t tc_dispatch_mode(int op, sho_prec prec, const ProjectLaunch* pp, const ExpandLaunch* pe) {
  switch (prec) {
    case SHO_P_TF32: return tc_dispatch_dtype<NU, TcMode::TF32>(op, pp, pe);
    case SHO_P_3XTF32: return tc_dispatch_dtype<NU, TcMode::X3TF32>(op, pp, pe);
    case SHO_P_BF16: return tc_dispatch_dtype<NU, TcMode::BF16>(op, pp, pe);
    case SHO_P_SPLIT_FP16: return tc_dispatch_dtype<NU, TcMode::SPLIT16>(op, pp, pe);
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t tc_dispatch(int op, int numax, sho_prec prec, const ProjectLaunch* pp, const ExpandLaunch* pe) {
  switch (numax) {
    case 0: return tc_dispatch_mode<0>(op, prec, pp, pe);
    case 1: return tc_dispatch_mode<1>(op, prec, pp, pe);
    case 2: return tc_dispatch_mode<2>(op, prec, pp, pe);
    case 3: return tc_dispatch_mode<3>(op, prec, pp, pe);
    case 4: return tc_dispatch_mode<4>(op, prec, pp, pe);
    case 5: return tc_dispatch_mode<5>(op, prec, pp, pe);
    case 6: return tc_dispatch_mode<6>(op, prec, pp, pe);
    case 7: return tc_dispatch_mode<7>(op, prec, pp, pe);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_project_tc(const ProjectLaunch& p, sho_prec prec) {
  return tc_dispatch(0, p.numax, prec, &p, nullptr);
}

cudaError_t launch_expand_tc(const ExpandLaunch& p, sho_prec prec) {
  return tc_dispatch(1, p.numax, prec, nullptr, &p);
}

}  // namespace sho
