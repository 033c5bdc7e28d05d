// sho_expand.cu -- SHO expansion on CUDA cores (FP64 and FP32 forms).
//
//   psi[j][b] += sum_a sum_k coeff[a][k][b] Psi_k(u)          (Sec. 3.2 step 3; adjoint of projection)
//
// evaluated with the passes of the projection in reverse order (z, then y, then x):
//   z-pass  T2[a][z][(nx,ny)][b] = sum_nz coeff[a][(nx,ny,nz)][b] phi_nz(z)      C N FMAs per atom-band
//   y-pass  T1[nx]               = sum_ny T2[(nx,ny)] phi_ny(y)                  C^2 P
//   x-pass  psi[z][y][x][b]     += sum_nx T1[nx] phi_nx(x)                       C^3 (numax+1)
//
// Kernel 1 (one warp per atom and 32-band tile) runs the z-pass and writes the x and y function
// tables; both go to the handle's workspace.  Kernel 2 is a gather over grid rows: one warp per
// (grid row (z, y), 32-band tile) loads the row once into shared memory, adds the y- and x-passes of
// every atom whose cube covers the row in ascending atom order, and writes the row back once.  No
// atomics: every psi element is written by exactly one warp, in a fixed order (deterministic).
#include "sho_device.cuh"
#include "sho_ff.cuh"

namespace sho {

// ------------------------------------------------------------------------------ kernel 1: z-pass
constexpr int kZChunk = 4;  // planes per shared-memory chunk of the band-tiled z-pass output

// TILED: T2 goes out band-tiled, [A][C][B/32][32][PP] with PP = tiled_pairs(P), zero for the padding
// pairs and for bands past B (the block-gather expansion stages one contiguous [32][PP] slice per
// atom and plane); otherwise [A][C][P][B].
// FFOUT (FP64-accurate form, TC = double): T2 goes out as float pairs in the same [A][C][P][B] slots
// (8 bytes each, the integer split of ff_from_double), a sum outside the float-pair range sets
// kStatusRange, and the x and y tables also go out as float pairs, x-major txff [A][C][NPX2] (NPX2 = NP
// rounded up to 2, zero padded) and tyff [A][NP][C].
template <int NU, typename TCo, typename TC, bool TILED = false, bool FFOUT = false>
__global__ void __launch_bounds__(kWarp) k_expand_zpass(GridDev g, const AtomDev* __restrict__ atoms,
                                                        const TCo* __restrict__ coeff, TC* __restrict__ tables,
                                                        TC* __restrict__ t2, TC* __restrict__ txm, double scale,
                                                        NonlocalIn nl, TC* __restrict__ tym = nullptr,
                                                        float2* __restrict__ txff = nullptr,
                                                        float2* __restrict__ tyff = nullptr,
                                                        int* __restrict__ status = nullptr) {
  using BS = Basis<NU>;
  constexpr int NP = BS::NP, P = BS::P, N = BS::N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int C = g.cube;
  TC* phz = reinterpret_cast<TC*>(smem_raw);  // [NP][C]
  // fused non-local action: unscaled z table [NP][C] (projection), then c and d as [N][32] columns
  TC* nls = phz + (size_t)NP * C + (TILED ? (size_t)kZChunk * kWarp * tiled_pairs(P) : 0);
  TC* pz = nls;
  TC* cs = pz + (nl.t2p ? (size_t)NP * C : 0);
  TC* ds = cs + (size_t)N * kWarp;
  const int lane = threadIdx.x;
  const int a = blockIdx.y;
  const int B = g.nbands;
  const int b = blockIdx.x * kWarp + lane;
  const bool bok = b < B;
  const AtomDev at = atoms[a];

  TC* tx = tables + (size_t)a * 2 * NP * C;  // [NP][C]
  TC* ty = tx + (size_t)NP * C;              // [NP][C]
  for (int i = lane; i < C; i += kWarp) {
    // z table times the caller's scale (psi += scale * E c), rounded once to the compute type
    double zc[NP];
    phi_column(cube_offset(at.o[2], i, g.h, at.X[2]), at.sigma, NU, zc, 1);
#pragma unroll
    for (int n = 0; n < NP; n++) phz[n * C + i] = (TC)(zc[n] * scale);
    if (nl.D && nl.t2p)
#pragma unroll
      for (int n = 0; n < NP; n++) pz[n * C + i] = (TC)zc[n];
    if (blockIdx.x == 0 && blockIdx.z == 0) {
      phi_column(cube_offset(at.o[0], i, g.h, at.X[0]), at.sigma, NU, tx + i, C);
      phi_column(cube_offset(at.o[1], i, g.h, at.X[1]), at.sigma, NU, ty + i, C);
      if (txm) {  // x table again, x-major [C][NPX] with NPX = NP rounded up to 4 (zero padded)
        constexpr int NPX = (NP + 3) & ~3;
        TC* row = txm + ((size_t)a * C + i) * NPX;
        phi_column(cube_offset(at.o[0], i, g.h, at.X[0]), at.sigma, NU, row, 1);
        for (int n = NP; n < NPX; n++) row[n] = (TC)0;
      }
      if (tym) {  // y table y-major [C][NPX] (tensor-memory expansion: a row's functions in 16-byte loads)
        constexpr int NPX = (NP + 3) & ~3;
        TC* row = tym + ((size_t)a * C + i) * NPX;
        phi_column(cube_offset(at.o[1], i, g.h, at.X[1]), at.sigma, NU, row, 1);
        for (int n = NP; n < NPX; n++) row[n] = (TC)0;
      }
      if constexpr (FFOUT) {  // the x and y tables as float pairs (each entry split once, in FP64)
        constexpr int NPX2 = (NP + 1) & ~1;
        double col[NP];
        phi_column(cube_offset(at.o[0], i, g.h, at.X[0]), at.sigma, NU, col, 1);
#pragma unroll
        for (int n = 0; n < NPX2; n++) {
          const ff f = n < NP ? ff_from_double_exact(col[n]) : ff{0.0f, 0.0f};
          txff[((size_t)a * C + i) * NPX2 + n] = make_float2(f.hi, f.lo);
        }
        phi_column(cube_offset(at.o[1], i, g.h, at.X[1]), at.sigma, NU, col, 1);
#pragma unroll
        for (int n = 0; n < NP; n++) {
          const ff f = ff_from_double_exact(col[n]);
          tyff[((size_t)a * NP + n) * C + i] = make_float2(f.hi, f.lo);
        }
      }
    }
  }
  __syncwarp();

  // coefficients of this (atom, band): from global memory, or (fused action) d = D c in shared memory
  const TCo* ca = coeff + (size_t)a * N * B + (bok ? b : 0);
  size_t cstr = (size_t)B;
  if (nl.D) {
    if (nl.t2p) {
      // the projection's z-pass over the per-plane sums, planes ascending (cube planes outside an open
      // grid, and every plane of a cube that misses the grid in y, contribute nothing)
      const TC* t2a = static_cast<const TC*>(nl.t2p) + (size_t)a * C * P * B + (bok ? b : 0);
      for (int k = 0; k < N; k++) cs[k * kWarp + lane] = (TC)0;
      const bool yrows = g.periodic || (at.o[1] < g.n[1] && at.o[1] + C > 0);
      if (bok && yrows) {
        if constexpr (N <= 56) {
          // accumulators in registers up to numax 5
          TC acc[N];
#pragma unroll
          for (int k = 0; k < N; k++) acc[k] = (TC)0;
          for (int iz = 0; iz < C; iz++) {
            if (cube_index(at.o[2], iz, g.n[2], g.periodic) < 0) continue;
            TC t2v[P];
#pragma unroll
            for (int p = 0; p < P; p++) t2v[p] = t2a[((size_t)iz * P + p) * B];
#pragma unroll
            for (int ny = 0; ny < NP; ny++)
#pragma unroll
              for (int nx = 0; nx + ny <= NU; nx++)
#pragma unroll
                for (int nz = 0; nx + ny + nz <= NU; nz++)
                  acc[BS::state(nx, ny, nz)] = fma(t2v[BS::pair(nx, ny)], pz[nz * C + iz], acc[BS::state(nx, ny, nz)]);
          }
#pragma unroll
          for (int k = 0; k < N; k++) cs[k * kWarp + lane] = acc[k];
        } else {
          for (int iz = 0; iz < C; iz++) {
            if (cube_index(at.o[2], iz, g.n[2], g.periodic) < 0) continue;
#pragma unroll
            for (int ny = 0; ny < NP; ny++)
#pragma unroll
              for (int nx = 0; nx + ny <= NU; nx++) {
                const TC v = t2a[((size_t)iz * P + BS::pair(nx, ny)) * B];
#pragma unroll
                for (int nz = 0; nx + ny + nz <= NU; nz++) {
                  const int k = BS::state(nx, ny, nz);
                  cs[k * kWarp + lane] = fma(v, pz[nz * C + iz], cs[k * kWarp + lane]);
                }
              }
          }
        }
      }
      const TC h3 = (TC)nl.h3;
      for (int k = 0; k < N; k++) cs[k * kWarp + lane] *= h3;
    } else {
      const TC* cg = static_cast<const TC*>(nl.c) + (size_t)a * N * B + (bok ? b : 0);
      for (int k = 0; k < N; k++) cs[k * kWarp + lane] = bok ? cg[(size_t)k * B] : (TC)0;
    }
    // d = D c (step 2 of the action), states k' ascending; eight output states at a time so that eight
    // independent FMA chains are in flight
    const TC* Da = static_cast<const TC*>(nl.D) + (size_t)a * N * N;
    for (int k0 = 0; k0 < N; k0 += 8) {
      TC acc[8];
#pragma unroll
      for (int j = 0; j < 8; j++) acc[j] = (TC)0;
      for (int kp = 0; kp < N; kp++) {
        const TC v = cs[kp * kWarp + lane];
#pragma unroll
        for (int j = 0; j < 8; j++)
          if (k0 + j < N) acc[j] = fma(__ldg(Da + (size_t)(k0 + j) * N + kp), v, acc[j]);
      }
#pragma unroll
      for (int j = 0; j < 8; j++)
        if (k0 + j < N) ds[(k0 + j) * kWarp + lane] = acc[j];
    }
    ca = reinterpret_cast<const TCo*>(ds + lane);
    cstr = kWarp;
  }
  if (!TILED && !bok) return;

  constexpr int PP = tiled_pairs(P);
  // planes of this block: its chunk of the cube's planes (the planes are independent here)
  const int zper = (C + (int)gridDim.z - 1) / (int)gridDim.z;
  const int zb = (int)blockIdx.z * zper, ze = min(C, zb + zper);
  if constexpr (!TILED) {
    TC* out = t2 + (size_t)a * C * P * B + b;
    bool range_bad = false;  // FFOUT: a sum the float pairs cannot carry
#pragma unroll
    for (int ny = 0; ny < NP; ny++) {
#pragma unroll
      for (int nx = 0; nx + ny <= NU; nx++) {
        TC cz[NP];
#pragma unroll
        for (int nz = 0; nz < NP; nz++)
          cz[nz] = (nx + ny + nz <= NU) ? to_real(ca[(size_t)BS::state(nx, ny, nz) * cstr], (TC)0) : (TC)0;
        const int p = BS::pair(nx, ny);
        for (int iz = zb; iz < ze; iz++) {
          TC s = (TC)0;
#pragma unroll
          for (int nz = 0; nz + nx + ny <= NU; nz++) s = fma(cz[nz], phz[nz * C + iz], s);
          if constexpr (FFOUT) {
            range_bad |= ff_out_of_range((double)s);
            const ff f = ff_from_double((double)s);  // integer split: no FP64-pipe work per element
            reinterpret_cast<float2*>(out)[((size_t)iz * P + p) * B] = make_float2(f.hi, f.lo);
          } else {
            out[((size_t)iz * P + p) * B] = s;
          }
        }
      }
    }
    if constexpr (FFOUT) {
      if (range_bad && status) atomicOr(status, kStatusRange);
    }
  } else {
    // band-tiled: kZChunk planes at a time are assembled in shared memory as [plane][32][PP] (this
    // lane's row of pairs, zero padded) and each plane's [32][PP] slice, contiguous in T2, is written
    // with 16-byte stores (a lane-strided store per pair would leave DRAM sectors half written)
    TC* stage = phz + (size_t)NP * C;  // [kZChunk][32][PP]
    const size_t nbt = gridDim.x;
    for (int z0 = zb; z0 < ze; z0 += kZChunk) {
      const int nzc = min(kZChunk, ze - z0);
#pragma unroll
      for (int ny = 0; ny < NP; ny++) {
#pragma unroll
        for (int nx = 0; nx + ny <= NU; nx++) {
          TC cz[NP];
#pragma unroll
          for (int nz = 0; nz < NP; nz++)
            cz[nz] = (bok && nx + ny + nz <= NU) ? to_real(ca[(size_t)BS::state(nx, ny, nz) * cstr], (TC)0) : (TC)0;
          const int p = BS::pair(nx, ny);
          for (int i = 0; i < nzc; i++) {
            TC s = (TC)0;
#pragma unroll
            for (int nz = 0; nz + nx + ny <= NU; nz++) s = fma(cz[nz], phz[nz * C + z0 + i], s);
            stage[((size_t)i * kWarp + lane) * PP + p] = s;
          }
        }
      }
      for (int i = 0; i < nzc; i++)
#pragma unroll
        for (int p = P; p < PP; p++) stage[((size_t)i * kWarp + lane) * PP + p] = (TC)0;
      __syncwarp();
      for (int i = 0; i < nzc; i++) {
        const float4* src = reinterpret_cast<const float4*>(stage + (size_t)i * kWarp * PP);
        float4* dst = reinterpret_cast<float4*>(t2 + (((size_t)a * C + z0 + i) * nbt + blockIdx.x) * kWarp * PP);
        for (int q = lane; q < kWarp * PP / 4; q += kWarp) dst[q] = src[q];
      }
      __syncwarp();
    }
  }
}

// ------------------------------------------------------------------------------ kernel 2: rows
// SPH: spherical support (one support mask per atom row), compiled separately from the cube form.
// CHK: device checks of every psi and z-pass-result index (sho_set_device_checks), a separate instantiation.
template <int NU, typename TP, typename TC, bool SPH = false, bool CHK = false>
__global__ void __launch_bounds__(kWarp) k_expand_rows(GridDev g, const AtomDev* __restrict__ atoms,
                                                       const int* __restrict__ plane_ptr,
                                                       const int* __restrict__ plane_atoms,
                                                       const TC* __restrict__ tables, const TC* __restrict__ t2,
                                                       TP* __restrict__ psi, DevCheck dc) {
  using BS = Basis<NU>;
  constexpr int NP = BS::NP, P = BS::P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* acc = reinterpret_cast<TC*>(smem_raw);  // [Nx][32]
  const int C = g.cube;
  const int Nx = g.n[0], Ny = g.n[1];
  const int lane = threadIdx.x;
  const int r = blockIdx.x;
  const int z = r / Ny, y = r - z * Ny;
  const int B = g.nbands;
  const int b = blockIdx.y * kWarp + lane;
  const bool bok = b < B;
  const int q0 = plane_ptr[z], q1 = plane_ptr[z + 1];

  // Does any atom's cube cover this row?  (Rows outside every cube are not touched at all.)
  bool any = false;
  for (int q = q0; q < q1 && !any; q++) {
    const int oy = atoms[plane_atoms[q]].o[1];
    int iy = y - oy;
    if (g.periodic) {
      iy %= Ny;
      if (iy < 0) iy += Ny;
    }
    any = (iy >= 0 && iy < C);
  }
  if (!any) return;

  const long long row0 = (long long)r * Nx * B + b;  // psi index of this row's x = 0
  TP* row = psi + row0;
  for (int jx = 0; jx < Nx; jx++)
    acc[jx * kWarp + lane] =
        (bok && dc_ok<CHK>(row0 + (long long)jx * B, dc.psi_n, dc.flag)) ? to_real(row[(size_t)jx * B], (TC)0) : (TC)0;

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
    unsigned long long sup = ~0ull;
    if constexpr (SPH) {
      sup = row_support(g, at, iy, iz, lane);  // spherical support of the row
      if (sup == 0) continue;
    }
    const TC* tx = tables + (size_t)a * 2 * NP * C;
    const TC* ty = tx + (size_t)NP * C;
    // y-pass (a6, middle pass)
    const long long t20 = ((long long)a * C + iz) * P * B + b;
    const TC* t2a = t2 + t20;
    TC t2r[P];
#pragma unroll
    for (int p = 0; p < P; p++)
      t2r[p] = (bok && dc_ok<CHK>(t20 + (long long)p * B, dc.t2_n, dc.flag)) ? t2a[(size_t)p * B] : (TC)0;
    TC t1[NP];
#pragma unroll
    for (int nx = 0; nx < NP; nx++) t1[nx] = (TC)0;
#pragma unroll
    for (int ny = 0; ny < NP; ny++) {
      const TC w = ty[ny * C + iy];
#pragma unroll
      for (int nx = 0; nx + ny <= NU; nx++) t1[nx] = fma(t2r[BS::pair(nx, ny)], w, t1[nx]);
    }
    // x-pass (a6, last pass) into the row accumulator: eight x points at a time, each chain seeded
    // with the accumulator value, so eight independent FMA chains are in flight and every point
    // costs exactly numax+1 FMAs.
    for (int ix0 = 0; ix0 < C; ix0 += 8) {
      if constexpr (SPH) {
        if (((sup >> ix0) & 0xffull) == 0) continue;
      }
      int jx[8];
      TC s[8];
#pragma unroll
      for (int u = 0; u < 8; u++) {
        jx[u] = (!SPH || ((sup >> (ix0 + u)) & 1ull)) ? cube_index(at.o[0], ix0 + u, Nx, g.periodic) : -1;
        s[u] = jx[u] >= 0 ? acc[jx[u] * kWarp + lane] : (TC)0;
      }
#pragma unroll
      for (int nx = 0; nx < NP; nx++) {
        const TC w = t1[nx];
#pragma unroll
        for (int u = 0; u < 8; u++) s[u] = fma(w, tx[nx * C + ix0 + u], s[u]);
      }
#pragma unroll
      for (int u = 0; u < 8; u++)
        if (jx[u] >= 0) acc[jx[u] * kWarp + lane] = s[u];
    }
  }
  if (bok)
    for (int jx = 0; jx < Nx; jx++)
      if (dc_ok<CHK>(row0 + (long long)jx * B, dc.psi_n, dc.flag))
        row[(size_t)jx * B] = store_cast(acc[jx * kWarp + lane], (TP*)nullptr);
}

// Shared memory of k_expand_zpass beyond its z table (and band-tiled staging): the fused action's unscaled
// z table and its c and d columns.
template <int NU, typename TC>
static size_t nl_smem(const ExpandLaunch& p) {
  if (!p.nl.D) return 0;
  return ((p.nl.t2p ? (size_t)(NU + 1) * p.g.cube : 0) + 2 * (size_t)Basis<NU>::N * kWarp) * sizeof(TC);
}

// Plane chunks of the expansion's z-pass (grid z): enough warps for the GPU when the (atom, band tile)
// warps alone are few; one chunk when the fused action's prologue runs (it needs every plane), and chunks
// of whole kZChunk planes.
static unsigned zpass_chunks(const ExpandLaunch& p) {
  if (p.nl.D) return 1;
  const long long warps = (long long)p.natoms * ((p.g.nbands + kWarp - 1) / kWarp);
  unsigned n = 1;
  while (warps * n * 2 <= 4096 && (int)(n * 2) * kZChunk <= p.g.cube) n *= 2;
  return n;
}

template <typename K>
static cudaError_t zpass_smem(K kern, size_t smem) {
  return smem > 48 * 1024 ? cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                          : cudaSuccess;
}

template <int NU, typename TP, typename TCo, typename TC, bool SPH = false, bool CHK = false>
static cudaError_t launch_expand_t(const ExpandLaunch& p) {
  if constexpr (!CHK) {
    if (p.chk.flag) return launch_expand_t<NU, TP, TCo, TC, SPH, true>(p);
  }
  const int C = p.g.cube;
  const int nbt = (p.g.nbands + kWarp - 1) / kWarp;
  {
    const size_t smem = (size_t)(NU + 1) * C * sizeof(TC) + nl_smem<NU, TC>(p);
    cudaError_t e = zpass_smem(k_expand_zpass<NU, TCo, TC>, smem);
    if (e != cudaSuccess) return e;
    k_expand_zpass<NU, TCo, TC><<<dim3(nbt, p.natoms, zpass_chunks(p)), kWarp, smem, p.stream>>>(
        p.g, p.atoms, static_cast<const TCo*>(p.coeff), static_cast<TC*>(p.tables), static_cast<TC*>(p.t2),
        (TC*)nullptr, p.scale, p.nl);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  {
    auto kern = k_expand_rows<NU, TP, TC, SPH, CHK>;
    const size_t smem = (size_t)p.g.n[0] * kWarp * sizeof(TC);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(p.g.n[1] * p.g.n[2], nbt), kWarp, smem, p.stream>>>(
        p.g, p.atoms, p.plane_ptr, p.plane_atoms, static_cast<const TC*>(p.tables), static_cast<const TC*>(p.t2),
        static_cast<TP*>(p.psi), p.chk);
    return cudaGetLastError();
  }
}

template <int NU>
static cudaError_t launch_expand_nu(const ExpandLaunch& p) {
  if (p.coeff_dtype == SHO_F64) {
    if (p.psi_dtype == SHO_F64)
      return p.g.r2max > 0.0 ? launch_expand_t<NU, double, double, double, true>(p)
                             : launch_expand_t<NU, double, double, double>(p);
    return cudaErrorInvalidValue;
  }
  if (p.g.r2max > 0.0) return cudaErrorInvalidValue;  // spherical support: FP64 forms only
  if (p.psi_dtype == SHO_F32) return launch_expand_t<NU, float, float, float>(p);
  if (p.psi_dtype == SHO_BF16) return launch_expand_t<NU, __nv_bfloat16, float, float>(p);
  return cudaErrorInvalidValue;
}

template <int NU>
static cudaError_t zpass_f32_nu(const ExpandLaunch& p) {
  const int nbt = (p.g.nbands + kWarp - 1) / kWarp;
  const size_t smem = (size_t)(NU + 1) * p.g.cube * sizeof(float) + nl_smem<NU, float>(p);
  const cudaError_t e = zpass_smem(k_expand_zpass<NU, float, float>, smem);
  if (e != cudaSuccess) return e;
  k_expand_zpass<NU, float, float><<<dim3(nbt, p.natoms, zpass_chunks(p)), kWarp, smem, p.stream>>>(
      p.g, p.atoms, static_cast<const float*>(p.coeff), static_cast<float*>(p.tables), static_cast<float*>(p.t2),
      static_cast<float*>(p.tables_xmajor), p.scale, p.nl);
  return cudaGetLastError();
}

template <int NU>
static cudaError_t zpass_f32_tiled_nu(const ExpandLaunch& p) {
  const int nbt = (p.g.nbands + kWarp - 1) / kWarp;
  constexpr int PP = tiled_pairs(Basis<NU>::P);
  const size_t smem = (size_t)(NU + 1) * p.g.cube * sizeof(float) + (size_t)kZChunk * kWarp * PP * sizeof(float) +
                      nl_smem<NU, float>(p);
  const cudaError_t e = zpass_smem(k_expand_zpass<NU, float, float, true>, smem);
  if (e != cudaSuccess) return e;
  k_expand_zpass<NU, float, float, true><<<dim3(nbt, p.natoms, zpass_chunks(p)), kWarp, smem, p.stream>>>(
      p.g, p.atoms, static_cast<const float*>(p.coeff), static_cast<float*>(p.tables), static_cast<float*>(p.t2),
      static_cast<float*>(p.tables_xmajor), p.scale, p.nl, static_cast<float*>(p.tables_ymajor));
  return cudaGetLastError();
}

template <int NU>
static cudaError_t zpass_f64_nu(const ExpandLaunch& p) {
  const int nbt = (p.g.nbands + kWarp - 1) / kWarp;
  const size_t smem = (size_t)(NU + 1) * p.g.cube * sizeof(double) + nl_smem<NU, double>(p);
  const cudaError_t e = zpass_smem(k_expand_zpass<NU, double, double>, smem);
  if (e != cudaSuccess) return e;
  k_expand_zpass<NU, double, double><<<dim3(nbt, p.natoms, zpass_chunks(p)), kWarp, smem, p.stream>>>(
      p.g, p.atoms, static_cast<const double*>(p.coeff), static_cast<double*>(p.tables), static_cast<double*>(p.t2),
      (double*)nullptr, p.scale, p.nl);
  return cudaGetLastError();
}

template <int NU>
static cudaError_t zpass_ff_nu(const ExpandLaunch& p, float2* txff, float2* tyff) {
  const int nbt = (p.g.nbands + kWarp - 1) / kWarp;
  const size_t smem = (size_t)(NU + 1) * p.g.cube * sizeof(double) + nl_smem<NU, double>(p);
  auto kern = k_expand_zpass<NU, double, double, false, true>;
  const cudaError_t e = zpass_smem(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<dim3(nbt, p.natoms, zpass_chunks(p)), kWarp, smem, p.stream>>>(
      p.g, p.atoms, static_cast<const double*>(p.coeff), static_cast<double*>(p.tables), static_cast<double*>(p.t2),
      (double*)nullptr, p.scale, p.nl, (double*)nullptr, txff, tyff, p.status);
  return cudaGetLastError();
}

cudaError_t launch_expand_zpass_ff(const ExpandLaunch& p, float2* txff, float2* tyff) {
  switch (p.numax) {
    case 0: return zpass_ff_nu<0>(p, txff, tyff);
    case 1: return zpass_ff_nu<1>(p, txff, tyff);
    case 2: return zpass_ff_nu<2>(p, txff, tyff);
    case 3: return zpass_ff_nu<3>(p, txff, tyff);
    case 4: return zpass_ff_nu<4>(p, txff, tyff);
    case 5: return zpass_ff_nu<5>(p, txff, tyff);
    case 6: return zpass_ff_nu<6>(p, txff, tyff);
    case 7: return zpass_ff_nu<7>(p, txff, tyff);
    case 8: return zpass_ff_nu<8>(p, txff, tyff);
    case 9: return zpass_ff_nu<9>(p, txff, tyff);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_expand_zpass_f64(const ExpandLaunch& p) {
  switch (p.numax) {
    case 0: return zpass_f64_nu<0>(p);
    case 1: return zpass_f64_nu<1>(p);
    case 2: return zpass_f64_nu<2>(p);
    case 3: return zpass_f64_nu<3>(p);
    case 4: return zpass_f64_nu<4>(p);
    case 5: return zpass_f64_nu<5>(p);
    case 6: return zpass_f64_nu<6>(p);
    case 7: return zpass_f64_nu<7>(p);
    case 8: return zpass_f64_nu<8>(p);
    case 9: return zpass_f64_nu<9>(p);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_expand_zpass_f32(const ExpandLaunch& p) {
  switch (p.numax) {
    case 0: return zpass_f32_nu<0>(p);
    case 1: return zpass_f32_nu<1>(p);
    case 2: return zpass_f32_nu<2>(p);
    case 3: return zpass_f32_nu<3>(p);
    case 4: return zpass_f32_nu<4>(p);
    case 5: return zpass_f32_nu<5>(p);
    case 6: return zpass_f32_nu<6>(p);
    case 7: return zpass_f32_nu<7>(p);
    case 8: return zpass_f32_nu<8>(p);
    case 9: return zpass_f32_nu<9>(p);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_expand_zpass_f32_tiled(const ExpandLaunch& p) {
  switch (p.numax) {
    case 0: return zpass_f32_tiled_nu<0>(p);
    case 1: return zpass_f32_tiled_nu<1>(p);
    case 2: return zpass_f32_tiled_nu<2>(p);
    case 3: return zpass_f32_tiled_nu<3>(p);
    case 4: return zpass_f32_tiled_nu<4>(p);
    case 5: return zpass_f32_tiled_nu<5>(p);
    case 6: return zpass_f32_tiled_nu<6>(p);
    case 7: return zpass_f32_tiled_nu<7>(p);
    case 8: return zpass_f32_tiled_nu<8>(p);
    case 9: return zpass_f32_tiled_nu<9>(p);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_expand(const ExpandLaunch& p) {
  switch (p.numax) {
    case 0: return launch_expand_nu<0>(p);
    case 1: return launch_expand_nu<1>(p);
    case 2: return launch_expand_nu<2>(p);
    case 3: return launch_expand_nu<3>(p);
    case 4: return launch_expand_nu<4>(p);
    case 5: return launch_expand_nu<5>(p);
    case 6: return launch_expand_nu<6>(p);
    case 7: return launch_expand_nu<7>(p);
    case 8: return launch_expand_nu<8>(p);
    case 9: return launch_expand_nu<9>(p);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sho
