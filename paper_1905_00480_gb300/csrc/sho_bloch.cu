// sho_bloch.cu -- projection and expansion of complex Bloch wave functions on a periodic grid (FP64).
//
// The SHO states span functions R^3 -> C (Sec. 2.5).  For a Bloch wave psi(r + T) = e^{i k.T} psi(r), a
// cube point i of an atom that lies outside the cell maps to grid point j(i) = r_i - T_i (T_i the lattice
// translation), so
//   projection  c[a][k][b] = h^3 sum_i Psi_k(u_i) e^{+i k.T_i} psi[j(i)][b]
//   expansion   psi[j][b] += sum_a sum_{i: j(i)=j} sum_k c[a][k][b] Psi_k(u_i) e^{-i k.T_i}
// The phase factorises over the axes (T_i = sum_d T_d(i_d)), so it rides on the 1D tables:
// phi~_n^d(i) = phi_n(u_d(i)) e^{i k_d T_d(i)}, and both operations keep the separable three-pass form of
// eq. TuckerTensor (Sec. 3.4) with complex tables and complex data (4 DFMA per complex FMA).
//   k_bloch_tables   per atom and axis: phi~ as (re, im) pairs
//   k_bloch_project  warp per (z-slab, 32 bands, atom): x, y passes in registers, z-pass into shared
//                    memory; the slab's partial coefficients go to a workspace
//   k_bloch_reduce   sums the slabs in fixed order and applies h^3
//   k_bloch_zpass    T2[a][iz][(nx,ny)][b] = sum_nz conj(phi~z) c  (expansion, per atom)
//   k_bloch_rows     warp per (grid row, 32 bands): y and x passes of every atom whose cube holds the
//                    row, in ascending atom order, into a shared row buffer; psi updated once
#include <algorithm>

#include "sho_device.cuh"

namespace sho {

struct cplx {
  double re, im;
};
__device__ __forceinline__ void cfma(cplx& acc, const cplx a, const cplx b) {  // acc += a b
  acc.re = fma(a.re, b.re, fma(-a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(a.im, b.re, acc.im));
}
__device__ __forceinline__ void cfma_conj(cplx& acc, const cplx a, const cplx b) {  // acc += conj(a) b
  acc.re = fma(a.re, b.re, fma(a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(-a.im, b.re, acc.im));
}
__device__ __forceinline__ cplx ld2(const double* p) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  return cplx{v.x, v.y};
}

// tab[a][d][n][i] (pairs): phi_n(u_d(i)) e^{i k_d T_d(i)}, T_d(i) = (o_d + i - j_d(i)) h
template <int NU>
__global__ void __launch_bounds__(kWarp) k_bloch_tables(GridDev g, const AtomDev* __restrict__ atoms, double3 kv,
                                                        double* __restrict__ tab) {
  constexpr int NP = NU + 1;
  const int a = blockIdx.x, C = g.cube;
  const AtomDev at = atoms[a];
  const double kd[3] = {kv.x, kv.y, kv.z};
  for (int i = threadIdx.x; i < C; i += kWarp)
    for (int d = 0; d < 3; d++) {
      double col[NP];
      phi_column(cube_offset(at.o[d], i, g.h, at.X[d]), at.sigma, NU, col, 1);
      const int j = cube_index(at.o[d], i, g.n[d], 1);
      const double shift = (double)(at.o[d] + i - j) * g.h;
      double sn, cs;
      sincos(kd[d] * shift, &sn, &cs);
      double* out = tab + (((size_t)a * 3 + d) * NP * C) * 2;
#pragma unroll
      for (int n = 0; n < NP; n++) {
        out[((size_t)n * C + i) * 2] = col[n] * cs;
        out[((size_t)n * C + i) * 2 + 1] = col[n] * sn;
      }
    }
}

template <int NU>
__global__ void __launch_bounds__(kWarp) k_bloch_project(GridDev g, const double* __restrict__ psi,
                                                         const AtomDev* __restrict__ atoms,
                                                         const double* __restrict__ tab, int zsplit,
                                                         double* __restrict__ part) {
  using BS = Basis<NU>;
  constexpr int NP = BS::NP, P = BS::P, N = BS::N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int C = g.cube, B = g.nbands, lane = threadIdx.x;
  const int a = blockIdx.z, b = blockIdx.y * kWarp + lane;
  const bool bok = b < B;
  double* ts = reinterpret_cast<double*>(smem_raw);           // [3][NP][C] pairs
  double* acc = ts + (size_t)3 * NP * C * 2;                   // [N][32] pairs
  const AtomDev at = atoms[a];
  const double* src = tab + (size_t)a * 3 * NP * C * 2;
  for (int q = lane; q < 3 * NP * C * 2; q += kWarp) ts[q] = src[q];
  for (int q = lane; q < N * kWarp * 2; q += kWarp) acc[q] = 0.0;
  __syncwarp();
  const double* tx = ts;
  const double* ty = ts + (size_t)NP * C * 2;
  const double* tz = ts + (size_t)2 * NP * C * 2;
  const int chunk = (C + zsplit - 1) / zsplit;
  const int iz0 = blockIdx.x * chunk, iz1 = min(C, iz0 + chunk);
  const int oxm = ((at.o[0] % g.n[0]) + g.n[0]) % g.n[0];
  for (int iz = iz0; iz < iz1; iz++) {
    const int jz = cube_index(at.o[2], iz, g.n[2], 1);
    cplx t2[P];
#pragma unroll
    for (int p = 0; p < P; p++) t2[p] = cplx{0.0, 0.0};
    for (int iy = 0; iy < C; iy++) {
      const int jy = cube_index(at.o[1], iy, g.n[1], 1);
      const double* row = psi + (((size_t)jz * g.n[1] + jy) * g.n[0] * B + b) * 2;
      cplx t1[NP];
#pragma unroll
      for (int n = 0; n < NP; n++) t1[n] = cplx{0.0, 0.0};
      for (int ix = 0; ix < C; ix++) {
        int jx = oxm + ix;
        if (jx >= g.n[0]) jx -= g.n[0];
        const cplx v = bok ? ld2(row + (size_t)jx * B * 2) : cplx{0.0, 0.0};
#pragma unroll
        for (int n = 0; n < NP; n++) cfma(t1[n], ld2(tx + ((size_t)n * C + ix) * 2), v);
      }
#pragma unroll
      for (int ny = 0; ny < NP; ny++) {
        const cplx w = ld2(ty + ((size_t)ny * C + iy) * 2);
#pragma unroll
        for (int nx = 0; nx + ny <= NU; nx++) cfma(t2[BS::pair(nx, ny)], w, t1[nx]);
      }
    }
    int k = 0;
#pragma unroll
    for (int nz = 0; nz < NP; nz++) {
      const cplx w = ld2(tz + ((size_t)nz * C + iz) * 2);
#pragma unroll
      for (int ny = 0; ny + nz <= NU; ny++)
#pragma unroll
        for (int nx = 0; nx + ny + nz <= NU; nx++) {
          cplx s = ld2(acc + ((size_t)k * kWarp + lane) * 2);
          cfma(s, w, t2[BS::pair(nx, ny)]);
          *reinterpret_cast<double2*>(acc + ((size_t)k * kWarp + lane) * 2) = make_double2(s.re, s.im);
          k++;
        }
    }
  }
  if (!bok) return;
  double* out = part + (((size_t)blockIdx.x * gridDim.z + a) * N * B + b) * 2;
  for (int k = 0; k < N; k++)
    *reinterpret_cast<double2*>(out + (size_t)k * B * 2) =
        *reinterpret_cast<const double2*>(acc + ((size_t)k * kWarp + lane) * 2);
}

// coeff[a][k][b] = h^3 sum over slabs s = 0 .. zsplit-1 (in order) of part[s][a][k][b]
__global__ void k_bloch_reduce(size_t count, int zsplit, double h3, const double* __restrict__ part,
                               double* __restrict__ coeff) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int s = 0; s < zsplit; s++) {
      re += part[((size_t)s * count + i) * 2];
      im += part[((size_t)s * count + i) * 2 + 1];
    }
    coeff[i * 2] = re * h3;
    coeff[i * 2 + 1] = im * h3;
  }
}

template <int NU>
__global__ void __launch_bounds__(kWarp) k_bloch_zpass(GridDev g, const double* __restrict__ tab,
                                                       const double* __restrict__ coeff, double* __restrict__ t2) {
  using BS = Basis<NU>;
  constexpr int NP = BS::NP, P = BS::P, N = BS::N;
  const int C = g.cube, B = g.nbands;
  const int a = blockIdx.y, b = blockIdx.x * kWarp + threadIdx.x;
  if (b >= B) return;
  const double* tz = tab + (((size_t)a * 3 + 2) * NP * C) * 2;
  const double* ca = coeff + ((size_t)a * N * B + b) * 2;
  double* out = t2 + ((size_t)a * C * P * B + b) * 2;
#pragma unroll
  for (int ny = 0; ny < NP; ny++)
#pragma unroll
    for (int nx = 0; nx + ny <= NU; nx++) {
      cplx cz[NP];
#pragma unroll
      for (int nz = 0; nz < NP; nz++)
        cz[nz] = (nx + ny + nz <= NU) ? ld2(ca + (size_t)BS::state(nx, ny, nz) * B * 2) : cplx{0.0, 0.0};
      const int p = BS::pair(nx, ny);
      for (int iz = 0; iz < C; iz++) {
        cplx s{0.0, 0.0};
#pragma unroll
        for (int nz = 0; nz + nx + ny <= NU; nz++) cfma_conj(s, ld2(tz + ((size_t)nz * C + iz) * 2), cz[nz]);
        *reinterpret_cast<double2*>(out + ((size_t)iz * P + p) * B * 2) = make_double2(s.re, s.im);
      }
    }
}

template <int NU>
__global__ void __launch_bounds__(kWarp) k_bloch_rows(GridDev g, const AtomDev* __restrict__ atoms,
                                                      const int* __restrict__ plane_ptr,
                                                      const int* __restrict__ plane_atoms,
                                                      const double* __restrict__ tab, const double* __restrict__ t2,
                                                      double* __restrict__ psi) {
  using BS = Basis<NU>;
  constexpr int NP = BS::NP, P = BS::P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* acc = reinterpret_cast<double*>(smem_raw);  // [Nx][32] pairs
  const int C = g.cube, B = g.nbands, lane = threadIdx.x;
  const int Nx = g.n[0], Ny = g.n[1], Nz = g.n[2];
  const int r = blockIdx.x, z = r / Ny, y = r - z * Ny;
  const int b = blockIdx.y * kWarp + lane;
  const bool bok = b < B;
  const int q0 = plane_ptr[z], q1 = plane_ptr[z + 1];
  bool any = false;
  for (int q = q0; q < q1 && !any; q++) {
    int iy = (y - atoms[plane_atoms[q]].o[1]) % Ny;
    if (iy < 0) iy += Ny;
    any = iy < C;
  }
  if (!any) return;
  for (int jx = 0; jx < Nx; jx++) *reinterpret_cast<double2*>(acc + ((size_t)jx * kWarp + lane) * 2) = make_double2(0.0, 0.0);
  for (int q = q0; q < q1; q++) {
    const int a = plane_atoms[q];
    const AtomDev at = atoms[a];
    int iy = (y - at.o[1]) % Ny, iz = (z - at.o[2]) % Nz;
    if (iy < 0) iy += Ny;
    if (iz < 0) iz += Nz;
    if (iy >= C) continue;
    const double* tx = tab + (((size_t)a * 3 + 0) * NP * C) * 2;
    const double* ty = tab + (((size_t)a * 3 + 1) * NP * C) * 2;
    const double* src = t2 + (((size_t)a * C + iz) * P * B + b) * 2;
    cplx t1[NP];
#pragma unroll
    for (int n = 0; n < NP; n++) t1[n] = cplx{0.0, 0.0};
#pragma unroll
    for (int ny = 0; ny < NP; ny++) {
      const cplx w = ld2(ty + ((size_t)ny * C + iy) * 2);
#pragma unroll
      for (int nx = 0; nx + ny <= NU; nx++) {
        const cplx v = bok ? ld2(src + (size_t)BS::pair(nx, ny) * B * 2) : cplx{0.0, 0.0};
        cfma_conj(t1[nx], w, v);
      }
    }
    const int oxm = ((at.o[0] % Nx) + Nx) % Nx;
    for (int ix = 0; ix < C; ix++) {
      int jx = oxm + ix;
      if (jx >= Nx) jx -= Nx;
      cplx s = ld2(acc + ((size_t)jx * kWarp + lane) * 2);
#pragma unroll
      for (int nx = 0; nx < NP; nx++) cfma_conj(s, ld2(tx + ((size_t)nx * C + ix) * 2), t1[nx]);
      *reinterpret_cast<double2*>(acc + ((size_t)jx * kWarp + lane) * 2) = make_double2(s.re, s.im);
    }
  }
  if (!bok) return;
  double* row = psi + (((size_t)z * Ny + y) * Nx * B + b) * 2;
  for (int jx = 0; jx < Nx; jx++) {
    double2 v = *reinterpret_cast<double2*>(row + (size_t)jx * B * 2);
    const double2 d = *reinterpret_cast<const double2*>(acc + ((size_t)jx * kWarp + lane) * 2);
    v.x += d.x;
    v.y += d.y;
    *reinterpret_cast<double2*>(row + (size_t)jx * B * 2) = v;
  }
}

// Phases of the real-kernel Bloch forms (BlochPh; FP64-accurate and FP32), one thread per atom: per axis the cube point w where
// floor((o + i) / n) steps from f0 to f0 + 1 (the cube crosses the cell boundary), and the eight
// e^{sgn i k.T} of the translations T_d = (f0_d + b_d) n_d h, split into float pairs.
__global__ void k_bloch_phases(GridDev g, const AtomDev* __restrict__ atoms, int natoms, double3 kv, double sgn,
                               BlochPh* __restrict__ out) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= natoms) return;
  const AtomDev at = atoms[a];
  const double kd[3] = {kv.x, kv.y, kv.z};
  BlochPh b;
  long long f0[3];
  for (int d = 0; d < 3; d++) {
    const long long n = g.n[d], o = at.o[d];
    f0[d] = o >= 0 ? o / n : -((-o + n - 1) / n);  // floor(o / n)
    b.w[d] = (int)((f0[d] + 1) * n - o);             // in [1, n]
  }
  b.w[3] = 0;
  auto put = [](double v, float& hi, float& lo) {
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
  };
  for (int bits = 0; bits < 8; bits++) {
    double ang = 0.0;
    for (int d = 0; d < 3; d++) ang += kd[d] * (double)(f0[d] + ((bits >> d) & 1)) * (double)g.n[d] * g.h;
    double sn, cs;
    sincos(sgn * ang, &sn, &cs);
    put(cs, b.ph[bits].x, b.ph[bits].y);
    put(sn, b.ph[bits].z, b.ph[bits].w);
  }
  double sn, cs;
  sincos(-sgn * kd[0] * (double)g.n[0] * g.h, &sn, &cs);
  put(cs, b.xstep.x, b.xstep.y);
  put(sn, b.xstep.z, b.xstep.w);
  out[a] = b;
}

cudaError_t launch_bloch_phases(const GridDev& g, const AtomDev* atoms, int natoms, const BlochArg& arg, BlochPh* ph,
                                cudaStream_t s) {
  if (natoms <= 0) return cudaSuccess;
  k_bloch_phases<<<(natoms + 63) / 64, 64, 0, s>>>(g, atoms, natoms, make_double3(arg.k[0], arg.k[1], arg.k[2]),
                                                  arg.sgn, ph);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------- launchers
template <int NU>
static cudaError_t bloch_nu(const BlochLaunch& p) {
  using BS = Basis<NU>;
  constexpr int NP = BS::NP, P = BS::P, N = BS::N;
  const int A = p.natoms, C = p.g.cube, B = p.g.nbands;
  const int nbt = (B + kWarp - 1) / kWarp;
  k_bloch_tables<NU><<<A, kWarp, 0, p.stream>>>(p.g, p.atoms, make_double3(p.k[0], p.k[1], p.k[2]), p.tab);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (p.op == 0) {
    const size_t smem = ((size_t)3 * NP * C + (size_t)N * kWarp) * 2 * sizeof(double);
    e = cudaFuncSetAttribute(k_bloch_project<NU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_bloch_project<NU><<<dim3(p.zsplit, nbt, A), kWarp, smem, p.stream>>>(p.g, p.psi_in, p.atoms, p.tab, p.zsplit,
                                                                           p.work);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t count = (size_t)A * N * B;
    k_bloch_reduce<<<(unsigned)std::min<size_t>((count + 255) / 256, 4096), 256, 0, p.stream>>>(
        count, p.zsplit, p.g.h * p.g.h * p.g.h, p.work, p.coeff_out);
    return cudaGetLastError();
  }
  k_bloch_zpass<NU><<<dim3(nbt, A), kWarp, 0, p.stream>>>(p.g, p.tab, p.coeff_in, p.work);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)p.g.n[0] * kWarp * 2 * sizeof(double);
  e = cudaFuncSetAttribute(k_bloch_rows<NU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_bloch_rows<NU><<<dim3(p.g.n[1] * p.g.n[2], nbt), kWarp, smem, p.stream>>>(p.g, p.atoms, p.plane_ptr, p.plane_atoms,
                                                                              p.tab, p.work, p.psi_out);
  (void)P;
  return cudaGetLastError();
}

cudaError_t launch_bloch(const BlochLaunch& p) {
  switch (p.numax) {
    case 0: return bloch_nu<0>(p);
    case 1: return bloch_nu<1>(p);
    case 2: return bloch_nu<2>(p);
    case 3: return bloch_nu<3>(p);
    case 4: return bloch_nu<4>(p);
    case 5: return bloch_nu<5>(p);
    case 6: return bloch_nu<6>(p);
    case 7: return bloch_nu<7>(p);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sho
