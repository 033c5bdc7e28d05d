// sho_forces.cu -- contraction of the numax+1 projection into position gradients.
//
// With C' the projection at numax + 1 (same cube, same origin), the ladder relation of the
// normalised Hermite functions, d phi_n/du = (1/sigma)[sqrt(n/2) phi_{n-1} - sqrt((n+1)/2) phi_{n+1}]
// (the derivative of the recursion of Sec. 3.7), and u = x - X give exactly, grid point by grid
// point,
//     d C_{n} / d X_d = (1/sigma) [ sqrt((n_d+1)/2) C'_{n + e_d} - sqrt(n_d/2) C'_{n - e_d} ].
// This kernel forms  dEdX[a][d] = sum_{k,b} dEdc[a][k][b] dC_k/dX_d  with one block per atom and a
// fixed-order FP64 tree reduction (deterministic).
#include "sho_device.cuh"

namespace sho {

constexpr int kForceThreads = 256;

template <typename TC, typename TCo>
__global__ void __launch_bounds__(kForceThreads) k_forces(int numax, int nbands, const AtomDev* __restrict__ atoms,
                                                          const TC* __restrict__ cp, const TCo* __restrict__ dEdc,
                                                          double* __restrict__ dEdX) {
  __shared__ int kup[kMaxStates][3];
  __shared__ int kdn[kMaxStates][3];
  __shared__ double sup[kMaxStates][3];
  __shared__ double sdn[kMaxStates][3];
  __shared__ double red[3][kForceThreads];
  const int a = blockIdx.x;
  const int t = threadIdx.x;
  const int N = (numax + 1) * (numax + 2) * (numax + 3) / 6;
  const int N1 = (numax + 2) * (numax + 3) * (numax + 4) / 6;
  const int B = nbands;

  // ladder index tables: state k = (nx, ny, nz) of numax  ->  k' of (n +- e_d) in numax + 1
  for (int k = t; k < N; k += kForceThreads) {
    int kk = 0, m[3] = {0, 0, 0};
    bool found = false;
    for (int nz = 0; nz <= numax && !found; nz++)
      for (int ny = 0; ny + nz <= numax && !found; ny++)
        for (int nx = 0; nx + ny + nz <= numax && !found; nx++) {
          if (kk == k) {
            m[0] = nx;
            m[1] = ny;
            m[2] = nz;
            found = true;
          }
          kk++;
        }
    for (int d = 0; d < 3; d++) {
      int up[3] = {m[0], m[1], m[2]};
      up[d] += 1;
      kup[k][d] = state_index(numax + 1, up[0], up[1], up[2]);
      sup[k][d] = sqrt(0.5 * (double)(m[d] + 1));
      if (m[d] > 0) {
        int dn[3] = {m[0], m[1], m[2]};
        dn[d] -= 1;
        kdn[k][d] = state_index(numax + 1, dn[0], dn[1], dn[2]);
        sdn[k][d] = sqrt(0.5 * (double)m[d]);
      } else {
        kdn[k][d] = -1;
        sdn[k][d] = 0.0;
      }
    }
  }
  __syncthreads();

  const TC* ca = cp + (size_t)a * N1 * B;
  const TCo* ga = dEdc + (size_t)a * N * B;
  double f[3] = {0.0, 0.0, 0.0};
  const long long total = (long long)N * B;
  for (long long idx = t; idx < total; idx += kForceThreads) {
    const int k = (int)(idx / B);
    const int b = (int)(idx - (long long)k * B);
    const double gk = (double)ga[idx];
#pragma unroll
    for (int d = 0; d < 3; d++) {
      double v = sup[k][d] * (double)ca[(size_t)kup[k][d] * B + b];
      if (kdn[k][d] >= 0) v -= sdn[k][d] * (double)ca[(size_t)kdn[k][d] * B + b];
      f[d] = fma(gk, v, f[d]);
    }
  }
  for (int d = 0; d < 3; d++) red[d][t] = f[d];
  __syncthreads();
  for (int s = kForceThreads / 2; s > 0; s >>= 1) {
    if (t < s)
      for (int d = 0; d < 3; d++) red[d][t] += red[d][t + s];
    __syncthreads();
  }
  if (t == 0) {
    const double inv_sigma = 1.0 / atoms[a].sigma;
    for (int d = 0; d < 3; d++) dEdX[3 * a + d] = red[d][0] * inv_sigma;
  }
}

cudaError_t launch_forces_contract(const ForcesLaunch& p) {
  if (p.natoms == 0) return cudaSuccess;
  if (p.coeff_dtype == SHO_F64)
    k_forces<double, double><<<p.natoms, kForceThreads, 0, p.stream>>>(
        p.numax, p.nbands, p.atoms, static_cast<const double*>(p.cp), static_cast<const double*>(p.dEdc), p.dEdX);
  else
    k_forces<float, float><<<p.natoms, kForceThreads, 0, p.stream>>>(
        p.numax, p.nbands, p.atoms, static_cast<const float*>(p.cp), static_cast<const float*>(p.dEdc), p.dEdX);
  return cudaGetLastError();
}

}  // namespace sho
