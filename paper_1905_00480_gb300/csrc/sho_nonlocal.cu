// sho_nonlocal.cu -- step (2) of the non-local action (Sec. 3.2): d[a][k][b] = sum_k' D[a][k][k'] c[a][k'][b],
// with the atomic matrix in the SHO basis (Sec. 3.5, D = U^T F^T D F U, one N x N matrix per atom).
// One warp per (atom, 32-band tile, block of output states); lane = band, so every coefficient load is
// 32 consecutive bands; D rows are read as warp-uniform broadcasts.  Work is A N^2 B FMAs, under 1 % of a
// projection, so the kernel is kept simple.
#include "sho_device.cuh"

namespace sho {

template <typename T>
__global__ void __launch_bounds__(128) k_dmatrix(int natoms, int nstates, int nbands, const T* __restrict__ D,
                                                 const T* __restrict__ c, T* __restrict__ d) {
  const int a = blockIdx.z;
  const int b = blockIdx.x * kWarp + (threadIdx.x & 31);
  const int k0 = (blockIdx.y * 4 + (threadIdx.x >> 5)) * 8;  // 8 output states per warp
  if (b >= nbands || k0 >= nstates) return;
  const T* Da = D + (size_t)a * nstates * nstates;
  const T* ca = c + (size_t)a * nstates * nbands + b;
  T acc[8];
#pragma unroll
  for (int j = 0; j < 8; j++) acc[j] = (T)0;
  for (int kp = 0; kp < nstates; kp++) {
    const T v = ca[(size_t)kp * nbands];
#pragma unroll
    for (int j = 0; j < 8; j++)
      if (k0 + j < nstates) acc[j] = fma(__ldg(Da + (size_t)(k0 + j) * nstates + kp), v, acc[j]);
  }
  T* da = d + (size_t)a * nstates * nbands + b;
#pragma unroll
  for (int j = 0; j < 8; j++)
    if (k0 + j < nstates) da[(size_t)(k0 + j) * nbands] = acc[j];
}

cudaError_t launch_dmatrix(int natoms, int nstates, int nbands, sho_dtype dt, const void* D, const void* c, void* d,
                           cudaStream_t s) {
  if (natoms == 0 || nbands == 0) return cudaSuccess;
  const dim3 grid((nbands + kWarp - 1) / kWarp, (nstates + 31) / 32, natoms);
  if (dt == SHO_F64)
    k_dmatrix<double><<<grid, 128, 0, s>>>(natoms, nstates, nbands, static_cast<const double*>(D),
                                           static_cast<const double*>(c), static_cast<double*>(d));
  else
    k_dmatrix<float><<<grid, 128, 0, s>>>(natoms, nstates, nbands, static_cast<const float*>(D),
                                          static_cast<const float*>(c), static_cast<float*>(d));
  return cudaGetLastError();
}

}  // namespace sho
