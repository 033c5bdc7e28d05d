// sho_noalloc.cu -- sho_forces_noalloc: the forces computation without any memory allocation.
//
// Some callers cannot let a library call cudaMalloc: an application whose own pool allocator owns
// all device memory and must account for every byte, a plug-in hosted inside a program that forbids
// foreign allocations, or a process running close to the memory limit that must not fail half-way
// through a step.  For them this entry point computes what sho_forces computes, but its scratch (the
// per-atom plan and the numax+1 projection) lives in one fixed, file-scope device array that is part
// of the library image.  The caller still owns and passes psi, dEdc and dEdX.  The projection runs on
// the generic per-atom kernels with the same slab split as sho_forces: for SHO_P_FP64 that is the same
// kernel and summation order as sho_forces; for SHO_P_FP32, where sho_forces may take the streaming
// kernels, the two agree within the FP32 form's tolerance, not bit for bit.
//
// The array is loaded with the library: every GPU that loads libsho.so holds
// SHO_NOALLOC_SCRATCH_BYTES of it until the process exits.  All calls on a device share it and it
// keeps the last call's contents; nothing in it needs to start at zero, because each call writes every
// element it later reads (the plan copy and the full projection) before reading it.  Two calls whose
// work overlaps on the GPU (different streams, no ordering between them) race on the array.
#include <cmath>
#include <mutex>
#include <vector>

#include "sho_internal.h"

namespace sho {
namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[SHO_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device
int g_sms[kMaxDevices] = {};

// Once per device, with that device current: look up the device address of the array.  In host
// code the array's name is only a host-side stand-in; kernels must be given this address instead.
int scratch_for_current_device(void** addr, int* sms) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SHO_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return SHO_ERR_CUDA;
    }
    int n = 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n = 1;
    g_scratch_addr[dev] = p;
    g_sms[dev] = n;
  }
  *addr = g_scratch_addr[dev];
  *sms = g_sms[dev];
  return SHO_OK;
}

int validate(const sho_grid* grid, const void* psi, sho_dtype psi_dtype, int nbands, int natoms,
             const double* pos, const double* sigma, int numax, int cube, sho_prec prec, const void* dEdc,
             sho_dtype coeff_dtype, const double* dEdX) {
  if (!grid || nbands < 0 || natoms < 0) return SHO_ERR_ARG;
  for (int d = 0; d < 3; d++)
    if (grid->n[d] <= 0) return SHO_ERR_ARG;
  if (!(grid->h > 0.0) || !std::isfinite(grid->h)) return SHO_ERR_ARG;
  if (natoms > 0 && (!pos || !sigma || !dEdX)) return SHO_ERR_ARG;
  if (natoms > 0 && nbands > 0 && (!psi || !dEdc)) return SHO_ERR_ARG;
  if (numax < 0 || numax > SHO_MAX_NUMAX) return SHO_ERR_NUMAX;
  if (cube < 8 || cube > kMaxCube || (cube % 8) != 0) return SHO_ERR_CUBE;
  if (grid->periodic)
    for (int d = 0; d < 3; d++)
      if (cube > grid->n[d]) return SHO_ERR_CUBE;
  for (int a = 0; a < natoms; a++) {
    if (!(sigma[a] > 0.0) || !std::isfinite(sigma[a])) return SHO_ERR_ARG;
    for (int d = 0; d < 3; d++)
      if (!std::isfinite(pos[3 * a + d])) return SHO_ERR_ARG;
  }
  if (prec == SHO_P_FP64) {
    if (psi_dtype != SHO_F64 || coeff_dtype != SHO_F64) return SHO_ERR_DTYPE;
  } else if (prec == SHO_P_FP32) {
    if ((psi_dtype != SHO_F32 && psi_dtype != SHO_BF16) || coeff_dtype != SHO_F32) return SHO_ERR_DTYPE;
  } else {
    return SHO_ERR_DTYPE;
  }
  return SHO_OK;
}

}  // namespace
}  // namespace sho

using namespace sho;

extern "C" int sho_forces_noalloc(const sho_grid* grid, const void* psi, sho_dtype psi_dtype, int nbands,
                                  int natoms, const double* pos, const double* sigma, int numax, int cube,
                                  sho_prec prec, const void* dEdc, sho_dtype coeff_dtype, double* dEdX,
                                  void* stream) {
  int st = validate(grid, psi, psi_dtype, nbands, natoms, pos, sigma, numax, cube, prec, dEdc, coeff_dtype, dEdX);
  if (st != SHO_OK) return st;
  if (natoms == 0) return SHO_OK;
  // Scratch layout: [AtomDev x natoms | 256-byte aligned | projection at numax+1, [A][N'][B]]
  const size_t tc = compute_size(coeff_dtype);
  const size_t atoms_bytes = ((size_t)natoms * sizeof(AtomDev) + 255) & ~(size_t)255;
  const size_t cp_bytes = (size_t)natoms * (size_t)nstates(numax + 1) * (size_t)nbands * tc;
  if (atoms_bytes + cp_bytes > (size_t)SHO_NOALLOC_SCRATCH_BYTES) return SHO_ERR_CAPACITY;

  void* base = nullptr;
  int sms = 1;
  st = scratch_for_current_device(&base, &sms);
  if (st != SHO_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (nbands == 0) {
    if (cudaMemsetAsync(dEdX, 0, sizeof(double) * 3 * (size_t)natoms, s) != cudaSuccess) return SHO_ERR_CUDA;
    return SHO_OK;
  }
  std::vector<AtomDev> at((size_t)natoms);
  for (int a = 0; a < natoms; a++) {
    AtomDev& t = at[(size_t)a];
    t = AtomDev{};
    for (int d = 0; d < 3; d++) {
      t.X[d] = pos[3 * a + d];
      t.o[d] = (int)std::floor(pos[3 * a + d] / grid->h) - cube / 2 + 1;
    }
    t.sigma = sigma[a];
  }
  char* ws = static_cast<char*>(base);
  // pageable source: the copy is staged before this call returns, so `at` may go out of scope
  if (cudaMemcpyAsync(ws, at.data(), (size_t)natoms * sizeof(AtomDev), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return SHO_ERR_CUDA;
  ProjectLaunch P;
  for (int d = 0; d < 3; d++) P.g.n[d] = grid->n[d];
  P.g.periodic = grid->periodic ? 1 : 0;
  P.g.h = grid->h;
  P.g.cube = cube;
  P.g.nbands = nbands;
  P.psi = psi;
  P.psi_dtype = psi_dtype;
  P.atoms = reinterpret_cast<const AtomDev*>(ws);
  P.natoms = natoms;
  P.numax = numax + 1;
  P.zsplit = choose_zsplit(natoms, nbands, cube, sms);
  P.coeff = ws + atoms_bytes;
  P.coeff_dtype = coeff_dtype;
  P.stream = s;
  if (launch_project(P) != cudaSuccess) return SHO_ERR_CUDA;
  ForcesLaunch F;
  F.natoms = natoms;
  F.numax = numax;
  F.nbands = nbands;
  F.atoms = P.atoms;
  F.cp = ws + atoms_bytes;
  F.dEdc = dEdc;
  F.coeff_dtype = coeff_dtype;
  F.dEdX = dEdX;
  F.stream = s;
  if (launch_forces_contract(F) != cudaSuccess) return SHO_ERR_CUDA;
  return SHO_OK;
}
