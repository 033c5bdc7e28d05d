// sho_api.cu -- host side of the C ABI declared in include/sho.h: argument validation, the per-call
// plan (cube origins, per-plane atom lists), workspace management and kernel launches.
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <vector>

#include "sho_internal.h"

struct sho_handle {
  int device = 0;
  int strict = 0;
  int sms = 1;
  void* ws = nullptr;          // device workspace (plan + intermediates), grows on demand
  size_t ws_bytes = 0;
  cudaEvent_t last = nullptr;  // completion of the handle's most recent call
  void* coeff_ws = nullptr;    // coefficient buffers of the non-local action (c and D c)
  size_t coeff_ws_bytes = 0;
  bool has_last = false;
  int device_error = SHO_OK;   // first device-side error since the last sho_sync
  cudaError_t last_cuda = cudaSuccess;  // CUDA error behind the most recent SHO_ERR_CUDA of this handle
  const char* last_where = "";          // and the step that raised it
  int* dstatus = nullptr;      // device status word (kStatusTimeout | kStatusRange bits) set by kernels
  long long wait_cycles = sho::kDefaultWaitCycles;  // fault injection: limit of the bounded device waits
  int stop_rows = 0x7fffffff;                       // fault injection: rows a plane-sweep producer issues
  double rprj = 0.0;                                // spherical support radius (0: the whole cube)
  int expand_kernel = SHO_KERNEL_AUTO;              // x-pass engine of the FP32-class / FF64 expansion
  int project_kernel = SHO_KERNEL_AUTO;             // x-pass engine of the FF64 projection
  bool dev_checks = false;                          // device checks of the FP64 / FF64 kernels' indices
  long long check_psi_cap = -1;                     // fault injection: psi extent the checks assume (-1: real)
  // device CSR of the radial transform per (numax, direction): rowp | col | val F64 | val F32
  struct RadialDev {
    void* mem = nullptr;
    int nnz = 0;
  } radial[SHO_MAX_NUMAX + 1][2];
  // per-geometry plan arrays of the most recent projection / expansion geometry on the device (atoms,
  // launch order or per-plane lists): repeated calls skip the host planning and the uploads, whose
  // pageable copies would stall the host until the stream drained
  struct GeoCache {
    uint64_t key = 0;
    void* mem = nullptr;
    size_t cap = 0;
    size_t off[4] = {0, 0, 0, 0};
    int extra = 0;
  } geo[2];
  // plane-sweep plan of the most recent geometry (atoms, items, slot lists, segments) on the device:
  // repeated projections with the same atoms skip the host planning and the uploads
  uint64_t plane_key = 0;
  void* plane_mem = nullptr;
  size_t plane_cap = 0;
  int plane_nitems = 0;
  size_t plane_off[4] = {0, 0, 0, 0};
};

namespace sho {
namespace {

// Makes the handle's device current for the duration of a call and restores the caller's device.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Bump allocator over the workspace; every region starts on a 256-byte boundary.
struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  }
};

int check_common(const sho_grid* grid, int nbands, int natoms, const double* pos, const double* sigma, int numax,
                 int cube, int max_numax) {
  if (!grid) return SHO_ERR_ARG;
  if (nbands < 0 || natoms < 0) return SHO_ERR_ARG;
  for (int d = 0; d < 3; d++)
    if (grid->n[d] <= 0) return SHO_ERR_ARG;
  if (!(grid->h > 0.0) || !std::isfinite(grid->h)) return SHO_ERR_ARG;
  if (grid->n[0] > 768) return SHO_ERR_ARG;  // one grid row of 32 bands must fit in shared memory
  if (natoms > 0 && (!pos || !sigma)) return SHO_ERR_ARG;
  if (numax < 0 || numax > max_numax) return SHO_ERR_NUMAX;
  if (cube < 8 || cube > kMaxCube || (cube % 8) != 0) return SHO_ERR_CUBE;
  if (grid->periodic)
    for (int d = 0; d < 3; d++)
      if (cube > grid->n[d]) return SHO_ERR_CUBE;
  for (int a = 0; a < natoms; a++) {
    if (!(sigma[a] > 0.0) || !std::isfinite(sigma[a])) return SHO_ERR_ARG;
    for (int d = 0; d < 3; d++)
      if (!std::isfinite(pos[3 * a + d])) return SHO_ERR_ARG;
  }
  return SHO_OK;
}

int check_spacing(const sho_handle* h, const sho_grid* grid, int natoms, const double* sigma, int numax) {
  if (!h->strict) return SHO_OK;
  for (int a = 0; a < natoms; a++)
    if (grid->h > sho_max_spacing(sigma[a], numax)) return SHO_ERR_SPACING;
  return SHO_OK;
}

int check_dtypes(sho_prec prec, sho_dtype psi_dt, sho_dtype coeff_dt) {
  switch (prec) {
    case SHO_P_FP64:
    case SHO_P_FF64:
      return (psi_dt == SHO_F64 && coeff_dt == SHO_F64) ? SHO_OK : SHO_ERR_DTYPE;
    case SHO_P_FP32:
      return ((psi_dt == SHO_F32 || psi_dt == SHO_BF16) && coeff_dt == SHO_F32) ? SHO_OK : SHO_ERR_DTYPE;
    case SHO_P_TF32:
    case SHO_P_3XTF32:
    case SHO_P_BF16:
    case SHO_P_SPLIT_FP16:
      return ((psi_dt == SHO_F32 || psi_dt == SHO_BF16) && coeff_dt == SHO_F32) ? SHO_OK : SHO_ERR_DTYPE;
    default:
      return SHO_ERR_ARG;
  }
}

std::vector<AtomDev> make_atoms(const sho_grid* grid, int natoms, const double* pos, const double* sigma, int cube) {
  std::vector<AtomDev> at((size_t)natoms);
  for (int a = 0; a < natoms; a++) {
    AtomDev& t = at[(size_t)a];
    std::memset(&t, 0, sizeof(t));
    for (int d = 0; d < 3; d++) {
      t.X[d] = pos[3 * a + d];
      t.o[d] = (int)std::floor(pos[3 * a + d] / grid->h) - cube / 2 + 1;
    }
    t.sigma = sigma[a];
  }
  return at;
}

int grid_index(int o, int i, int n, int periodic) {
  int j = o + i;
  if (periodic) {
    j %= n;
    if (j < 0) j += n;
    return j;
  }
  return (j >= 0 && j < n) ? j : -1;
}

// Per-plane atom lists (CSR): atom a is listed under plane jz for every cube plane it covers,
// atoms in ascending order within a plane.
void plane_lists(const sho_grid* grid, const std::vector<AtomDev>& at, int cube, std::vector<int>& ptr,
                 std::vector<int>& list) {
  const int nz = grid->n[2];
  ptr.assign((size_t)nz + 1, 0);
  for (size_t a = 0; a < at.size(); a++)
    for (int i = 0; i < cube; i++) {
      int j = grid_index(at[a].o[2], i, nz, grid->periodic);
      if (j >= 0) ptr[(size_t)j + 1]++;
    }
  for (int z = 0; z < nz; z++) ptr[(size_t)z + 1] += ptr[(size_t)z];
  list.assign((size_t)ptr[(size_t)nz], 0);
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  for (size_t a = 0; a < at.size(); a++)
    for (int i = 0; i < cube; i++) {
      int j = grid_index(at[a].o[2], i, nz, grid->periodic);
      if (j >= 0) list[(size_t)fill[(size_t)j]++] = (int)a;
    }
}

// Atoms sorted by the Morton code of their cube origins (wrapped into the grid): CTAs launched
// together then work on nearby cubes and share psi rows through L2.  Only the launch order changes;
// every atom's coefficients are computed the same way.
std::vector<int> spatial_order(const sho_grid* grid, const std::vector<AtomDev>& at) {
  auto spread = [](uint32_t v) {
    uint64_t x = v & 0x1fffff;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
  };
  std::vector<std::pair<uint64_t, int>> key(at.size());
  for (size_t a = 0; a < at.size(); a++) {
    uint32_t c[3];
    for (int d = 0; d < 3; d++) {
      int o = at[a].o[d] % grid->n[d];
      if (o < 0) o += grid->n[d];
      c[d] = (uint32_t)o;
    }
    key[a] = {spread(c[0]) | spread(c[1]) << 1 | spread(c[2]) << 2, (int)a};
  }
  std::stable_sort(key.begin(), key.end());
  std::vector<int> order(at.size());
  for (size_t i = 0; i < at.size(); i++) order[i] = key[i].second;
  return order;
}

// Number of cube z-slabs per (atom, band tile) so that the CTAs spread evenly over the SMs.
int zsplit_balanced(int natoms, int nbands, int cube, int sms) {
  const int nbt = (nbands + kWarp - 1) / kWarp;
  int best = 1;
  double best_score = -1.0;
  for (int zs = 1; zs <= 8; zs *= 2) {
    if (zs > 1 && cube / zs < 4) break;
    const double ctas = (double)natoms * nbt * zs;
    const double per_sm = std::ceil(ctas / sms);
    const double eff = ctas / (per_sm * sms);
    const double fill = std::min(1.0, ctas / (4.0 * sms));
    const double score = eff * fill;
    if (score > best_score + 1e-9) {
      best_score = score;
      best = zs;
    }
  }
  return best;
}

int ensure_workspace(sho_handle* h, size_t bytes) {
  if (bytes <= h->ws_bytes) return SHO_OK;
  if (h->has_last && cudaEventSynchronize(h->last) != cudaSuccess) return SHO_ERR_CUDA;
  if (h->ws) cudaFree(h->ws);
  h->ws = nullptr;
  h->ws_bytes = 0;
  size_t want = bytes + bytes / 4 + (1 << 20);
  if (cudaMalloc(&h->ws, want) != cudaSuccess) {
    cudaGetLastError();
    return SHO_ERR_OOM;
  }
  h->ws_bytes = want;
  return SHO_OK;
}

int begin_call(sho_handle* h, cudaStream_t s) {
  // a launch-time error left by unrelated work of the process must not be taken for ours (the launchers
  // check cudaGetLastError after their own launches)
  (void)cudaGetLastError();
  if (h->has_last) {
    const cudaError_t e = cudaStreamWaitEvent(s, h->last, 0);
    if (e != cudaSuccess) {
      h->last_cuda = e;
      h->last_where = "stream wait";
      return SHO_ERR_CUDA;
    }
  }
  return SHO_OK;
}

int end_call(sho_handle* h, cudaStream_t s) {
  if (cudaEventRecord(h->last, s) != cudaSuccess) return SHO_ERR_CUDA;
  h->has_last = true;
  return SHO_OK;
}

int upload(sho_handle* h, size_t off, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return SHO_OK;
  if (cudaMemcpyAsync(static_cast<char*>(h->ws) + off, src, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return SHO_ERR_CUDA;
  return SHO_OK;
}

// Extra limits of the tensor-core forms: numax (of the projection actually run) <= 7 and a cube of
// whole 16-point MMA steps.
int check_tc(sho_prec prec, int numax_run, int cube) {
  if (!is_tc(prec)) return SHO_OK;
  if (numax_run > kTcMaxNumax) return SHO_ERR_NUMAX;
  if (cube % 16) return SHO_ERR_CUBE;
  return SHO_OK;
}

GridDev make_grid(const sho_grid* grid, int cube, int nbands, double rprj = 0.0) {
  GridDev g;
  for (int d = 0; d < 3; d++) g.n[d] = grid->n[d];
  g.periodic = grid->periodic ? 1 : 0;
  g.h = grid->h;
  g.cube = cube;
  g.nbands = nbands;
  g.r2max = rprj > 0.0 ? rprj * rprj : 0.0;
  return g;
}

// Spherical support is implemented by the FP64 and FP64-accurate kernels (and the stored-projector build).
int check_support(const sho_handle* h, sho_prec prec) {
  return (h->rprj > 0.0 && !is_f64_form(prec)) ? SHO_ERR_DTYPE : SHO_OK;
}

#define SHO_TRY(x)                \
  do {                            \
    int _st = (x);                \
    if (_st != SHO_OK) return _st; \
  } while (0)

// Plane-sweep projection (FP32 psi, FP32 coefficients): plan the row segments on the host, upload
// the plan and run tables -> plane sweep -> z-pass (sho_plane.cu).
// FNV-1a over the geometry a plane plan depends on (grid, cube, the atoms with their origins).
uint64_t geometry_key(const sho_grid* grid, const std::vector<AtomDev>& at, int cube) {
  uint64_t k = 1469598103934665603ull;
  auto mix = [&k](const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; i++) {
      k ^= c[i];
      k *= 1099511628211ull;
    }
  };
  mix(grid->n, sizeof(grid->n));
  mix(&grid->h, sizeof(grid->h));
  mix(&grid->periodic, sizeof(grid->periodic));
  mix(&cube, sizeof(cube));
  const size_t A = at.size();
  mix(&A, sizeof(A));
  if (A) mix(at.data(), A * sizeof(AtomDev));
  return k | 1ull;  // never 0 (0 marks "no plan")
}

// Make the handle's cache slot hold `parts` for geometry `key` (uploaded, stream-ordered on s, only when
// the key changed).  Call after begin_call.
int geo_cache(sho_handle* h, int slot, uint64_t key, const std::vector<std::pair<const void*, size_t>>& parts,
              cudaStream_t s) {
  auto& gc = h->geo[slot];
  if (gc.key == key && gc.mem) return SHO_OK;
  Carve cv;
  size_t off[4] = {0, 0, 0, 0};
  for (size_t i = 0; i < parts.size() && i < 4; i++) off[i] = cv.take(std::max<size_t>(1, parts[i].second));
  if (cv.off > gc.cap) {
    if (h->has_last) {
      const cudaError_t e = cudaEventSynchronize(h->last);
      if (e != cudaSuccess) {
        h->last_cuda = e;
        h->last_where = "plan cache: wait";
        return SHO_ERR_CUDA;
      }
    }
    if (gc.mem) {
      const cudaError_t e = cudaFree(gc.mem);
      if (e != cudaSuccess) {
        h->last_cuda = e;
        h->last_where = "plan cache: free";
        gc.mem = nullptr;
        gc.cap = 0;
        gc.key = 0;
        (void)cudaGetLastError();
        return SHO_ERR_CUDA;
      }
    }
    gc.mem = nullptr;
    gc.cap = 0;
    gc.key = 0;
    if (cudaMalloc(&gc.mem, cv.off) != cudaSuccess) {
      cudaGetLastError();
      gc.mem = nullptr;
      return SHO_ERR_OOM;
    }
    gc.cap = cv.off;
  }
  for (size_t i = 0; i < parts.size() && i < 4; i++) {
    if (parts[i].second == 0) continue;
    const cudaError_t e = cudaMemcpyAsync(static_cast<char*>(gc.mem) + off[i], parts[i].first, parts[i].second,
                                          cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      h->last_cuda = e;
      h->last_where = "plan cache: upload";
      gc.key = 0;
      return SHO_ERR_CUDA;
    }
  }
  for (int i = 0; i < 4; i++) gc.off[i] = off[i];
  gc.key = key;
  return SHO_OK;
}

// t2_out != nullptr: stop after the per-plane sums and leave them in t2_out ([A][cube][P][B] FP32, owned by
// the caller) for a fused z-pass; coeff is then not written.
int project_planes(sho_handle* h, const sho_grid* grid, const std::vector<AtomDev>& at, const void* psi,
                   sho_dtype psi_dtype, int nbands, int numax, int cube, sho_prec prec, float* coeff, cudaStream_t s,
                   float* t2_out = nullptr) {
  const size_t A = at.size();
  const uint64_t key = geometry_key(grid, at, cube);
  SHO_TRY(begin_call(h, s));
  if (h->plane_key != key) {
    PlanePlan plan;
    plan_planes(grid, at, cube, plan);
    Carve pc;
    const size_t o_atoms = pc.take(A * sizeof(AtomDev));
    const size_t o_items = pc.take(std::max<size_t>(1, plan.items.size()) * sizeof(int4));
    const size_t o_ptr = pc.take(plan.slot_ptr.size() * sizeof(int));
    const size_t o_segs = pc.take(std::max<size_t>(1, plan.segs.size()) * sizeof(PlaneSeg));
    if (pc.off > h->plane_cap) {
      if (h->has_last && cudaEventSynchronize(h->last) != cudaSuccess) return SHO_ERR_CUDA;
      if (h->plane_mem) cudaFree(h->plane_mem);
      h->plane_mem = nullptr;
      h->plane_cap = 0;
      h->plane_key = 0;
      if (cudaMalloc(&h->plane_mem, pc.off) != cudaSuccess) {
        cudaGetLastError();
        h->plane_mem = nullptr;
        return SHO_ERR_OOM;
      }
      h->plane_cap = pc.off;
    }
    char* pm = static_cast<char*>(h->plane_mem);
    // stream-ordered after the handle's earlier work (begin_call), which may still read the old plan
    auto up = [&](size_t off, const void* src, size_t bytes) {
      return bytes == 0 || cudaMemcpyAsync(pm + off, src, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess;
    };
    if (!up(o_atoms, at.data(), A * sizeof(AtomDev)) || !up(o_items, plan.items.data(), plan.items.size() * sizeof(int4)) ||
        !up(o_ptr, plan.slot_ptr.data(), plan.slot_ptr.size() * sizeof(int)) ||
        !up(o_segs, plan.segs.data(), plan.segs.size() * sizeof(PlaneSeg))) {
      h->plane_key = 0;
      return SHO_ERR_CUDA;
    }
    // pageable sources: the copies have been staged before cudaMemcpyAsync returns, so the vectors
    // may go out of scope here
    h->plane_key = key;
    h->plane_nitems = (int)plan.items.size();
    h->plane_off[0] = o_atoms;
    h->plane_off[1] = o_items;
    h->plane_off[2] = o_ptr;
    h->plane_off[3] = o_segs;
  }
  Carve cv;
  const size_t o_xt = cv.take(A * cube * 8 * sizeof(float));
  const size_t o_yt = cv.take(A * cube * 8 * sizeof(float));
  const size_t o_bf = cv.take(A * kPlaneBfragBytesPerAtom);
  const size_t o_t2 = t2_out ? 0 : cv.take(A * cube * (size_t)npairs(numax) * nbands * sizeof(float));
  SHO_TRY(ensure_workspace(h, cv.off));
  char* ws = static_cast<char*>(h->ws);
  const char* pm = static_cast<const char*>(h->plane_mem);
  PlaneLaunch L;
  L.g = make_grid(grid, cube, nbands);
  L.psi = psi;
  L.psi_dtype = psi_dtype;
  L.atoms = reinterpret_cast<const AtomDev*>(pm + h->plane_off[0]);
  L.natoms = (int)A;
  L.numax = numax;
  L.items = reinterpret_cast<const int4*>(pm + h->plane_off[1]);
  L.nitems = h->plane_nitems;
  L.slot_ptr = reinterpret_cast<const int*>(pm + h->plane_off[2]);
  L.segs = reinterpret_cast<const PlaneSeg*>(pm + h->plane_off[3]);
  L.xtab = reinterpret_cast<float*>(ws + o_xt);
  L.ytab = reinterpret_cast<float*>(ws + o_yt);
  L.bfrag = reinterpret_cast<uint32_t*>(ws + o_bf);
  L.t2p = t2_out ? t2_out : reinterpret_cast<float*>(ws + o_t2);
  L.t2_only = t2_out != nullptr;
  L.coeff = coeff;
  L.status = h->dstatus;
  L.wait_cycles = h->wait_cycles;
  L.stop_rows = h->stop_rows;
  L.stream = s;
  if (launch_project_plane(L, prec) != cudaSuccess) return SHO_ERR_CUDA;
  return end_call(h, s);
}

}  // namespace

// Workspace a call needs (an upper bound: the per-plane lists are counted as natoms * cube entries).
size_t workspace_bytes(sho_op op, const sho_grid* grid, int natoms, int numax, int cube, int nbands,
                       sho_dtype coeff_dtype) {
  const size_t tc = compute_size(coeff_dtype);
  Carve cv;
  cv.take((size_t)natoms * sizeof(AtomDev));
  if (op == SHO_OP_PROJECT) {
    cv.take((size_t)natoms * sizeof(int));
    if (coeff_dtype == SHO_F64) {  // FP64-accurate form: per-plane sums, tensor-core tables
      cv.take(ff_t2_bytes(natoms, cube, numax, nbands));
      cv.take(op_layout(natoms, cube, numax).total);
    }
    if (coeff_dtype == SHO_F32 && numax <= kTcMaxNumax) {
      // plane-sweep path (an upper bound: every (atom, plane) split into two row segments)
      const size_t segs = 2 * (size_t)natoms * cube + 1;
      cv.take((segs + grid->n[2]) * sizeof(int4));
      cv.take(((segs + grid->n[2]) * 36 + 1) * sizeof(int));
      cv.take(segs * sizeof(PlaneSeg));
      cv.take(2 * (size_t)natoms * cube * 8 * sizeof(float));
      cv.take((size_t)natoms * kPlaneBfragBytesPerAtom);
      cv.take((size_t)natoms * cube * npairs(numax) * (size_t)nbands * sizeof(float));
    }
  }
  if (op == SHO_OP_EXPAND) {
    cv.take(((size_t)grid->n[2] + 1) * sizeof(int));
    cv.take(std::max<size_t>(1, (size_t)natoms * cube) * sizeof(int));
    cv.take((size_t)natoms * 2 * (numax + 1) * cube * tc);
    cv.take(t2_bytes(natoms, cube, numax, nbands, tc));
    cv.take((size_t)natoms * cube * txm_bytes_per_point(numax));
    if (coeff_dtype == SHO_F64) cv.take(oz_layout(natoms, cube, nbands).total);  // FP64-accurate form
  }
  return cv.off;
}

// Grow the handle's workspace to exactly `bytes` (no growth margin) when it is smaller.
int handle_reserve(sho_handle* h, size_t bytes) {
  if (bytes <= h->ws_bytes) return SHO_OK;
  DeviceGuard guard(h->device);
  if (h->has_last && cudaEventSynchronize(h->last) != cudaSuccess) return SHO_ERR_CUDA;
  if (h->ws) cudaFree(h->ws);
  h->ws = nullptr;
  h->ws_bytes = 0;
  if (cudaMalloc(&h->ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    return SHO_ERR_OOM;
  }
  h->ws_bytes = bytes;
  return SHO_OK;
}

size_t handle_workspace(const sho_handle* h) { return h->ws_bytes; }

int choose_zsplit(int natoms, int nbands, int cube, int sms) { return zsplit_balanced(natoms, nbands, cube, sms); }

// Extents for the device checks of a call (sho_set_device_checks); checks off: flag null.
DevCheck make_check(const sho_handle* h, const sho_grid* grid, int nbands, int natoms, int numax, int cube) {
  DevCheck d;
  if (!h->dev_checks) return d;
  d.psi_n = (long long)grid->n[0] * grid->n[1] * grid->n[2] * nbands;
  if (h->check_psi_cap >= 0 && h->check_psi_cap < d.psi_n) d.psi_n = h->check_psi_cap;
  d.coeff_n = (long long)natoms * nstates(numax) * nbands;
  d.t2_n = (long long)natoms * cube * npairs(numax) * nbands;
  d.flag = h->dstatus;
  return d;
}

int handle_take_status(sho_handle* h) {
  DeviceGuard guard(h->device);
  int flag = 0;
  if (cudaMemcpy(&flag, h->dstatus, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SHO_ERR_CUDA;
  if (flag == 0) return SHO_OK;
  if (cudaMemset(h->dstatus, 0, sizeof(int)) != cudaSuccess) return SHO_ERR_CUDA;
  return (flag & kStatusTimeout) ? SHO_ERR_TIMEOUT : SHO_ERR_DEVICE;
}

}  // namespace sho

using namespace sho;

extern "C" {

int sho_version(void) { return SHO_VERSION; }

int sho_nstates(int numax) { return sho::nstates(numax); }

double sho_max_spacing(double sigma, int numax) {
  if (numax < 0) return 0.0;
  return 3.14159265358979323846 * sigma / std::sqrt(2.0 * numax + 1.0);
}

const char* sho_strerror(int status) {
  switch (status) {
    case SHO_OK: return "success";
    case SHO_ERR_ARG: return "invalid argument";
    case SHO_ERR_NUMAX: return "numax out of range";
    case SHO_ERR_CUBE: return "unsupported cube size";
    case SHO_ERR_SPACING: return "grid spacing above the sampling limit h_max";
    case SHO_ERR_DTYPE: return "unsupported dtype / precision combination";
    case SHO_ERR_OOM: return "out of memory";
    case SHO_ERR_CUDA: return "CUDA error";
    case SHO_ERR_TIMEOUT: return "timed out";
    case SHO_ERR_DEVICE: return "device-side check failed";
    case SHO_ERR_CAPACITY: return "request exceeds the memory budget";
    case SHO_ERR_STATE: return "invalid state";
    case SHO_ERR_CANCELLED: return "request cancelled";
    default: return "unknown status";
  }
}

int sho_create(sho_handle** out, int device) {
  if (!out) return SHO_ERR_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess) {
    cudaGetLastError();
    return SHO_ERR_CUDA;
  }
  if (device < 0 || device >= count) return SHO_ERR_ARG;
  DeviceGuard guard(device);
  if (!guard.ok) return SHO_ERR_CUDA;
  sho_handle* h = new sho_handle();
  h->device = device;
  if (cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) h->sms = 1;
  if (cudaEventCreateWithFlags(&h->last, cudaEventDisableTiming) != cudaSuccess) {
    delete h;
    return SHO_ERR_CUDA;
  }
  if (cudaMalloc(&h->dstatus, sizeof(int)) != cudaSuccess || cudaMemset(h->dstatus, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    if (h->dstatus) cudaFree(h->dstatus);
    cudaEventDestroy(h->last);
    delete h;
    return SHO_ERR_OOM;
  }
  *out = h;
  return SHO_OK;
}

int sho_destroy(sho_handle* h) {
  if (!h) return SHO_ERR_ARG;
  int st = SHO_OK;
  {
    DeviceGuard guard(h->device);
    if (h->has_last && cudaEventSynchronize(h->last) != cudaSuccess) st = SHO_ERR_CUDA;
    if (h->ws) cudaFree(h->ws);
    if (h->coeff_ws) cudaFree(h->coeff_ws);
    if (h->dstatus) cudaFree(h->dstatus);
    if (h->plane_mem) cudaFree(h->plane_mem);
    for (auto& gc : h->geo)
      if (gc.mem) cudaFree(gc.mem);
    for (auto& row : h->radial)
      for (auto& r : row)
        if (r.mem) cudaFree(r.mem);
    if (h->last) cudaEventDestroy(h->last);
  }
  delete h;
  return st;
}

const char* sho_last_cuda_error(const sho_handle* h) {
  if (!h) return "no handle";
  static thread_local char buf[256];
  std::snprintf(buf, sizeof(buf), "%s%s%s", cudaGetErrorString(h->last_cuda), h->last_where[0] ? " at " : "",
                h->last_where);
  return buf;
}

int sho_set_strict(sho_handle* h, int strict) {
  if (!h) return SHO_ERR_ARG;
  h->strict = strict ? 1 : 0;
  return SHO_OK;
}

int sho_sync(sho_handle* h) {
  if (!h) return SHO_ERR_ARG;
  DeviceGuard guard(h->device);
  if (h->has_last && cudaEventSynchronize(h->last) != cudaSuccess) return SHO_ERR_CUDA;
  const int dst = handle_take_status(h);
  if (dst != SHO_OK && h->device_error == SHO_OK) h->device_error = dst;
  int e = h->device_error;
  h->device_error = SHO_OK;
  return e;
}

int sho_radial_labels(int numax, int* nr, int* ell, int* m) {
  if (numax < 0 || numax > SHO_MAX_NUMAX) return SHO_ERR_NUMAX;
  if (!nr || !ell || !m) return SHO_ERR_ARG;
  radial_labels(numax, nr, ell, m);
  return SHO_OK;
}

int sho_radial_matrix(int numax, double* U) {
  if (numax < 0 || numax > SHO_MAX_NUMAX) return SHO_ERR_NUMAX;
  if (!U) return SHO_ERR_ARG;
  const size_t N = (size_t)nstates(numax);
  std::memcpy(U, radial_matrix(numax), N * N * sizeof(double));
  return SHO_OK;
}

int sho_radial_transform(sho_handle* h, int natoms, int numax, int nbands, const void* in, void* out, sho_dtype dtype,
                         int direction, void* stream) {
  if (!h) return SHO_ERR_ARG;
  if (numax < 0 || numax > SHO_MAX_NUMAX) return SHO_ERR_NUMAX;
  if (natoms < 0 || nbands < 0 || (direction != 0 && direction != 1)) return SHO_ERR_ARG;
  if (dtype != SHO_F64 && dtype != SHO_F32) return SHO_ERR_DTYPE;
  if (natoms == 0 || nbands == 0) return SHO_OK;
  if (!in || !out || in == out) return SHO_ERR_ARG;
  DeviceGuard guard(h->device);
  if (!guard.ok) return SHO_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int N = nstates(numax);
  auto& rd = h->radial[numax][direction];
  if (!rd.mem) {
    std::vector<int> rowp, col;
    std::vector<double> val;
    radial_csr(numax, direction, rowp, col, val);
    std::vector<float> valf(val.begin(), val.end());
    const size_t nnz = col.size();
    const size_t bytes = (rowp.size() + nnz) * sizeof(int) + nnz * (sizeof(double) + sizeof(float)) + 64;
    std::vector<char> blob(bytes, 0);
    size_t off = 0;
    std::memcpy(blob.data() + off, rowp.data(), rowp.size() * sizeof(int));
    off += rowp.size() * sizeof(int);
    std::memcpy(blob.data() + off, col.data(), nnz * sizeof(int));
    off = (off + nnz * sizeof(int) + 7) & ~(size_t)7;
    std::memcpy(blob.data() + off, val.data(), nnz * sizeof(double));
    off += nnz * sizeof(double);
    std::memcpy(blob.data() + off, valf.data(), nnz * sizeof(float));
    if (h->has_last && cudaEventSynchronize(h->last) != cudaSuccess) return SHO_ERR_CUDA;
    if (cudaMalloc(&rd.mem, bytes) != cudaSuccess) {
      cudaGetLastError();
      rd.mem = nullptr;
      return SHO_ERR_OOM;
    }
    if (cudaMemcpy(rd.mem, blob.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) return SHO_ERR_CUDA;
    rd.nnz = (int)nnz;
  }
  const char* base = static_cast<const char*>(rd.mem);
  const int* rowp = reinterpret_cast<const int*>(base);
  const int* col = rowp + N + 1;
  const size_t off_val = (((size_t)(N + 1) + rd.nnz) * sizeof(int) + 7) & ~(size_t)7;
  const void* val = dtype == SHO_F64 ? (const void*)(base + off_val)
                                     : (const void*)(base + off_val + (size_t)rd.nnz * sizeof(double));
  SHO_TRY(begin_call(h, s));
  if (launch_radial(natoms, N, nbands, dtype, rowp, col, val, in, out, s) != cudaSuccess) return SHO_ERR_CUDA;
  return end_call(h, s);
}

static int project_impl(sho_handle* h, const sho_grid* grid, const void* psi, sho_dtype psi_dtype, int nbands,
                        int natoms, const double* pos, const double* sigma, int numax, int cube, sho_prec prec,
                        void* coeff, sho_dtype coeff_dtype, void* stream, void* t2_out, bool* at_t2,
                        const BlochArg* bloch = nullptr);
static int add_impl(sho_handle* h, const sho_grid* grid, double alpha, int overwrite, const void* coeff,
                    sho_dtype coeff_dtype, int nbands, int natoms, const double* pos, const double* sigma, int numax,
                    int cube, sho_prec prec, void* psi, sho_dtype psi_dtype, void* stream,
                    const NonlocalIn* nl = nullptr, const BlochArg* bloch = nullptr);

static int bloch_call(sho_handle* h, const sho_grid* grid, const double* kvec, int op, const void* src, void* dst,
                      int nbands, int natoms, const double* pos, const double* sigma, int numax, int cube,
                      sho_prec prec, void* stream) {
  if (!h) return SHO_ERR_ARG;
  SHO_TRY(check_common(grid, nbands, natoms, pos, sigma, numax, cube, kTcMaxNumax));
  if (!grid->periodic || !kvec) return SHO_ERR_ARG;
  if (prec != SHO_P_FP64 && prec != SHO_P_FF64 && prec != SHO_P_FP32) return SHO_ERR_DTYPE;
  if (h->rprj > 0.0) return SHO_ERR_DTYPE;  // spherical support: the real forms only
  for (int d = 0; d < 3; d++)
    if (!std::isfinite(kvec[d])) return SHO_ERR_ARG;
  if (op == 1 && prec == SHO_P_FP64 && grid->n[0] > kBlochMaxNx) return SHO_ERR_ARG;
  if (nbands > INT_MAX / 2) return SHO_ERR_ARG;
  SHO_TRY(check_spacing(h, grid, natoms, sigma, numax));
  if (natoms == 0 || nbands == 0) return SHO_OK;
  if (!src || !dst) return SHO_ERR_ARG;
  // FP32: the streaming CUDA-core kernels, which want 16-byte aligned psi rows
  if (prec == SHO_P_FP32 && !fp32_stream_ok(op == 0 ? src : dst, SHO_F32, 2 * nbands)) return SHO_ERR_ARG;
  if (prec != SHO_P_FP64) {
    // the real FP64-accurate or FP32 kernels over the (re, im) pairs as 2 nbands real bands, with the phases
    const BlochArg bl{{kvec[0], kvec[1], kvec[2]}, op == 0 ? 1.0 : -1.0};
    const sho_dtype dt = prec == SHO_P_FF64 ? SHO_F64 : SHO_F32;
    if (op == 0)
      return project_impl(h, grid, src, dt, 2 * nbands, natoms, pos, sigma, numax, cube, prec, dst, dt, stream,
                          nullptr, nullptr, &bl);
    return add_impl(h, grid, 1.0, 0, src, dt, 2 * nbands, natoms, pos, sigma, numax, cube, prec, dst, dt, stream,
                    nullptr, &bl);
  }
  DeviceGuard guard(h->device);
  if (!guard.ok) return SHO_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<AtomDev> at = make_atoms(grid, natoms, pos, sigma, cube);
  const int N = nstates(numax), NP = numax + 1;
  const int zsplit = op == 0 ? zsplit_balanced(natoms, nbands, cube, h->sms) : 1;
  std::vector<int> ptr, list;
  if (op == 1) plane_lists(grid, at, cube, ptr, list);
  Carve cv;
  const size_t o_atoms = cv.take(at.size() * sizeof(AtomDev));
  const size_t o_ptr = cv.take(std::max<size_t>(1, ptr.size()) * sizeof(int));
  const size_t o_list = cv.take(std::max<size_t>(1, list.size()) * sizeof(int));
  const size_t o_tab = cv.take((size_t)natoms * 3 * NP * cube * 2 * sizeof(double));
  const size_t work = op == 0 ? (size_t)zsplit * natoms * N * nbands : (size_t)natoms * cube * npairs(numax) * nbands;
  const size_t o_work = cv.take(work * 2 * sizeof(double));
  SHO_TRY(begin_call(h, s));
  SHO_TRY(ensure_workspace(h, cv.off));
  SHO_TRY(upload(h, o_atoms, at.data(), at.size() * sizeof(AtomDev), s));
  if (op == 1) {
    SHO_TRY(upload(h, o_ptr, ptr.data(), ptr.size() * sizeof(int), s));
    SHO_TRY(upload(h, o_list, list.data(), list.size() * sizeof(int), s));
  }
  char* ws = static_cast<char*>(h->ws);
  BlochLaunch L = {};
  L.g = make_grid(grid, cube, nbands);
  L.atoms = reinterpret_cast<const AtomDev*>(ws + o_atoms);
  L.natoms = natoms;
  L.numax = numax;
  for (int d = 0; d < 3; d++) L.k[d] = kvec[d];
  L.op = op;
  L.zsplit = zsplit;
  L.psi_in = op == 0 ? static_cast<const double*>(src) : nullptr;
  L.coeff_out = op == 0 ? static_cast<double*>(dst) : nullptr;
  L.coeff_in = op == 1 ? static_cast<const double*>(src) : nullptr;
  L.psi_out = op == 1 ? static_cast<double*>(dst) : nullptr;
  L.plane_ptr = reinterpret_cast<const int*>(ws + o_ptr);
  L.plane_atoms = reinterpret_cast<const int*>(ws + o_list);
  L.tab = reinterpret_cast<double*>(ws + o_tab);
  L.work = reinterpret_cast<double*>(ws + o_work);
  L.stream = s;
  if (launch_bloch(L) != cudaSuccess) return SHO_ERR_CUDA;
  return end_call(h, s);
}

int sho_project_bloch(sho_handle* h, const sho_grid* grid, const double* kvec, const void* psi, int nbands,
                      int natoms, const double* pos, const double* sigma, int numax, int cube, sho_prec prec,
                      void* coeff, void* stream) {
  return bloch_call(h, grid, kvec, 0, psi, coeff, nbands, natoms, pos, sigma, numax, cube, prec, stream);
}

int sho_add_bloch(sho_handle* h, const sho_grid* grid, const double* kvec, const void* coeff, int nbands, int natoms,
                  const double* pos, const double* sigma, int numax, int cube, sho_prec prec, void* psi,
                  void* stream) {
  return bloch_call(h, grid, kvec, 1, coeff, psi, nbands, natoms, pos, sigma, numax, cube, prec, stream);
}

int sho_plane_plan_check(const sho_grid* grid, int natoms, const double* pos, const double* sigma, int cube,
                         int* nitems, int* nsegs) {
  SHO_TRY(check_common(grid, 0, natoms, pos, sigma, 0, cube, SHO_MAX_NUMAX));
  std::vector<AtomDev> at = make_atoms(grid, natoms, pos, sigma, cube);
  PlanePlan plan;
  plan_planes(grid, at, cube, plan);
  if (nitems) *nitems = (int)plan.items.size();
  if (nsegs) *nsegs = (int)plan.segs.size();
  const int r = plane_plan_check(grid, at, cube, plan);
  return r == 0 ? SHO_OK : SHO_ERR_STATE;
}

int sho_project_path(const sho_grid* grid, const void* psi, sho_dtype psi_dtype, int nbands, int numax, int cube,
                     sho_prec prec, sho_dtype coeff_dtype) {
  if (!grid) return SHO_ERR_ARG;
  return (coeff_dtype == SHO_F32 && plane_ok(grid, psi, psi_dtype, nbands, numax, cube, prec)) ? SHO_PATH_PLANE
                                                                                              : SHO_PATH_ATOM;
}

// t2_out != nullptr (fused non-local action): where the path has a separate z-pass (FP64-accurate form,
// plane sweep) stop after the per-plane y-pass sums, leave them in t2_out ([A][cube][P][B], compute type)
// and set *at_t2; other paths write coeff as usual.
// bloch != nullptr: the FP64-accurate or FP32 Bloch projection (complex psi and coeff as 2 real bands per
// band, nbands counting both), its per-atom phases computed into the workspace (behind the per-plane sums
// of the FP64-accurate form).
static int project_impl(sho_handle* h, const sho_grid* grid, const void* psi, sho_dtype psi_dtype, int nbands,
                        int natoms, const double* pos, const double* sigma, int numax, int cube, sho_prec prec,
                        void* coeff, sho_dtype coeff_dtype, void* stream, void* t2_out, bool* at_t2,
                        const BlochArg* bloch) {
  if (at_t2) *at_t2 = false;
  if (!h) return SHO_ERR_ARG;
  SHO_TRY(check_common(grid, nbands, natoms, pos, sigma, numax, cube, SHO_MAX_NUMAX));
  SHO_TRY(check_dtypes(prec, psi_dtype, coeff_dtype));
  SHO_TRY(check_tc(prec, numax, cube));
  SHO_TRY(check_spacing(h, grid, natoms, sigma, numax));
  SHO_TRY(check_support(h, prec));
  if (natoms == 0 || nbands == 0) return SHO_OK;
  if (!psi || !coeff) return SHO_ERR_ARG;
  DeviceGuard guard(h->device);
  if (!guard.ok) return SHO_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<AtomDev> at = make_atoms(grid, natoms, pos, sigma, cube);
  if (!bloch && coeff_dtype == SHO_F32 && plane_ok(grid, psi, psi_dtype, nbands, numax, cube, prec)) {
    if (t2_out && at_t2) *at_t2 = true;
    return project_planes(h, grid, at, psi, psi_dtype, nbands, numax, cube, prec, static_cast<float*>(coeff), s,
                          static_cast<float*>(t2_out));
  }
  SHO_TRY(begin_call(h, s));
  const bool ff_t2 = prec == SHO_P_FF64 && t2_out;
  // FP64-accurate form: per-plane sums (unless the caller provides them), Bloch phases, tensor-core tables
  const bool ff = prec == SHO_P_FF64;
  Carve fcv;
  if (ff && !ff_t2) fcv.take(ff_t2_bytes(natoms, cube, numax, nbands));
  const size_t o_bloch = bloch ? fcv.take((size_t)natoms * sizeof(BlochPh)) : 0;
  const size_t o_op = ff ? fcv.take(op_layout(natoms, cube, numax).total) : 0;
  if (ff || bloch) SHO_TRY(ensure_workspace(h, fcv.off));
  const uint64_t key = geometry_key(grid, at, cube);
  if (h->geo[0].key != key) {
    std::vector<int> order = spatial_order(grid, at);
    SHO_TRY(geo_cache(h, 0, key, {{at.data(), at.size() * sizeof(AtomDev)}, {order.data(), order.size() * sizeof(int)}},
                      s));
  }
  const char* gm = static_cast<const char*>(h->geo[0].mem);
  ProjectLaunch L;
  L.order = reinterpret_cast<const int*>(gm + h->geo[0].off[1]);
  L.g = make_grid(grid, cube, nbands, h->rprj);
  L.psi = psi;
  L.psi_dtype = psi_dtype;
  L.atoms = reinterpret_cast<const AtomDev*>(gm + h->geo[0].off[0]);
  L.natoms = natoms;
  L.numax = numax;
  L.zsplit = prec == SHO_P_FF64 ? ff_zsplit(natoms, nbands, cube, h->sms) : zsplit_balanced(natoms, nbands, cube, h->sms);
  L.coeff = coeff;
  L.coeff_dtype = coeff_dtype;
  L.t2 = ff_t2 ? t2_out : h->ws;
  L.t2_only = ff_t2;
  L.status = h->dstatus;
  if (prec == SHO_P_FF64) L.op = static_cast<char*>(h->ws) + o_op;
  L.kernel = h->project_kernel;
  L.wait_cycles = h->wait_cycles;
  L.chk = make_check(h, grid, nbands, natoms, numax, cube);
  if (bloch) {
    L.chk = DevCheck{};  // the Bloch kernels run unchecked
    BlochPh* ph = reinterpret_cast<BlochPh*>(static_cast<char*>(h->ws) + o_bloch);
    L.bloch = ph;
    const cudaError_t e = launch_bloch_phases(L.g, L.atoms, natoms, *bloch, ph, s);
    if (e != cudaSuccess) {
      h->last_cuda = e;
      h->last_where = "Bloch phases";
      return SHO_ERR_CUDA;
    }
  }
  L.stream = s;
  const cudaError_t e = prec == SHO_P_FP64 ? launch_project(L)
                        : prec == SHO_P_FF64 ? launch_project_ff(L)
                        : fp32_stream_ok(psi, psi_dtype, nbands) ? launch_project_fp32(L, prec)
                        : is_tc(prec) ? launch_project_tc(L, prec)
                        : launch_project(L);
  if (e != cudaSuccess) {
    h->last_cuda = e;
    h->last_where = "projection launch";
    return SHO_ERR_CUDA;
  }
  if (ff_t2 && at_t2) *at_t2 = true;
  return end_call(h, s);
}

int sho_project(sho_handle* h, const sho_grid* grid, const void* psi, sho_dtype psi_dtype, int nbands, int natoms,
                const double* pos, const double* sigma, int numax, int cube, sho_prec prec, void* coeff,
                sho_dtype coeff_dtype, void* stream) {
  return project_impl(h, grid, psi, psi_dtype, nbands, natoms, pos, sigma, numax, cube, prec, coeff, coeff_dtype,
                      stream, nullptr, nullptr);
}

static int add_impl(sho_handle* h, const sho_grid* grid, double alpha, int overwrite, const void* coeff,
                    sho_dtype coeff_dtype, int nbands, int natoms, const double* pos, const double* sigma, int numax,
                    int cube, sho_prec prec, void* psi, sho_dtype psi_dtype, void* stream,
                    const NonlocalIn* nl, const BlochArg* bloch) {
  if (!h) return SHO_ERR_ARG;
  if (!std::isfinite(alpha)) return SHO_ERR_ARG;
  SHO_TRY(check_common(grid, nbands, natoms, pos, sigma, numax, cube, SHO_MAX_NUMAX));
  SHO_TRY(check_dtypes(prec, psi_dtype, coeff_dtype));
  SHO_TRY(check_tc(prec, numax, cube));
  SHO_TRY(check_spacing(h, grid, natoms, sigma, numax));
  SHO_TRY(check_support(h, prec));
  if (nbands == 0) return SHO_OK;
  if (!psi || (natoms > 0 && !coeff)) return SHO_ERR_ARG;
  DeviceGuard guard(h->device);
  if (!guard.ok) return SHO_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (overwrite) {
    // psi = alpha E c: clear the whole grid first (points outside every cube end as zero)
    const size_t es = psi_dtype == SHO_F64 ? 8 : (psi_dtype == SHO_F32 ? 4 : 2);
    const size_t bytes = (size_t)grid->n[0] * grid->n[1] * grid->n[2] * (size_t)nbands * es;
    SHO_TRY(begin_call(h, s));
    const cudaError_t e = cudaMemsetAsync(psi, 0, bytes, s);
    if (e != cudaSuccess) {
      h->last_cuda = e;
      h->last_where = "expansion: clear psi";
      return SHO_ERR_CUDA;
    }
    SHO_TRY(end_call(h, s));
  }
  if (natoms == 0) return SHO_OK;
  std::vector<AtomDev> at = make_atoms(grid, natoms, pos, sigma, cube);
  const size_t tc = compute_size(coeff_dtype);
  Carve cv;
  const size_t o_tab = cv.take((size_t)natoms * 2 * (numax + 1) * cube * tc);
  const size_t o_t2 = cv.take(t2_bytes(natoms, cube, numax, nbands, tc));
  const size_t o_txm = cv.take((size_t)natoms * cube * txm_bytes_per_point(numax));
  const size_t o_oz = prec == SHO_P_FF64 ? cv.take(oz_layout(natoms, cube, nbands).total) : 0;
  const size_t o_bloch = bloch ? cv.take((size_t)natoms * sizeof(BlochPh)) : 0;
  SHO_TRY(begin_call(h, s));
  const uint64_t key = geometry_key(grid, at, cube);
  if (h->geo[1].key != key) {
    std::vector<int> ptr, list;
    plane_lists(grid, at, cube, ptr, list);
    int max_plane = 0;
    for (size_t z = 0; z + 1 < ptr.size(); z++) max_plane = std::max(max_plane, ptr[z + 1] - ptr[z]);
    SHO_TRY(geo_cache(h, 1, key,
                      {{at.data(), at.size() * sizeof(AtomDev)},
                       {ptr.data(), ptr.size() * sizeof(int)},
                       {list.data(), list.size() * sizeof(int)}},
                      s));
    h->geo[1].extra = max_plane;
  }
  SHO_TRY(ensure_workspace(h, cv.off));
  char* ws = static_cast<char*>(h->ws);
  const char* gm = static_cast<const char*>(h->geo[1].mem);
  ExpandLaunch L;
  L.g = make_grid(grid, cube, nbands, h->rprj);
  L.coeff = coeff;
  L.coeff_dtype = coeff_dtype;
  L.psi = psi;
  L.psi_dtype = psi_dtype;
  L.atoms = reinterpret_cast<const AtomDev*>(gm + h->geo[1].off[0]);
  L.natoms = natoms;
  L.numax = numax;
  L.plane_ptr = reinterpret_cast<const int*>(gm + h->geo[1].off[1]);
  L.plane_atoms = reinterpret_cast<const int*>(gm + h->geo[1].off[2]);
  L.max_plane = h->geo[1].extra;
  L.tables = ws + o_tab;
  L.t2 = ws + o_t2;
  L.tables_xmajor = ws + o_txm;
  if (prec == SHO_P_FF64) L.oz = ws + o_oz;
  L.stop_stage = h->stop_rows;
  L.chk = make_check(h, grid, nbands, natoms, numax, cube);
  if (bloch) {
    L.chk = DevCheck{};  // the Bloch kernels run unchecked
    BlochPh* ph = reinterpret_cast<BlochPh*>(ws + o_bloch);
    L.bloch = ph;
    const cudaError_t e = launch_bloch_phases(L.g, L.atoms, natoms, *bloch, ph, s);
    if (e != cudaSuccess) {
      h->last_cuda = e;
      h->last_where = "Bloch phases";
      return SHO_ERR_CUDA;
    }
  }
  L.scale = alpha;
  if (nl) L.nl = *nl;
  L.kernel = h->expand_kernel;
  L.wait_cycles = h->wait_cycles;
  L.status = h->dstatus;
  L.stream = s;
  const cudaError_t e = prec == SHO_P_FP64 ? launch_expand(L)
                        : prec == SHO_P_FF64 ? launch_expand_ff(L)
                        : fp32_stream_ok(psi, psi_dtype, nbands) ? launch_expand_fp32(L, prec)
                        : is_tc(prec) ? launch_expand_tc(L, prec)
                        : launch_expand(L);
  if (e != cudaSuccess) {
    h->last_cuda = e;
    h->last_where = "expansion launch";
    return SHO_ERR_CUDA;
  }
  return end_call(h, s);
}

int sho_add(sho_handle* h, const sho_grid* grid, const void* coeff, sho_dtype coeff_dtype, int nbands, int natoms,
            const double* pos, const double* sigma, int numax, int cube, sho_prec prec, void* psi,
            sho_dtype psi_dtype, void* stream) {
  return add_impl(h, grid, 1.0, 0, coeff, coeff_dtype, nbands, natoms, pos, sigma, numax, cube, prec, psi, psi_dtype,
                  stream);
}

int sho_add_scaled(sho_handle* h, const sho_grid* grid, double alpha, int overwrite, const void* coeff,
                   sho_dtype coeff_dtype, int nbands, int natoms, const double* pos, const double* sigma, int numax,
                   int cube, sho_prec prec, void* psi, sho_dtype psi_dtype, void* stream) {
  return add_impl(h, grid, alpha, overwrite, coeff, coeff_dtype, nbands, natoms, pos, sigma, numax, cube, prec, psi,
                  psi_dtype, stream);
}

int sho_forces(sho_handle* h, const sho_grid* grid, const void* psi, sho_dtype psi_dtype, int nbands, int natoms,
               const double* pos, const double* sigma, int numax, int cube, sho_prec prec, const void* dEdc,
               sho_dtype coeff_dtype, double* dEdX, void* stream) {
  if (!h) return SHO_ERR_ARG;
  SHO_TRY(check_common(grid, nbands, natoms, pos, sigma, numax, cube, SHO_MAX_NUMAX));
  SHO_TRY(check_dtypes(prec, psi_dtype, coeff_dtype));
  SHO_TRY(check_tc(prec, numax + 1, cube));
  SHO_TRY(check_spacing(h, grid, natoms, sigma, numax));
  SHO_TRY(check_support(h, prec));
  if (natoms == 0) return SHO_OK;
  if (!dEdX) return SHO_ERR_ARG;
  if (nbands > 0 && (!psi || !dEdc)) return SHO_ERR_ARG;
  DeviceGuard guard(h->device);
  if (!guard.ok) return SHO_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (nbands == 0) {
    SHO_TRY(begin_call(h, s));
    if (cudaMemsetAsync(dEdX, 0, sizeof(double) * 3 * (size_t)natoms, s) != cudaSuccess) return SHO_ERR_CUDA;
    return end_call(h, s);
  }
  std::vector<AtomDev> at = make_atoms(grid, natoms, pos, sigma, cube);
  std::vector<int> order = spatial_order(grid, at);
  const size_t tc = compute_size(coeff_dtype);
  Carve cv;
  const size_t o_atoms = cv.take(at.size() * sizeof(AtomDev));
  const size_t o_order = cv.take(order.size() * sizeof(int));
  const size_t o_cp = cv.take((size_t)natoms * nstates(numax + 1) * (size_t)nbands * tc);
  const size_t o_ft2 = prec == SHO_P_FF64 ? cv.take(ff_t2_bytes(natoms, cube, numax + 1, nbands)) : 0;
  SHO_TRY(begin_call(h, s));
  SHO_TRY(ensure_workspace(h, cv.off));
  SHO_TRY(upload(h, o_atoms, at.data(), at.size() * sizeof(AtomDev), s));
  SHO_TRY(upload(h, o_order, order.data(), order.size() * sizeof(int), s));
  char* ws = static_cast<char*>(h->ws);
  ProjectLaunch P;
  P.order = reinterpret_cast<const int*>(ws + o_order);
  P.g = make_grid(grid, cube, nbands, h->rprj);
  P.psi = psi;
  P.psi_dtype = psi_dtype;
  P.atoms = reinterpret_cast<const AtomDev*>(ws + o_atoms);
  P.natoms = natoms;
  P.numax = numax + 1;
  P.zsplit = prec == SHO_P_FF64 ? ff_zsplit(natoms, nbands, cube, h->sms) : zsplit_balanced(natoms, nbands, cube, h->sms);
  P.coeff = ws + o_cp;
  P.coeff_dtype = coeff_dtype;
  P.t2 = prec == SHO_P_FF64 ? ws + o_ft2 : nullptr;
  P.status = h->dstatus;
  P.chk = make_check(h, grid, nbands, natoms, numax + 1, cube);
  P.stream = s;
  const cudaError_t e = prec == SHO_P_FP64 ? launch_project(P)
                        : prec == SHO_P_FF64 ? launch_project_ff(P)
                        : fp32_stream_ok(psi, psi_dtype, nbands) ? launch_project_fp32(P, prec)
                        : is_tc(prec) ? launch_project_tc(P, prec)
                        : launch_project(P);
  if (e != cudaSuccess) return SHO_ERR_CUDA;
  ForcesLaunch F;
  F.natoms = natoms;
  F.numax = numax;
  F.nbands = nbands;
  F.atoms = P.atoms;
  F.cp = ws + o_cp;
  F.dEdc = dEdc;
  F.coeff_dtype = coeff_dtype;
  F.dEdX = dEdX;
  F.stream = s;
  if (launch_forces_contract(F) != cudaSuccess) return SHO_ERR_CUDA;
  return end_call(h, s);
}

// ------------------------------------------------------------------ non-local action
int sho_apply_nonlocal(sho_handle* h, const sho_grid* grid, const void* psi, sho_dtype psi_dtype, int nbands,
                       int natoms, const double* pos, const double* sigma, int numax, int cube, sho_prec prec,
                       const void* D, void* hpsi, void* stream) {
  if (!h) return SHO_ERR_ARG;
  SHO_TRY(check_common(grid, nbands, natoms, pos, sigma, numax, cube, SHO_MAX_NUMAX));
  const sho_dtype cdt = is_f64_form(prec) ? SHO_F64 : SHO_F32;
  SHO_TRY(check_dtypes(prec, psi_dtype, cdt));
  SHO_TRY(check_tc(prec, numax, cube));
  SHO_TRY(check_spacing(h, grid, natoms, sigma, numax));
  SHO_TRY(check_support(h, prec));
  if (natoms == 0 || nbands == 0) return SHO_OK;
  if (!psi || !hpsi || !D || psi == hpsi) return SHO_ERR_ARG;
  DeviceGuard guard(h->device);
  if (!guard.ok) return SHO_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The projection leaves its per-plane y-pass sums (paths with a separate z-pass: FP64-accurate form, plane
  // sweep) or its coefficients (the other paths) in a buffer of the handle; the expansion's z-pass kernel
  // then finishes the projection, multiplies by D and expands, with c and d in shared memory only.
  const size_t es = compute_size(cdt);
  const size_t nco = (size_t)natoms * nstates(numax) * (size_t)nbands * es;
  const size_t nt2 = (size_t)natoms * cube * (size_t)npairs(numax) * (size_t)nbands * es;
  const size_t need = std::max(nco, nt2);
  const size_t inner = std::max(workspace_bytes(SHO_OP_PROJECT, grid, natoms, numax, cube, nbands, cdt),
                                workspace_bytes(SHO_OP_EXPAND, grid, natoms, numax, cube, nbands, cdt));
  SHO_TRY(begin_call(h, s));
  if (!h->coeff_ws || h->coeff_ws_bytes < need) {
    if (h->has_last && cudaEventSynchronize(h->last) != cudaSuccess) return SHO_ERR_CUDA;
    if (h->coeff_ws) cudaFree(h->coeff_ws);
    h->coeff_ws = nullptr;
    h->coeff_ws_bytes = 0;
    if (cudaMalloc(&h->coeff_ws, need) != cudaSuccess) {
      cudaGetLastError();
      return SHO_ERR_OOM;
    }
    h->coeff_ws_bytes = need;
  }
  SHO_TRY(ensure_workspace(h, inner));
  void* buf = h->coeff_ws;
  bool at_t2 = false;
  SHO_TRY(project_impl(h, grid, psi, psi_dtype, nbands, natoms, pos, sigma, numax, cube, prec, buf, cdt, stream, buf,
                       &at_t2));
  NonlocalIn nl;
  nl.D = D;
  nl.t2p = at_t2 ? buf : nullptr;
  nl.c = at_t2 ? nullptr : buf;
  nl.h3 = grid->h * grid->h * grid->h;
  return add_impl(h, grid, 1.0, 0, buf, cdt, nbands, natoms, pos, sigma, numax, cube, prec, hpsi, psi_dtype, stream,
                  &nl);
}

// ------------------------------------------------------------------ stored-projector baseline
int sho_usu_build(sho_handle* h, const sho_grid* grid, int natoms, const double* pos, const double* sigma, int numax,
                  int nproj, int cube, sho_dtype dtype, void* proj, void* stream) {
  if (!h) return SHO_ERR_ARG;
  if (dtype != SHO_F64 && dtype != SHO_F32) return SHO_ERR_DTYPE;
  SHO_TRY(check_common(grid, 0, natoms, pos, sigma, numax, cube, SHO_USU_MAX_NUMAX));
  if (nproj < 1 || nproj > nstates(numax) || !usu_supported_nproj(nproj)) return SHO_ERR_ARG;
  if (natoms == 0) return SHO_OK;
  if (!proj) return SHO_ERR_ARG;
  DeviceGuard guard(h->device);
  if (!guard.ok) return SHO_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<AtomDev> at = make_atoms(grid, natoms, pos, sigma, cube);
  Carve cv;
  const size_t o_atoms = cv.take(at.size() * sizeof(AtomDev));
  SHO_TRY(begin_call(h, s));
  SHO_TRY(ensure_workspace(h, cv.off));
  SHO_TRY(upload(h, o_atoms, at.data(), at.size() * sizeof(AtomDev), s));
  UsuLaunch L = {};
  L.g = make_grid(grid, cube, 0, h->rprj);
  L.atoms = reinterpret_cast<const AtomDev*>(static_cast<char*>(h->ws) + o_atoms);
  L.natoms = natoms;
  L.numax = numax;
  L.nproj = nproj;
  L.dtype = dtype;
  L.proj = proj;
  L.stream = s;
  if (launch_usu(0, L) != cudaSuccess) return SHO_ERR_CUDA;
  return end_call(h, s);
}

int sho_usu_project(sho_handle* h, const sho_grid* grid, const void* psi, int nbands, int natoms,
                    const double* pos, const double* sigma, int nproj, int cube, sho_dtype dtype, const void* proj,
                    void* coeff, void* stream) {
  if (!h) return SHO_ERR_ARG;
  if (dtype != SHO_F64 && dtype != SHO_F32) return SHO_ERR_DTYPE;
  SHO_TRY(check_common(grid, nbands, natoms, pos, sigma, 0, cube, SHO_USU_MAX_NUMAX));
  if (!usu_supported_nproj(nproj)) return SHO_ERR_ARG;
  if (natoms == 0 || nbands == 0) return SHO_OK;
  if (!psi || !proj || !coeff) return SHO_ERR_ARG;
  DeviceGuard guard(h->device);
  if (!guard.ok) return SHO_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<AtomDev> at = make_atoms(grid, natoms, pos, sigma, cube);
  Carve cv;
  const size_t o_atoms = cv.take(at.size() * sizeof(AtomDev));
  SHO_TRY(begin_call(h, s));
  SHO_TRY(ensure_workspace(h, cv.off));
  SHO_TRY(upload(h, o_atoms, at.data(), at.size() * sizeof(AtomDev), s));
  UsuLaunch L = {};
  L.g = make_grid(grid, cube, nbands, h->rprj);
  L.atoms = reinterpret_cast<const AtomDev*>(static_cast<char*>(h->ws) + o_atoms);
  L.natoms = natoms;
  L.nproj = nproj;
  L.zsplit = zsplit_balanced(natoms, nbands, cube, h->sms);
  L.dtype = dtype;
  L.proj = const_cast<void*>(proj);
  L.psi_in = psi;
  L.coeff_out = coeff;
  L.stream = s;
  if (launch_usu(1, L) != cudaSuccess) return SHO_ERR_CUDA;
  return end_call(h, s);
}

int sho_usu_add(sho_handle* h, const sho_grid* grid, const void* coeff, int nbands, int natoms, const double* pos,
                const double* sigma, int nproj, int cube, sho_dtype dtype, const void* proj, void* psi, void* stream) {
  if (!h) return SHO_ERR_ARG;
  if (dtype != SHO_F64 && dtype != SHO_F32) return SHO_ERR_DTYPE;
  SHO_TRY(check_common(grid, nbands, natoms, pos, sigma, 0, cube, SHO_USU_MAX_NUMAX));
  if (!usu_supported_nproj(nproj)) return SHO_ERR_ARG;
  if (natoms == 0 || nbands == 0) return SHO_OK;
  if (!psi || !proj || !coeff) return SHO_ERR_ARG;
  DeviceGuard guard(h->device);
  if (!guard.ok) return SHO_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<AtomDev> at = make_atoms(grid, natoms, pos, sigma, cube);
  std::vector<int> ptr, list;
  plane_lists(grid, at, cube, ptr, list);
  Carve cv;
  const size_t o_atoms = cv.take(at.size() * sizeof(AtomDev));
  const size_t o_ptr = cv.take(ptr.size() * sizeof(int));
  const size_t o_list = cv.take(std::max<size_t>(1, list.size()) * sizeof(int));
  SHO_TRY(begin_call(h, s));
  SHO_TRY(ensure_workspace(h, cv.off));
  SHO_TRY(upload(h, o_atoms, at.data(), at.size() * sizeof(AtomDev), s));
  SHO_TRY(upload(h, o_ptr, ptr.data(), ptr.size() * sizeof(int), s));
  SHO_TRY(upload(h, o_list, list.data(), list.size() * sizeof(int), s));
  char* ws = static_cast<char*>(h->ws);
  UsuLaunch L = {};
  L.g = make_grid(grid, cube, nbands, h->rprj);
  L.atoms = reinterpret_cast<const AtomDev*>(ws + o_atoms);
  L.natoms = natoms;
  L.nproj = nproj;
  L.dtype = dtype;
  L.proj = const_cast<void*>(proj);
  L.coeff_in = coeff;
  L.psi_out = psi;
  L.plane_ptr = reinterpret_cast<const int*>(ws + o_ptr);
  L.plane_atoms = reinterpret_cast<const int*>(ws + o_list);
  L.stream = s;
  if (launch_usu(2, L) != cudaSuccess) return SHO_ERR_CUDA;
  return end_call(h, s);
}

int sho_set_expand_kernel(sho_handle* h, int kernel) {
  if (!h || kernel < SHO_KERNEL_AUTO || kernel > SHO_KERNEL_TCGEN05) return SHO_ERR_ARG;
  h->expand_kernel = kernel;
  return SHO_OK;
}

int sho_set_project_kernel(sho_handle* h, int kernel) {
  if (!h || kernel < SHO_KERNEL_AUTO || kernel > SHO_KERNEL_TCGEN05) return SHO_ERR_ARG;
  h->project_kernel = kernel;
  return SHO_OK;
}

int sho_set_device_checks(sho_handle* h, int on) {
  if (!h) return SHO_ERR_ARG;
  h->dev_checks = on != 0;
  return SHO_OK;
}

int sho_set_support_radius(sho_handle* h, double rprj) {
  if (!h || !std::isfinite(rprj) || rprj < 0.0) return SHO_ERR_ARG;
  h->rprj = rprj;
  return SHO_OK;
}

// ------------------------------------------------------------------ fault injection (include/sho_fault.h)
int sho_fault_wait_limit(sho_handle* h, long long cycles) {
  if (!h || cycles < 0) return SHO_ERR_ARG;
  h->wait_cycles = cycles == 0 ? kDefaultWaitCycles : cycles;
  return SHO_OK;
}

int sho_fault_stop_rows(sho_handle* h, int rows) {
  if (!h) return SHO_ERR_ARG;
  h->stop_rows = rows < 0 ? 0x7fffffff : rows;
  return SHO_OK;
}

int sho_fault_check_extent(sho_handle* h, long long psi_elems) {
  if (!h) return SHO_ERR_ARG;
  h->check_psi_cap = psi_elems < 0 ? -1 : psi_elems;
  return SHO_OK;
}

}  // extern "C"
