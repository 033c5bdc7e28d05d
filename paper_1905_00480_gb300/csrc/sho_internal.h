// sho_internal.h -- structures shared by the host API and the kernels of libsho (not installed).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sho.h"
#include "../../include/sho_fault.h"
#include "../../include/sho_selftest.h"

namespace sho {

constexpr int kMaxCube = 64;      // largest cube edge (points), a multiple of 8
constexpr int kWarp = 32;         // bands per warp tile
constexpr int kMaxTableNu = SHO_MAX_NUMAX + 1;  // forces project at numax + 1
constexpr int kMaxStates = (SHO_MAX_NUMAX + 1) * (SHO_MAX_NUMAX + 2) * (SHO_MAX_NUMAX + 3) / 6;

// Per-atom data uploaded by the host plan: position, width and the integer cube origin
// o_d = floor(X_d / h) - cube/2 + 1 computed on the host.
struct AtomDev {
  double X[3];
  double sigma;
  int o[3];
  int pad;
};
static_assert(sizeof(AtomDev) == 48, "AtomDev layout");

// Geometry common to all kernels.
struct GridDev {
  int n[3];          // Nx, Ny, Nz
  int periodic;
  double h;
  int cube;
  int nbands;
  double r2max = 0.0;  // spherical support: R^2 of the projection sphere; 0 = the whole cube
};

enum class Real { F64, F32 };

// Bits of a handle's device status word (read and cleared by sho_sync): a bounded wait on the kernel's
// own data pipeline expired; an FP64-accurate (float-float) input lay outside the float normal range.
constexpr int kStatusTimeout = 1;
constexpr int kStatusRange = 2;
constexpr int kStatusBounds = 4;  // device checks: an index outside its buffer (the access was skipped)

// Device checks (sho_set_device_checks): the extents, in elements, of the buffers the checked kernels
// index -- psi, the coefficients and the z-pass / per-plane intermediate -- and the status word that an
// index outside its extent sets (kStatusBounds).  flag == nullptr: checks off, unchecked kernels run.
struct DevCheck {
  long long psi_n = 0, coeff_n = 0, t2_n = 0;
  int* flag = nullptr;
};

// Bloch transforms on the real kernels (Sec. 2.5; periodic grid; FP64-accurate and FP32 forms): per atom
// the phase factors of its cube's lattice translations as float pairs (re.hi, re.lo, im.hi, im.lo; the
// FP32 form reads the leading floats).  Along axis d the cube points
// i < w[d] map into the cell with translation T_d = f0_d n_d h and those from w[d] on with (f0_d + 1) n_d h
// (w[d] >= cube: no crossing); ph[bx + 2 by + 4 bz] = e^{s i k.T} for the translation with bits b_d =
// (i_d >= w[d]), s = +1 for the projection and -1 for the expansion; xstep = ph[0] / ph[1] = e^{-s i k_x n_x h}.
struct BlochPh {
  float4 ph[8];
  float4 xstep;
  int w[4];
};
static_assert(sizeof(BlochPh) == 160, "BlochPh layout");
constexpr int kBlochRealMaxNumax = 7;  // Bloch variants of the real kernels (FP64-accurate, FP32): numax 0..7
struct BlochArg {
  double k[3];  // Bloch vector
  double sgn;   // +1 projection, -1 expansion
};
// ph[a] for every atom from its cube origin (one thread per atom, FP64 sincos)
cudaError_t launch_bloch_phases(const GridDev& g, const AtomDev* atoms, int natoms, const BlochArg& arg, BlochPh* ph,
                                cudaStream_t s);

// Bounded waits of the device pipelines give up after this many SM clock cycles (~2 s at 2.07 GHz)
// unless a handle's fault-injection setting (include/sho_fault.h) shortens it.
constexpr long long kDefaultWaitCycles = 4000000000ll;

struct ProjectLaunch {
  GridDev g;
  const void* psi;          // [Nz][Ny][Nx][B]
  sho_dtype psi_dtype;
  const AtomDev* atoms;     // device [A]
  int natoms;
  int numax;
  int zsplit;               // cube z-planes split over this many CTAs (of one cluster, FP64 form)
  const int* order = nullptr;  // optional device [A]: atoms in spatial (Morton) order of their cubes
  void* coeff;              // [A][N][B], FP64 or FP32
  void* t2 = nullptr;       // FP64-accurate form: workspace [A][cube][P][B] FP64 of per-plane y-pass sums
  sho_dtype coeff_dtype;
  int* status = nullptr;    // FP64-accurate form: device status word (kStatusRange), may be null
  bool t2_only = false;     // FP64-accurate form: stop after the per-plane sums (the z-pass runs fused later)
  DevCheck chk;             // device checks (FP64 and FP64-accurate kernels), off by default
  const BlochPh* bloch = nullptr;  // Bloch projection (FP64-accurate, FP32): device [A] phases; psi and coeff
                                   // are complex, their (re, im) pairs counted as 2 real bands (g.nbands)
  void* op = nullptr;       // FP64-accurate form on the tensor cores: op_layout() workspace, may be null
  int kernel = 0;           // FP64-accurate x-pass engine: 0 automatic, 1 float-float, 2 tcgen05
  long long wait_cycles = kDefaultWaitCycles;  // limit of the bounded waits (tensor-core kernel)
  cudaStream_t stream;
};

// Workspace of the FP64-accurate projection on the tensor cores (sho_ozaki_project.cu), offsets in bytes
// from ProjectLaunch::op, each region 256-byte aligned: the stacked digit tables of the x functions
// [A][6][4][64][8] BF16, the per-atom power of two G_a [A] and the y functions as float pairs
// [A][numax+1][cube].
struct OpLayout {
  size_t btab, gpow, tyff, total;
};
inline OpLayout op_layout(int natoms, int cube, int numax) {
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  OpLayout L;
  L.btab = 0;
  L.gpow = up((size_t)natoms * 6 * 4 * 64 * 8 * 2);
  L.tyff = L.gpow + up((size_t)natoms * sizeof(float));
  L.total = L.tyff + up((size_t)natoms * (numax + 1) * cube * 2 * sizeof(float));
  return L;
}
bool ozaki_project_ok(const ProjectLaunch& p);
cudaError_t launch_project_ozaki(const ProjectLaunch& p);

// Inputs of the fused non-local action (Sec. 3.2 steps 1-3) taken by the expansion's z-pass kernel: the
// projection coefficients c of each (atom, band) -- from the projection's per-plane y-pass sums t2p
// ([A][cube][P][B], z-pass and h^3 applied here) or, when t2p is null, from c ([A][N][B]) -- are multiplied
// by the atom's matrix, d = D c, in shared memory, and d feeds the expansion; neither c nor d goes to
// global memory.  All arrays in the expansion's compute type.  D == nullptr: a plain expansion.
struct NonlocalIn {
  const void* D = nullptr;    // [A][N][N]
  const void* t2p = nullptr;  // [A][cube][P][B] per-plane y-pass sums of the projection
  const void* c = nullptr;    // [A][N][B] projection coefficients (when t2p is null)
  double h3 = 1.0;            // projection weight applied with the projection's z-pass
};

struct ExpandLaunch {
  GridDev g;
  const void* coeff;        // [A][N][B]
  sho_dtype coeff_dtype;
  void* psi;                // [Nz][Ny][Nx][B], read-modify-write
  sho_dtype psi_dtype;
  const AtomDev* atoms;     // device [A]
  int natoms;
  int numax;
  const int* plane_ptr;     // [Nz + 1]: atoms whose cube covers plane z are
  const int* plane_atoms;   //   plane_atoms[plane_ptr[z] .. plane_ptr[z+1]), ascending
  int max_plane;            // longest per-plane list
  void* tables;             // workspace [A][2][numax+1][cube] of the compute type (x and y tables)
  void* t2;                 // workspace [A][cube][P][B] of the compute type (z-pass result); the FP32
                            // block gather takes it band-tiled, t2_bytes() covers both
  void* tables_xmajor = nullptr;  // optional workspace, txm_bytes_per_point(numax) bytes per (atom, cube
                                  // point): the FP32 x table x-major [A][cube][NPX], then (tensor forms)
                                  // the B fragments of the x-pass; FP64-accurate form: float-pair tables
  void* tables_ymajor = nullptr;  // optional: the FP32 y table y-major [A][cube][NPX] (tensor-memory kernel)
  double scale = 1.0;       // psi += scale * E c: applied to the z table of the z-pass
  NonlocalIn nl;            // fused non-local action (nl.D set): the coefficients are D times a projection
  int kernel = 0;           // FP32-class x-pass engine: 0 automatic, 1 warp-level mma.sync, 2 tcgen05
  long long wait_cycles = kDefaultWaitCycles;  // limit of the bounded waits (tcgen05 kernel)
  int* status = nullptr;    // FP64-accurate form: device status word (kStatusRange), may be null
  void* oz = nullptr;       // FP64-accurate form on the tensor cores: oz_layout() workspace, may be null
  int stop_stage = 0x7fffffff;  // fault injection: that kernel stages the z-pass slices of this many atoms
  DevCheck chk;             // device checks (FP64 and FP64-accurate kernels), off by default
  const BlochPh* bloch = nullptr;  // Bloch expansion (FP64-accurate, FP32): device [A] phases (complex data as
                                   // 2 real bands per band, as for the projection)
  cudaStream_t stream;
};

// Workspace of the FP64-accurate expansion on the tensor cores (sho_ozaki.cu), offsets in bytes from
// ExpandLaunch::oz, each region 256-byte aligned: the digit tables of the x functions
// [A][6 digits][2 state chunks][96 rows][4] floats, the per-atom power of two G_a [A], and the bound
// max_y max_nx |T1[nx]| of each (atom, plane, band) [A][C][B] (floats).
struct OzLayout {
  size_t dtab, gpow, tmax, total;
};
inline OzLayout oz_layout(int natoms, int cube, int nbands) {
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  OzLayout L;
  L.dtab = 0;
  L.gpow = up((size_t)natoms * 6 * 2 * 96 * 4 * sizeof(float));
  L.tmax = L.gpow + up((size_t)natoms * sizeof(float));
  L.total = L.tmax + up((size_t)natoms * cube * (size_t)nbands * sizeof(float));
  return L;
}

// Bytes per (atom, cube point) of ExpandLaunch::tables_xmajor, NPX = numax + 1 rounded up to 4: the
// float-pair tables of the FP64-accurate form fit in 16 NPX; the FP32 x table with up to four
// 16-byte B-fragment entries behind it in 4 NPX + 64.
// Pairs per band row of the band-tiled z-pass result [A][C][B/32][32][PP]: P rounded up to 4, plus 4
// when that is a multiple of 8, so that the 16-byte row loads of 8 consecutive lanes hit distinct banks.
__host__ __device__ constexpr int tiled_pairs(int P) {
  return ((P + 3) / 4 * 4) % 8 == 0 ? (P + 3) / 4 * 4 + 4 : (P + 3) / 4 * 4;
}

// Bytes of ExpandLaunch::t2: [A][cube][P][B] of the compute type, or band-tiled FP32
// [A][cube][ceil(B/32)][32][tiled_pairs(P)], whichever is larger.
inline size_t t2_bytes(int natoms, int cube, int numax, int nbands, size_t elem) {
  const size_t P = (size_t)((numax + 1) * (numax + 2) / 2);
  const size_t PP = (size_t)tiled_pairs((int)P);
  const size_t plain = (size_t)natoms * cube * P * (size_t)nbands * elem;
  const size_t tiled = (size_t)natoms * cube * (size_t)((nbands + 31) / 32) * 32 * PP * sizeof(float);
  return plain > tiled ? plain : tiled;
}

// Bytes of ProjectLaunch::t2 for the FP64-accurate form.
inline size_t ff_t2_bytes(int natoms, int cube, int numax, int nbands) {
  return (size_t)natoms * cube * (size_t)((numax + 1) * (numax + 2) / 2) * (size_t)nbands * sizeof(double);
}

// Cube z-slabs per (atom, band tile) of the FP64-accurate projection: enough CTAs for about two waves
// of eleven one-warp CTAs per SM, at least two planes per slab.
inline int ff_zsplit(int natoms, int nbands, int cube, int sms) {
  const long long ctas = (long long)natoms * ((nbands + 31) / 32);
  int zs = 1;
  while (zs * 2 <= cube / 2 && ctas * zs < 22LL * sms) zs *= 2;
  return zs;
}

inline size_t txm_bytes_per_point(int numax) {
  const size_t npx = (size_t)((numax + 4) & ~3);
  return npx * 16 > npx * 4 + 64 ? npx * 16 : npx * 4 + 64;
}

struct ForcesLaunch {
  int natoms;
  int numax;                // numax of dEdc; cp holds numax + 1
  int nbands;
  const AtomDev* atoms;
  const void* cp;           // [A][N(numax+1)][B], compute type
  const void* dEdc;         // [A][N(numax)][B], coefficient type
  sho_dtype coeff_dtype;
  double* dEdX;             // [A][3]
  cudaStream_t stream;
};

// Stored-projector baseline: op 0 = sample projectors, 1 = project, 2 = add.
struct UsuLaunch {
  GridDev g;
  const AtomDev* atoms;
  int natoms;
  int numax;                // build: basis the stored projectors are taken from
  int nproj;                // number of stored projectors (the first nproj states of that basis)
  int zsplit;
  sho_dtype dtype;          // F64 or F32: type of every array below
  void* proj;               // [A][C^3][nproj]
  const void* psi_in;       // project: psi
  void* coeff_out;          // project: coefficients
  const void* coeff_in;     // add: coefficients
  void* psi_out;            // add: psi (read-modify-write)
  const int* plane_ptr;
  const int* plane_atoms;
  cudaStream_t stream;
};

// Plane-sweep projection of the FP32-class forms (sho_plane.cu).  A row segment is the run of grid
// rows [ys, ye) of plane z that atom `atom` covers at cube plane iz, starting at cube row iy0; x0 is
// the grid x of the atom's first cube point (wrapped when periodic).  flags: 0 whole, 1 tail of a
// wrapped atom (rows [0, e)), 2 head (rows [s, Ny), continues from the tail's partial sums).
struct PlaneSeg {
  int atom, iz, iy0, x0;
  int ys, ye, flags, t2i;  // t2i = atom * cube + iz: row of the T2 buffer
};
struct PlanePlan {
  std::vector<int4> items;   // per CTA row: (z, ylo, yhi, first slot list)
  std::vector<int> slot_ptr; // CSR over items x warps x slots -> segs
  std::vector<PlaneSeg> segs;
};
struct PlaneLaunch {
  GridDev g;
  const void* psi;           // [Nz][Ny][Nx][B] FP32 or BF16, 16-byte aligned, rows of whole 16-byte units
  sho_dtype psi_dtype;       // SHO_F32 or SHO_BF16
  const AtomDev* atoms;
  int natoms;
  int numax;
  const int4* items;
  int nitems;
  const int* slot_ptr;
  const PlaneSeg* segs;
  float* xtab;               // [A][C][8]
  float* ytab;               // [A][C][8]
  uint32_t* bfrag;           // [A][32][kMaxCube / 8][4]
  float* t2p;                // [A][C][P][B]
  float* coeff;              // [A][N][B]
  int* status;               // device status word: kStatusTimeout when a bounded wait expired
  long long wait_cycles = kDefaultWaitCycles;  // limit of every mbarrier wait
  int stop_rows = 0x7fffffff;  // fault injection: producers issue only this many rows per sweep
  bool t2_only = false;        // stop after the per-plane sums t2p (the z-pass runs fused later)
  cudaStream_t stream;
};
bool plane_ok(const sho_grid* grid, const void* psi, sho_dtype psi_dt, int nbands, int numax, int cube,
              sho_prec prec);
void plan_planes(const sho_grid* grid, const std::vector<AtomDev>& at, int cube, PlanePlan& plan);
cudaError_t launch_project_plane(const PlaneLaunch& p, sho_prec prec);
int plane_plan_check(const sho_grid* grid, const std::vector<AtomDev>& at, int cube, const PlanePlan& plan);
constexpr size_t kPlaneBfragBytesPerAtom = 32 * (kMaxCube / 8) * 4 * sizeof(uint32_t);

// Cartesian <-> radial transform (sho_radial.cu): labels and U on the host, CSR rows for the kernel.
int radial_labels(int numax, int* nr, int* l, int* m);
const double* radial_matrix(int numax);
void radial_csr(int numax, int direction, std::vector<int>& rowp, std::vector<int>& col, std::vector<double>& val);
cudaError_t launch_radial(int natoms, int N, int nbands, sho_dtype dt, const int* rowp, const int* col,
                          const void* val, const void* in, void* out, cudaStream_t s);

// Bloch (complex) projection / expansion, FP64 (sho_bloch.cu).  Complex arrays hold (re, im) pairs.
struct BlochLaunch {
  GridDev g;                // periodic
  const AtomDev* atoms;
  int natoms;
  int numax;
  double k[3];              // Bloch vector
  int op;                   // 0: project, 1: expand
  int zsplit;               // projection: cube z-slabs per (atom, band tile)
  const double* psi_in;     // project: psi [Nz][Ny][Nx][B][2]
  double* coeff_out;        // project: [A][N][B][2]
  const double* coeff_in;   // expand: [A][N][B][2]
  double* psi_out;          // expand: psi, read-modify-write
  const int* plane_ptr;     // expand: per-plane atom lists (CSR), ascending
  const int* plane_atoms;
  double* tab;              // [A][3][numax+1][C][2]
  double* work;             // project: [zsplit][A][N][B][2]; expand: [A][C][P][B][2]
  cudaStream_t stream;
};
cudaError_t launch_bloch(const BlochLaunch& p);
constexpr int kBlochMaxNx = 448;  // the expansion keeps one grid row of 32 complex bands in shared memory

// Kernel launchers (return a CUDA error code).
cudaError_t launch_usu(int op, const UsuLaunch& p);
bool usu_supported_nproj(int n);
cudaError_t launch_expand_zpass_f32(const ExpandLaunch& p);
cudaError_t launch_expand_zpass_f32_tiled(const ExpandLaunch& p);  // T2 as [A][C][B/32][32][tiled_pairs(P)]
cudaError_t launch_expand_zpass_f64(const ExpandLaunch& p);
// the same z-pass with T2 and the x / y tables written as float pairs (FP64-accurate expansion)
cudaError_t launch_expand_zpass_ff(const ExpandLaunch& p, float2* txff, float2* tyff);
cudaError_t launch_project_ff(const ProjectLaunch& p);
cudaError_t launch_expand_ff(const ExpandLaunch& p);
// FP64-accurate expansion with the x-pass on the tensor cores (exact digit slices); the caller has run the
// float-pair z-pass (T2 as float pairs, float-pair y tables at `tyff`)
bool ozaki_expand_ok(const ExpandLaunch& p);
cudaError_t launch_expand_ozaki(const ExpandLaunch& p, const void* tyff);
cudaError_t launch_project_tc(const ProjectLaunch& p, sho_prec prec);
cudaError_t launch_expand_tc(const ExpandLaunch& p, sho_prec prec);
// Streaming FP32-class kernels (cp.async row pipeline / block gather), used when rows of bands are
// 16-byte aligned (fp32_stream_ok); the CUDA-core / tensor-core row kernels serve the other cases.
bool fp32_stream_ok(const void* psi, sho_dtype dt, int nbands);
cudaError_t launch_project_fp32(const ProjectLaunch& p, sho_prec prec);
// Block-gather expansion with the x-pass on tcgen05 MMAs and the tile in tensor memory (TF32 and BF16
// forms, numax <= 7, FP32 or BF16 psi, no spherical support; sho_umma_expand.cu).
bool umma_expand_ok(const ExpandLaunch& p, sho_prec prec);
cudaError_t launch_expand_umma(const ExpandLaunch& p, sho_prec prec);
cudaError_t launch_expand_fp32(const ExpandLaunch& p, sho_prec prec);

// Host helpers shared with the serving loop and the allocation-free entry point (sho_api.cu).
int choose_zsplit(int natoms, int nbands, int cube, int sms);
// Read and clear the handle's device status word (the handle's work must have completed): SHO_OK,
// SHO_ERR_TIMEOUT (a bounded wait expired) or SHO_ERR_DEVICE (an input outside the form's range).
int handle_take_status(sho_handle* h);
size_t workspace_bytes(sho_op op, const sho_grid* grid, int natoms, int numax, int cube, int nbands,
                       sho_dtype coeff_dtype);
int handle_reserve(sho_handle* h, size_t bytes);
size_t handle_workspace(const sho_handle* h);

constexpr int kTcMaxNumax = 7;  // tensor-core forms: eight 1D functions fill one MMA tile

inline bool is_tc(sho_prec p) {
  return p == SHO_P_TF32 || p == SHO_P_3XTF32 || p == SHO_P_BF16 || p == SHO_P_SPLIT_FP16;
}
cudaError_t launch_project(const ProjectLaunch& p);
cudaError_t launch_expand(const ExpandLaunch& p);
cudaError_t launch_forces_contract(const ForcesLaunch& p);

// Bytes of compute-type scalars for a dtype.
inline size_t compute_size(sho_dtype coeff_dtype) { return coeff_dtype == SHO_F64 ? 8 : 4; }
inline bool is_f64_form(sho_prec p) { return p == SHO_P_FP64 || p == SHO_P_FF64; }

inline int nstates(int nu) { return nu < 0 ? 0 : (nu + 1) * (nu + 2) * (nu + 3) / 6; }
inline int npairs(int nu) { return nu < 0 ? 0 : (nu + 1) * (nu + 2) / 2; }

}  // namespace sho
