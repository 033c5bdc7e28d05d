// sho_ff.cu -- the FP64-accurate form with float-float x-passes (SHO_P_FF64).
//
// Same decomposition, cube convention and deterministic reductions as the FP64 kernels
// (sho_project.cu, sho_expand.cu).  On GB300 the FP64 pipe runs at 1/61 of the FP32 pipe, and the
// x-pass is 89 % of the FMAs of a projection or expansion (C^3 (numax+1) of C^3 (numax+1) + C^2 P + C N
// per atom-band).  Here that pass and the y-pass run as float-float dot products on the FP32 pipe
// (sho_ff.cuh); the 1D tables are generated in FP64 and split once, and the z-pass and the final
// accumulation into psi are FP64.
//   projection  T1[n] = sum_x psi[x] phi_n(x): psi split into float pairs with integer instructions,
//               then one float-float dot step per (x, n); the y-pass sums of each cube plane go to a
//               workspace in FP64 and a second kernel runs the z-pass over the planes in order.
//   expansion   the update sum_a sum_n T1_a[n] phi_n(x) of each grid point is one float-float dot
//               product over all atoms and states, its running pair kept in shared memory (block gather
//               over 8-row x 32-point tiles), and added to psi in FP64 once.
#include <type_traits>

#include "sho_device.cuh"
#include "sho_ff.cuh"

namespace sho {

// ------------------------------------------------------------------------------- projection
constexpr int kFfStages = 2;   // cp.async ring depth (rows of 32 x points x 32 bands x 8 bytes)
constexpr int kFfRowBytes = 32 * 8;

__device__ __forceinline__ uint32_t ff_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void ff_cp16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void ff_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void ff_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

template <int NU>
struct FfProjectSmem {
  static constexpr int NP = NU + 1, NPX = (NP + 1) & ~1;
  static size_t bytes(int cube) {
    size_t t = (size_t)kFfStages * cube * kFfRowBytes;             // ring of psi rows
    t += (size_t)cube * NPX * sizeof(float2);                      // x table (pairs), x-major
    t += (size_t)NP * cube * sizeof(float2);                       // y table (pairs)
    t += (size_t)cube * sizeof(long long);                         // x offsets
    t += (size_t)2 * cube * sizeof(int);                           // y and z grid indices
    return t;
  }
};

// x- and y-passes of one (atom, 32-band tile, slab of cube planes): T2[a][iz][P][B] of each plane of
// the slab, converted from its float pair to FP64, goes to a workspace; the z-pass is k_project_ff_zpass.
// Without z-pass accumulators a lane holds about 130 registers, and the ring two rows.
// CHK: device checks of every psi and workspace index (sho_set_device_checks), a separate instantiation.
// BLOCH: complex psi of a Bloch wave (Sec. 2.5), its (re, im) pairs as two real bands in neighbouring
// lanes; the x-pass sum turns by the x translation's phase where the cube row crosses the cell boundary,
// and each row's x-pass result by the phase of its translation, so that the y- and z-passes stay real.
template <int NU, bool CHK = false, bool BLOCH = false>
__global__ void __launch_bounds__(kWarp) k_project_ff(GridDev g, const double* __restrict__ psi,
                                                      const AtomDev* __restrict__ atoms, int zsplit,
                                                      double* __restrict__ t2g, int* __restrict__ status,
                                                      DevCheck dc, const BlochPh* __restrict__ bph) {
  using BS = Basis<NU>;
  using SM = FfProjectSmem<NU>;
  constexpr int NP = BS::NP, P = BS::P, NPX = SM::NPX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int C = g.cube;
  unsigned char* ring = smem_raw;
  float2* phx = reinterpret_cast<float2*>(ring + (size_t)kFfStages * C * kFfRowBytes);  // [C][NPX] pairs
  float2* phy = phx + (size_t)C * NPX;                                       // [NP][C] pairs
  long long* xoff = reinterpret_cast<long long*>(phy + (size_t)NP * C);      // [C]
  int* yidx = reinterpret_cast<int*>(xoff + C);                              // [C] grid row of cube row
  int* zidx = yidx + C;                                                      // [C] grid plane of cube plane

  const int lane = threadIdx.x;
  const int a = blockIdx.z;
  const int B = g.nbands;
  const int b0 = blockIdx.y * kWarp;
  const bool bok = b0 + lane < B;
  const AtomDev at = atoms[a];

  for (int i = lane; i < C; i += kWarp) {
    double col[NP];
    phi_column(cube_offset(at.o[0], i, g.h, at.X[0]), at.sigma, NU, col, 1);
#pragma unroll
    for (int n = 0; n < NPX; n++) {
      const ff f = n < NP ? ff_from_double_exact(col[n]) : ff{0.0f, 0.0f};
      phx[i * NPX + n] = make_float2(f.hi, f.lo);
    }
    phi_column(cube_offset(at.o[1], i, g.h, at.X[1]), at.sigma, NU, col, 1);
#pragma unroll
    for (int n = 0; n < NP; n++) {
      const ff f = ff_from_double_exact(col[n]);
      phy[n * C + i] = make_float2(f.hi, f.lo);
    }
    const int jx = cube_index(at.o[0], i, g.n[0], g.periodic);
    xoff[i] = jx < 0 ? -1ll : (long long)jx * B;
    yidx[i] = cube_index(at.o[1], i, g.n[1], g.periodic);
    zidx[i] = cube_index(at.o[2], i, g.n[2], g.periodic);
  }
  __syncwarp();

  const int chunk = (C + zsplit - 1) / zsplit;
  const int iz0 = blockIdx.x * chunk, iz1 = min(C, iz0 + chunk);
  const int R = max(0, iz1 - iz0) * C;
  const long long rowlen = (long long)g.n[0] * B;
  const int valid_bytes = (B - b0) * 8;
  const int cpart = lane & 15;                                      // this lane's 16-byte chunk of a point
  const int cbytes = min(16, max(0, valid_bytes - cpart * 16));     // its bytes inside the band tile
  // 16-byte asynchronous copies need every (grid point, band tile) run of psi to start on a 16-byte
  // boundary: an even band count and a 16-byte aligned base.  Otherwise the ring is filled with
  // plain 8-byte loads (same data layout, no overlap of loads and compute).
  const bool async_ok = ((B & 1) == 0) && (((uintptr_t)psi & 15u) == 0);

  // copies of the next slab row r (x points x 32 bands) into ring stage r % kFfStages; rows are issued
  // in order, their cube plane and row kept as counters
  int qr = 0, qz = iz0, qy = 0;
  auto issue_next = [&]() {
    const int r = qr, iz = qz, iy = qy;
    qr++;
    if (++qy == C) {
      qy = 0;
      qz++;
    }
    if (r >= R) return;
    const int jz = zidx[iz], jy = yidx[iy];
    if (jz < 0 || jy < 0) return;
    const long long row0 = ((long long)jz * g.n[1] + jy) * rowlen + b0;  // psi index of the row's x = 0
    const double* row = psi + row0;
    unsigned char* st = ring + (size_t)(r % kFfStages) * C * kFfRowBytes;
    if (async_ok) {
      // 16 chunks of 16 bytes per x point: this lane copies chunk `cpart` of every other x point
      const unsigned char* rowb = reinterpret_cast<const unsigned char*>(row) + cpart * 16;
      const uint32_t dst0 = ff_smem_u32(st + cpart * 16);
      for (int x = lane >> 4; x < C; x += 2) {
        const long long o = xoff[x];
        const bool ok = o >= 0 && cbytes > 0 &&
                        dc_ok<CHK>(row0 + o + cpart * 2 + cbytes / 8 - 1, dc.psi_n, dc.flag);  // last element
        ff_cp16(dst0 + x * kFfRowBytes, ok ? (const void*)(rowb + o * 8) : (const void*)psi, ok ? cbytes : 0);
      }
    } else {
      double* sd = reinterpret_cast<double*>(st);
      for (int x = 0; x < C; x++) {
        const long long o = xoff[x];
        sd[x * 32 + lane] = (o >= 0 && bok && dc_ok<CHK>(row0 + o + lane, dc.psi_n, dc.flag)) ? row[o + lane] : 0.0;
      }
    }
  };

#pragma unroll
  for (int r = 0; r < kFfStages - 1; r++) {
    issue_next();
    ff_commit();
  }
  float t2s[P], t2c[P];  // y-pass accumulators of the current plane, float pairs
#pragma unroll
  for (int p = 0; p < P; p++) t2s[p] = t2c[p] = 0.0f;
  bool range_bad = false;  // a psi value the float pairs cannot carry (reported through the status word)

  for (int r = 0, iz = iz0, iy = 0; r < R; r++) {
    ff_wait<kFfStages - 2>();
    __syncwarp();
    issue_next();  // row r + kFfStages - 1
    ff_commit();
    // spherical support of the row: the points inside are the contiguous run [xlo, xhi) of the cube row
    int xlo = 0, xhi = 0;
    if (zidx[iz] >= 0 && yidx[iy] >= 0) support_run(row_support(g, at, iy, iz, lane), xlo, xhi);
    if (xhi > xlo) {
      const double* st = reinterpret_cast<const double*>(ring + (size_t)(r % kFfStages) * C * kFfRowBytes);
      // x-pass (a3) as float-float dot products
      float S[NP], E[NP];
#pragma unroll
      for (int n = 0; n < NP; n++) S[n] = E[n] = 0.0f;
      auto xpass = [&](int x0, int x1) {
#pragma unroll 4
        for (int ix = x0; ix < x1; ix++) {
          const double pd = st[ix * 32 + lane];
          range_bad |= ff_out_of_range(pd);
          const ff pv = ff_from_double(pd);
          const float4* f4 = reinterpret_cast<const float4*>(phx + (size_t)ix * NPX);
#pragma unroll
          for (int q = 0; q < NPX / 2; q++) {
            const float4 f = f4[q];
            if (2 * q < NP) ff_dot_step(S[2 * q], E[2 * q], pv, ff{f.x, f.y});
            if (2 * q + 1 < NP) ff_dot_step(S[2 * q + 1], E[2 * q + 1], pv, ff{f.z, f.w});
          }
        }
      };
      ff t1[NP];
      if constexpr (BLOCH) {
        // points before the crossing w, the sum turned by ph(before) / ph(after), the points after it, and
        // the row's sum turned by the phase of the last run (y and z bits of this row and plane)
        const BlochPh& bp = bph[a];
        const int wx = bp.w[0];
        xpass(xlo, min(xhi, wx));
        const float4 xst = bp.xstep;
        if (wx > xlo && wx < xhi && !ff_is_one(xst)) {
#pragma unroll
          for (int n = 0; n < NP; n++) {
            const ff v = ff_rotate(ff_norm(S[n], E[n]), xst, lane);
            S[n] = v.hi;
            E[n] = v.lo;
          }
        }
        xpass(max(xlo, wx), xhi);
        const float4 ph = bp.ph[(xhi > wx ? 1 : 0) + (iy >= bp.w[1] ? 2 : 0) + (iz >= bp.w[2] ? 4 : 0)];
        const bool one = ff_is_one(ph);
#pragma unroll
        for (int n = 0; n < NP; n++) {
          t1[n] = ff_norm(S[n], E[n]);
          if (!one) t1[n] = ff_rotate(t1[n], ph, lane);
        }
      } else {
        xpass(xlo, xhi);
#pragma unroll
        for (int n = 0; n < NP; n++) t1[n] = ff_norm(S[n], E[n]);
      }
      // y-pass (a4) as float-float dot steps
#pragma unroll
      for (int ny = 0; ny < NP; ny++) {
        const float2 w = phy[ny * C + iy];
#pragma unroll
        for (int nx = 0; nx + ny <= NU; nx++)
          ff_dot_step(t2s[BS::pair(nx, ny)], t2c[BS::pair(nx, ny)], t1[nx], ff{w.x, w.y});
      }
    }
    __syncwarp();
    if (iy == C - 1) {
      // the finished plane's T2 (zero for a plane outside an open grid), in FP64, for the z-pass
      if (bok) {
        const long long o0 = ((long long)a * C + iz) * P * B + b0 + lane;
        double* out = t2g + o0;
#pragma unroll
        for (int p = 0; p < P; p++)
          if (dc_ok<CHK>(o0 + (long long)p * B, dc.t2_n, dc.flag)) out[(size_t)p * B] = ff_to_double(t2s[p], t2c[p]);
      }
#pragma unroll
      for (int p = 0; p < P; p++) t2s[p] = t2c[p] = 0.0f;
    }
    if (++iy == C) {
      iy = 0;
      iz++;
    }
  }
  ff_wait<0>();
  if (__any_sync(0xffffffffu, range_bad) && lane == 0 && status) atomicOr(status, kStatusRange);
}

// z-pass (a5) of the FP64-accurate projection in FP64, one warp per (atom, 32-band tile):
// c[a][(nx,ny,nz)][b] = h^3 sum_iz phi_nz(z_iz) T2[a][iz][(nx,ny)][b], planes in ascending order.
template <int NU>
struct FfZpassSmem {
  static constexpr int NP = NU + 1, P = Basis<NU>::P, N = Basis<NU>::N;
  static constexpr bool ACCR = N <= 56;  // accumulators and the plane's T2 in registers up to numax 5
  static size_t bytes(int cube) {
    return (size_t)NP * cube * sizeof(double) + (ACCR ? 0 : (size_t)(N + P) * kWarp * sizeof(double));
  }
};

template <int NU>
__global__ void __launch_bounds__(kWarp) k_project_ff_zpass(GridDev g, const AtomDev* __restrict__ atoms,
                                                            const double* __restrict__ t2g,
                                                            double* __restrict__ coeff) {
  using BS = Basis<NU>;
  using SM = FfZpassSmem<NU>;
  constexpr int NP = BS::NP, P = BS::P, N = BS::N;
  constexpr bool ACCR = SM::ACCR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int C = g.cube, B = g.nbands;
  double* phz = reinterpret_cast<double*>(smem_raw);  // [NP][C]
  double* acc = phz + (size_t)NP * C;                 // [N][32] when not in registers
  double* t2p = acc + (size_t)N * kWarp;              // [P][32] the plane's T2, same case
  const int lane = threadIdx.x;
  const int a = blockIdx.y;
  const int b = blockIdx.x * kWarp + lane;
  const bool bok = b < B;
  const AtomDev at = atoms[a];
  for (int i = lane; i < C; i += kWarp) phi_column(cube_offset(at.o[2], i, g.h, at.X[2]), at.sigma, NU, phz + i, C);
  __syncwarp();
  if (!bok) return;
  const double* src = t2g + (size_t)a * C * P * B + b;
  double accr[ACCR ? N : 1];
  if constexpr (ACCR) {
    // grid z splits the states between two warps by nz: nz in half ((nz + 1) / 2) % 2 (numax 5: 30 and
    // 26 states), each warp over all planes in order (the same sums, twice the warps)
    auto run = [&](auto hz) {
      constexpr int HZ = decltype(hz)::value;
      auto own = [](int nz) { return (((nz + 1) >> 1) & 1) == HZ; };
      double acch[N];
#pragma unroll
      for (int k = 0; k < N; k++) acch[k] = 0.0;
      for (int iz = 0; iz < C; iz++) {
        double t2[P];
#pragma unroll
        for (int p = 0; p < P; p++) t2[p] = src[((size_t)iz * P + p) * B];
        int k = 0;
#pragma unroll
        for (int nz = 0; nz < NP; nz++) {
          const double w = phz[nz * C + iz];
#pragma unroll
          for (int ny = 0; ny + nz <= NU; ny++)
#pragma unroll
            for (int nx = 0; nx + ny + nz <= NU; nx++) {
              if (own(nz)) acch[k] = fma(t2[BS::pair(nx, ny)], w, acch[k]);
              k++;
            }
        }
      }
      const double h3 = g.h * g.h * g.h;
      double* out = coeff + (size_t)a * N * B + b;
      int k = 0;
#pragma unroll
      for (int nz = 0; nz < NP; nz++)
#pragma unroll
        for (int ny = 0; ny + nz <= NU; ny++)
#pragma unroll
          for (int nx = 0; nx + ny + nz <= NU; nx++) {
            if (own(nz)) out[(size_t)k * B] = acch[k] * h3;
            k++;
          }
    };
    if (blockIdx.z == 0)
      run(std::integral_constant<int, 0>{});
    else
      run(std::integral_constant<int, 1>{});
    return;
  } else {
    // larger bases: accumulators and the plane's T2 in this lane's columns of shared memory, loops kept
    // rolled (states in the order nz, ny, nx, so k counts up)
    for (int k = 0; k < N; k++) acc[k * kWarp + lane] = 0.0;
#pragma unroll 1
    for (int iz = 0; iz < C; iz++) {
      for (int p = 0; p < P; p++) t2p[p * kWarp + lane] = src[((size_t)iz * P + p) * B];
      int k = 0;
#pragma unroll 1
      for (int nz = 0; nz < NP; nz++) {
        const double w = phz[nz * C + iz];
#pragma unroll 1
        for (int ny = 0; ny + nz <= NU; ny++) {
          const int p0 = BS::pair(0, ny);
#pragma unroll 1
          for (int nx = 0; nx + ny + nz <= NU; nx++, k++)
            acc[k * kWarp + lane] = fma(t2p[(p0 + nx) * kWarp + lane], w, acc[k * kWarp + lane]);
        }
      }
    }
  }
  const double h3 = g.h * g.h * g.h;
  double* out = coeff + (size_t)a * N * B + b;
  for (int k = 0; k < N; k++) out[(size_t)k * B] = (ACCR ? accr[k] : acc[k * kWarp + lane]) * h3;
}

// ------------------------------------------------------------------------------- expansion, block gather
// Tiles of 8 grid rows x 32 x points x 32 bands of one z plane (8 warps, one per row).  For each atom
// whose cube meets the tile, its z-pass slice T2[a][z][P][32] (FP64), its x table as float pairs
// [C][NPX] and its y table [NP][C] (FP64) are staged once in shared memory, two atoms ahead in three
// buffers, and shared by the 8 row-warps.  Each warp keeps the update of its 32 x points as float pairs
// in registers and adds it to psi in FP64 at the end.  Atoms in ascending order; deterministic.
constexpr int kFfRows = 8;
constexpr int kFfXSeg = 32;

template <int NU>
struct FfBlkSmem {
  static constexpr int NP = NU + 1, P = Basis<NU>::P, NPX = (NP + 1) & ~1;
  // bytes of one staging buffer: T2 [P][32] pairs + x pairs [C][NPX] + y pairs [NP][C]
  __host__ __device__ static size_t buf_bytes(int cube) {
    return (size_t)P * 32 * 8 + (size_t)cube * NPX * 8 + (size_t)NP * cube * 8;
  }
  // 3 staging buffers + per-warp update accumulators [8 warps][32 x][32 bands] float pairs + atom list
  static size_t bytes(int cube, int max_plane) {
    return 3 * buf_bytes(cube) + (size_t)kFfRows * kFfXSeg * kWarp * 8 + (size_t)(max_plane + 1) * sizeof(int4);
  }
};

// CHK: device checks of every psi and z-pass-result index (sho_set_device_checks), a separate instantiation.
// BLOCH: complex coefficients and psi of a Bloch wave (Sec. 2.5), (re, im) pairs as two real bands in
// neighbouring lanes; the y-pass result of each (atom, row) turns by the phase of the translation of the
// tile points it updates (one per run of the tile row), so that the z-, y- and x-passes stay real.
template <int NU, bool CHK = false, bool BLOCH = false>
__global__ void __launch_bounds__(kFfRows * kWarp) k_expand_blk_ff(GridDev g, const AtomDev* __restrict__ atoms,
                                                                   const int* __restrict__ plane_ptr,
                                                                   const int* __restrict__ plane_atoms,
                                                                   const float2* __restrict__ tyff,
                                                                   const float2* __restrict__ txff,
                                                                   const float2* __restrict__ t2,
                                                                   double* __restrict__ psi, DevCheck dc,
                                                                   const BlochPh* __restrict__ bph) {
  using BS = Basis<NU>;
  using SM = FfBlkSmem<NU>;
  constexpr int NP = BS::NP, P = BS::P, NPX = SM::NPX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int C = g.cube;
  const int Nx = g.n[0], Ny = g.n[1], Nz = g.n[2];
  const size_t bufb = SM::buf_bytes(C);
  float2* accs = reinterpret_cast<float2*>(smem_raw + 3 * bufb);  // [warps][32 x][32 bands]
  int4* slist = reinterpret_cast<int4*>(accs + kFfRows * kFfXSeg * kWarp);  // (atom, offsets), ascending
  __shared__ int wcount[kFfRows];
  __shared__ int s_nlist;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nseg = (Nx + kFfXSeg - 1) / kFfXSeg, nyb = (Ny + kFfRows - 1) / kFfRows;
  int bid = blockIdx.x;
  const int seg = bid % nseg;
  bid /= nseg;
  const int yb = bid % nyb;
  const int z = bid / nyb;
  const int xs = seg * kFfXSeg;
  const int y = yb * kFfRows + warp;
  const bool yok = y < Ny;
  const int B = g.nbands;
  const int b0 = blockIdx.y * kWarp;
  const bool bok = b0 + lane < B;
  const int q0 = plane_ptr[z], q1 = plane_ptr[z + 1];
  // the tile's psi (this warp's row, this lane's x point, the band tile's 256 bytes) to L2 for the final
  // read-modify-write
  if (yok && xs + lane < Nx) {
    const double* pp = psi + (((size_t)z * Ny + y) * Nx + xs + lane) * (size_t)B + b0;
    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(pp));
    if (B - b0 > 16) asm volatile("prefetch.global.L2 [%0];\n" ::"l"(pp + 16));
  }
  // Offsets of atom a's cube against this tile, wrapped into [0, N) on a periodic grid: r.y = cube
  // row of the tile's first row, r.z = cube point of its first x point, r.w = cube plane of z.  True
  // when the cube meets the tile's rows and x segment.  Computed once per (tile, atom) here, so the
  // atom loop below does no integer division.
  auto locate = [&](const AtomDev& at, int4& r) {
    int dy = yb * kFfRows - at.o[1], dx = xs - at.o[0], dz = z - at.o[2];
    bool m;
    if (g.periodic) {
      dy %= Ny;
      if (dy < 0) dy += Ny;
      dx %= Nx;
      if (dx < 0) dx += Nx;
      dz %= Nz;
      if (dz < 0) dz += Nz;
      m = (dy < C || dy + kFfRows > Ny) && (dx < C || dx + kFfXSeg > Nx);
    } else {
      m = dy < C && dy + kFfRows > 0 && dx < C && dx + kFfXSeg > 0;
    }
    r = make_int4(0, dy, dx, dz);
    return m;
  };

  // staging with 8-byte asynchronous copies (FP64 rows of an arbitrary band count are 8-byte aligned)
  auto cp8 = [](void* dst, const void* src, int bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(ff_smem_u32(dst)), "l"(src), "r"(bytes));
  };
  auto stage = [&](const int4 r, int buf) {
    const int a = r.x, iz = r.w;
    unsigned char* dst = smem_raw + (size_t)buf * bufb;
    float2* dt2 = reinterpret_cast<float2*>(dst);
    const long long s0 = ((long long)a * C + iz) * P * B + b0;
    const float2* src_t2 = t2 + s0;
    for (int q = tid; q < P * 32; q += kFfRows * kWarp) {
      const int p = q >> 5, bl = q & 31;
      const bool ok = b0 + bl < B && dc_ok<CHK>(s0 + (long long)p * B + bl, dc.t2_n, dc.flag);
      cp8(dt2 + q, ok ? (const void*)(src_t2 + (size_t)p * B + bl) : (const void*)t2, ok ? 8 : 0);
    }
    float2* dx = reinterpret_cast<float2*>(dst + (size_t)P * 32 * 8);
    const float2* src_x = txff + (size_t)a * C * NPX;
    for (int q = tid; q < C * NPX; q += kFfRows * kWarp) cp8(dx + q, src_x + q, 8);
    float2* dy = reinterpret_cast<float2*>(dst + (size_t)P * 32 * 8 + (size_t)C * NPX * 8);
    const float2* src_y = tyff + (size_t)a * NP * C;
    for (int q = tid; q < NP * C; q += kFfRows * kWarp) cp8(dy + q, src_y + q, 8);
  };

  // the plane's atoms that meet the tile, compacted in ascending order
  if (tid == 0) s_nlist = 0;
  __syncthreads();
  for (int base = q0; base < q1; base += kFfRows * kWarp) {
    const int q = base + tid;
    int4 r = make_int4(-1, 0, 0, 0);
    bool m = false;
    if (q < q1) {
      const int a = plane_atoms[q];
      m = locate(atoms[a], r);
      r.x = a;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, m);
    if (lane == 0) wcount[warp] = __popc(bal);
    __syncthreads();
    int off = s_nlist;
    for (int w = 0; w < warp; w++) off += wcount[w];
    if (m) slist[off + __popc(bal & ((1u << lane) - 1u))] = r;
    __syncthreads();
    if (tid == 0)
      for (int w = 0; w < kFfRows; w++) s_nlist += wcount[w];
    __syncthreads();
  }
  const int nlist = s_nlist;

  float2* accw = accs + warp * kFfXSeg * kWarp;  // this row's update of the 32 x points, float pairs
#pragma unroll
  for (int x = 0; x < kFfXSeg; x++) accw[x * kWarp + lane] = make_float2(0.0f, 0.0f);
  const int xend = min(kFfXSeg, Nx - xs);       // tile points that exist on the grid

  // three staging buffers, atoms staged two ahead: the one barrier per atom also shows that every warp
  // is done with atom li - 1, whose buffer is refilled with atom li + 2
  if (nlist > 0) stage(slist[0], 0);
  ff_commit();
  if (nlist > 1) stage(slist[1], 1);
  ff_commit();
  for (int li = 0, buf = 0; li < nlist; li++, buf = buf == 2 ? 0 : buf + 1) {
    const int4 r = slist[li];
    ff_wait<1>();  // this thread's copies of atom li have landed
    __syncthreads();
    if (li + 2 < nlist) stage(slist[li + 2], buf == 0 ? 2 : buf - 1);
    ff_commit();
    const unsigned char* src = smem_raw + (size_t)buf * bufb;
    const float2* t2s = reinterpret_cast<const float2*>(src);
    const float2* txs = reinterpret_cast<const float2*>(src + (size_t)P * 32 * 8);
    const float2* tys = reinterpret_cast<const float2*>(src + (size_t)P * 32 * 8 + (size_t)C * NPX * 8);
    int iy = r.y + warp;  // cube row of this warp's grid row
    if (g.periodic && iy >= Ny) iy -= Ny;
    const bool rowin = yok && iy >= 0 && iy < C;
    // spherical support of the row in cube x coordinates, [slo, shi) (the whole row without a sphere)
    int slo = 0, shi = C;
    if (g.r2max > 0.0) support_run(row_support(g, atoms[r.x], rowin ? iy : 0, r.w, lane), slo, shi);
    if (rowin && shi > slo) {
      // y-pass as float-float dot steps
      float ys[NP], yc[NP];
#pragma unroll
      for (int n = 0; n < NP; n++) ys[n] = yc[n] = 0.0f;
#pragma unroll
      for (int ny = 0; ny < NP; ny++) {
        const float2 w = tys[ny * C + iy];
#pragma unroll
        for (int nx = 0; nx + ny <= NU; nx++) {
          const float2 v = t2s[BS::pair(nx, ny) * 32 + lane];
          ff_dot_step(ys[nx], yc[nx], ff{v.x, v.y}, ff{w.x, w.y});
        }
      }
      ff t1f[NP];
#pragma unroll
      for (int n = 0; n < NP; n++) t1f[n] = ff_norm(ys[n], yc[n]);
      const int dx = r.z;  // cube index of tile point x is dx + x (mod Nx when periodic)
      // x-pass as float-float dot products over the tile points inside the cube: one contiguous run
      // of x (two when the cube wraps around a periodic grid)
      int r0a, r0b, r1a, r1b;
      if (g.periodic) {
        r0a = 0;
        r0b = dx < C ? min(xend, C - dx) : 0;           // ix = dx + x
        r1a = Nx - dx;                                  // ix = dx + x - Nx
        r1b = min(xend, Nx - dx + C);
      } else {
        r0a = max(0, -dx);
        r0b = min(xend, C - dx);
        r1a = r1b = 0;
      }
      for (int run = 0; run < 2; run++) {
        const int shift = run ? dx - Nx : dx;
        // tile points of this run whose cube index ix = x + shift lies in the row's support
        const int xa = max(run ? max(r1a, r0b) : r0a, slo - shift), xb = min(run ? r1b : r0b, shi - shift);
        ff t1r[NP];
#pragma unroll
        for (int n = 0; n < NP; n++) t1r[n] = t1f[n];
        if constexpr (BLOCH) {
          // the run's points share one translation: its phase from the bits of cube point xa + shift,
          // cube row iy and cube plane r.w
          if (xa < xb) {
            const BlochPh& bp = bph[r.x];
            const float4 ph = bp.ph[(xa + shift >= bp.w[0] ? 1 : 0) + (iy >= bp.w[1] ? 2 : 0) + (r.w >= bp.w[2] ? 4 : 0)];
            if (!ff_is_one(ph)) {
#pragma unroll
              for (int n = 0; n < NP; n++) t1r[n] = ff_rotate(t1f[n], ph, lane);
            }
          }
        }
#pragma unroll 2
        for (int x = xa; x < xb; x++) {
          const int ix = x + shift;
          // the point's dot product over all atoms and states continues from its running (s, c)
          float2 v = accw[x * kWarp + lane];
          const float4* f4 = reinterpret_cast<const float4*>(txs + ix * NPX);
#pragma unroll
          for (int qn = 0; qn < NPX / 2; qn++) {
            const float4 f = f4[qn];
            if (2 * qn < NP) ff_dot_step(v.x, v.y, t1r[2 * qn], ff{f.x, f.y});
            if (2 * qn + 1 < NP) ff_dot_step(v.x, v.y, t1r[2 * qn + 1], ff{f.z, f.w});
          }
          accw[x * kWarp + lane] = v;
        }
      }
    }
  }
  ff_wait<0>();
  if (!yok || !bok || nlist == 0) return;
  const long long row0 = ((long long)z * Ny + y) * Nx * B + b0 + lane;  // psi index of the row's x = 0
  double* rowp = psi + row0;
  // loads of 16 points first, so that they are in flight together, then their adds and stores
#pragma unroll
  for (int x0 = 0; x0 < kFfXSeg; x0 += 16) {
    double pv[16];
    bool in[16];
#pragma unroll
    for (int i = 0; i < 16; i++) {
      in[i] = x0 + i < xend && dc_ok<CHK>(row0 + (long long)(xs + x0 + i) * B, dc.psi_n, dc.flag);
      pv[i] = in[i] ? rowp[(size_t)(xs + x0 + i) * B] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < 16; i++) {
      if (in[i]) {
        const float2 v = accw[(x0 + i) * kWarp + lane];
        rowp[(size_t)(xs + x0 + i) * B] = pv[i] + ff_to_double(v.x, v.y);
      }
    }
  }
}

// ------------------------------------------------------------------------------- launchers
template <int NU>
static cudaError_t ff_project_nu(const ProjectLaunch& p) {
  if (!p.t2) return cudaErrorInvalidValue;
  const unsigned nbt = (unsigned)((p.g.nbands + kWarp - 1) / kWarp);
  cudaError_t e;
  if (p.kernel == 2 && !p.bloch && !p.chk.flag && ozaki_project_ok(p)) {
    // the x-pass on the tensor cores by exact digit slicing when chosen (kernel choice tcgen05): correct,
    // but measured about 20 % slower than the float-float kernel (its digit warps are the bound)
    e = launch_project_ozaki(p);
  } else {
    const size_t smem = FfProjectSmem<NU>::bytes(p.g.cube);
    auto kern = p.chk.flag ? k_project_ff<NU, true> : k_project_ff<NU, false>;
    if constexpr (NU <= kBlochRealMaxNumax) {
      if (p.bloch) kern = k_project_ff<NU, false, true>;
    } else if (p.bloch) {
      return cudaErrorInvalidValue;
    }
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3((unsigned)p.zsplit, nbt, (unsigned)p.natoms), kWarp, smem, p.stream>>>(
        p.g, static_cast<const double*>(p.psi), p.atoms, p.zsplit, static_cast<double*>(p.t2), p.status, p.chk,
        p.bloch);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess || p.t2_only) return e;
  const size_t zsmem = FfZpassSmem<NU>::bytes(p.g.cube);
  auto zk = k_project_ff_zpass<NU>;
  e = cudaFuncSetAttribute(zk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zsmem);
  if (e != cudaSuccess) return e;
  zk<<<dim3(nbt, (unsigned)p.natoms, FfZpassSmem<NU>::ACCR ? 2u : 1u), kWarp, zsmem, p.stream>>>(
      p.g, p.atoms, static_cast<const double*>(p.t2), static_cast<double*>(p.coeff));
  return cudaGetLastError();
}

template <int NU>
static cudaError_t ff_expand_nu(const ExpandLaunch& p) {
  constexpr int NPX = (NU + 2) & ~1;
  // y pairs go after the x pairs in the x-major region (sized for [A][C][4 * ceil(NP/4)] doubles); the
  // z-pass writes T2 and both tables as float pairs
  float2* txff = static_cast<float2*>(p.tables_xmajor);
  float2* tyff = txff + (size_t)p.natoms * p.g.cube * NPX;
  cudaError_t e = launch_expand_zpass_ff(p, txff, tyff);
  if (e != cudaSuccess) return e;
  // the x-pass on the tensor cores by exact digit slicing where it applies (kernel choice tcgen05; or
  // automatic when its 128-band tiles are at least three quarters full, since a tile costs the same
  // whatever its band count); the float-float block gather when chosen (kernel choice 1), under device
  // checks, and in the other cases
  const int obt = (p.g.nbands + 127) / 128;
  const bool full_tiles = 4 * p.g.nbands >= 3 * 128 * obt;
  if ((p.kernel == 2 || (p.kernel == 0 && full_tiles)) && !p.chk.flag && ozaki_expand_ok(p))
    return launch_expand_ozaki(p, tyff);
  auto kern = p.chk.flag ? k_expand_blk_ff<NU, true> : k_expand_blk_ff<NU, false>;
  if constexpr (NU <= kBlochRealMaxNumax) {
    if (p.bloch) kern = k_expand_blk_ff<NU, false, true>;
  } else if (p.bloch) {
    return cudaErrorInvalidValue;
  }
  const size_t smem = FfBlkSmem<NU>::bytes(p.g.cube, p.max_plane);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int nseg = (p.g.n[0] + kFfXSeg - 1) / kFfXSeg, nyb = (p.g.n[1] + kFfRows - 1) / kFfRows;
  kern<<<dim3((unsigned)nseg * nyb * p.g.n[2], (p.g.nbands + kWarp - 1) / kWarp), kFfRows * kWarp, smem, p.stream>>>(
      p.g, p.atoms, p.plane_ptr, p.plane_atoms, tyff, txff, static_cast<const float2*>(p.t2),
      static_cast<double*>(p.psi), p.chk, p.bloch);
  return cudaGetLastError();
}

cudaError_t launch_project_ff(const ProjectLaunch& p) {
  switch (p.numax) {
    case 0: return ff_project_nu<0>(p);
    case 1: return ff_project_nu<1>(p);
    case 2: return ff_project_nu<2>(p);
    case 3: return ff_project_nu<3>(p);
    case 4: return ff_project_nu<4>(p);
    case 5: return ff_project_nu<5>(p);
    case 6: return ff_project_nu<6>(p);
    case 7: return ff_project_nu<7>(p);
    case 8: return ff_project_nu<8>(p);
    case 9: return ff_project_nu<9>(p);
    case 10: return ff_project_nu<10>(p);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_expand_ff(const ExpandLaunch& p) {
  switch (p.numax) {
    case 0: return ff_expand_nu<0>(p);
    case 1: return ff_expand_nu<1>(p);
    case 2: return ff_expand_nu<2>(p);
    case 3: return ff_expand_nu<3>(p);
    case 4: return ff_expand_nu<4>(p);
    case 5: return ff_expand_nu<5>(p);
    case 6: return ff_expand_nu<6>(p);
    case 7: return ff_expand_nu<7>(p);
    case 8: return ff_expand_nu<8>(p);
    case 9: return ff_expand_nu<9>(p);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sho
