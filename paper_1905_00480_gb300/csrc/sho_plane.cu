// sho_plane.cu -- plane-sweep projection of the FP32-class forms (FP32 psi, numax <= 7).
//
// The per-atom kernels (sho_fp32.cu) stream every atom's cube on its own, so a psi element that lies in
// the cubes of k atoms is fetched k times (k ~ 4 in dense systems) and DRAM traffic is a multiple of
// the data.  Here one CTA owns one grid plane z and one tile of 32 bands and sweeps the plane's rows
// once: each row (all Nx points x 32 bands) is copied into shared memory by one TMA load and then
// serves every atom whose cube contains it.  The projection is split where the sweep needs it
// (eq. TuckerTensor, Sec. 3.4; Sec. 3.2 step 1):
//
//   k_plane_tables   per atom: the y table phi_ny(iy) and the x table, the latter also pre-arranged as
//                    tensor-core B fragments (FP64 recursion of Sec. 3.7, rounded once)
//   k_project_plane  per (plane z, band tile): x-pass and y-pass of every atom whose cube meets plane
//                    z, T2[a][iz][(nx,ny)][b] = sum_y phi_ny(y) sum_x phi_nx(x) psi[z][y][x][b]
//   k_plane_zpass    per (atom, band tile): c[k][b] = h^3 sum_iz phi_nz(iz) T2[a][iz][(nx,ny)][b]
//
// Inside k_project_plane, 11 consumer warps each carry 3 register slots of y-pass accumulators; the
// host assigns every (atom, plane) row segment to a (warp, slot) so that the segments of one slot do
// not overlap in y (interval colouring, plan_planes), so each row needs no dynamic indexing.  A 12th
// warp issues the TMA row loads into a ring of `stages` rows guarded by mbarriers (full: TMA bytes
// landed; empty: all consumer warps done with the row).  Every wait is bounded (a launch parameter,
// ~2 s by default): when it runs out the waiting warp records kStatusTimeout in the status word and
// leaves its loop; the producer then waits, again bounded, for the copies it issued before it returns.
//
// x-pass on the tensor cores: T1[b][n] = sum_x psi[x][b] phi_n(x) is an m16n8 (bands x states) product
// with K = x.  Row m of the two m-tiles maps to band 4g + 2j (+1 for m = g + 8), and for the TF32
// forms k maps to x = 8s + 2t (+1 for k = t + 4), so each lane reads its four bands at one x with one
// 16-byte shared load; with the 128-byte TMA swizzle these loads are free of bank conflicts.  The
// B fragments (phi) are stored in the same order by k_plane_tables.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>

#include "sho_tc.cuh"

namespace sho {

constexpr int kPlaneWarps = 11;                        // consumer warps per CTA (+ 1 producer: 384 threads, 168 registers)
constexpr int kPlaneSlots = 3;                         // y-pass accumulator slots per warp
constexpr int kPlaneThreads = (kPlaneWarps + 1) * 32;  // + the producer warp
constexpr int kPlaneMaxStages = 8;
constexpr int kT1Stride = 36;                          // padded row of the T1 transpose buffer
// Bytes of one x point of a row buffer: 32 bands of the storage type (SB bytes each).  FP32 rows are
// 128-byte swizzled (one swizzle row per point); BF16 rows (64 bytes) are not swizzled: their MMA A loads
// take x = base + t (+4, +8, +12) for lane quad t, so the quads alternate between the two bank halves.
template <int SB>
__host__ __device__ constexpr int plane_row_bytes() { return 32 * SB; }
constexpr int kSimtMode = -1;

// --------------------------------------------------------------------------------- mbarrier / TMA
__device__ __forceinline__ uint32_t pl_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0u;
}
// Wait for the phase of `parity` to complete; false after `limit` SM clock cycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
__device__ __forceinline__ void tma_load_row(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          dst),
      "l"(map), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}
__device__ __forceinline__ float4 lds128(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];\n" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
  return v;
}
__device__ __forceinline__ float lds32(uint32_t addr) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(v) : "r"(addr));
  return v;
}

// Byte offset of bands 4c..4c+3 of x point x in a 128-byte-swizzled row buffer.
__device__ __forceinline__ uint32_t swz(int x, int c) {
  return (uint32_t)x * 128u + ((uint32_t)(c ^ (x & 7)) << 4);
}
// Byte offset of bands 4c..4c+3 of x point x in a BF16 row buffer (64 bytes per point, no swizzle).
__device__ __forceinline__ uint32_t bfo(int x, int c) { return (uint32_t)x * 64u + ((uint32_t)c << 3); }
// Four BF16 values (8 bytes of shared memory) widened exactly to FP32.
__device__ __forceinline__ float4 lds_bf16x4(uint32_t addr) {
  uint32_t u0, u1;
  asm volatile("ld.shared.v2.u32 {%0,%1}, [%2];\n" : "=r"(u0), "=r"(u1) : "r"(addr));
  return make_float4(__uint_as_float(u0 << 16), __uint_as_float(u0 & 0xffff0000u), __uint_as_float(u1 << 16),
                     __uint_as_float(u1 & 0xffff0000u));
}
__device__ __forceinline__ float lds_bf16(uint32_t addr) {
  unsigned short v;
  asm volatile("ld.shared.u16 %0, [%1];\n" : "=h"(v) : "r"(addr));
  return __uint_as_float((uint32_t)v << 16);
}

// Grid x of cube point i for an atom whose first x is x0 (periodic: x0 in [0, Nx), one wrap at most;
// otherwise clamped into the grid -- the tables are zero for points outside it).
__device__ __forceinline__ int plane_x(int x0, int i, int nx, int periodic) {
  int x = x0 + i;
  if (periodic) return x >= nx ? x - nx : x;
  return x < 0 ? 0 : (x >= nx ? nx - 1 : x);
}

// --------------------------------------------------------------------------------- tables
// One warp per atom.  ytab[a][iy][8] and xtab[a][ix][8] (FP32, zero beyond numax and, when not
// periodic, at cube points outside the grid); bfrag[a][lane][s][4] B fragments of the x table.
template <int NU, int MODE, int SB>
__global__ void __launch_bounds__(kWarp) k_plane_tables(GridDev g, const AtomDev* __restrict__ atoms,
                                                        float* __restrict__ xtab, float* __restrict__ ytab,
                                                        uint32_t* __restrict__ bfrag) {
  constexpr int NP = NU + 1;
  __shared__ float xs[kMaxCube][8];
  const int a = blockIdx.x, lane = threadIdx.x, C = g.cube;
  const AtomDev at = atoms[a];
  for (int i = lane; i < C; i += kWarp) {
    double col[NP];
    phi_column(cube_offset(at.o[0], i, g.h, at.X[0]), at.sigma, NU, col, 1);
    const bool inside = cube_index(at.o[0], i, g.n[0], g.periodic) >= 0;
#pragma unroll
    for (int n = 0; n < 8; n++) {
      const float v = (n < NP && inside) ? (float)col[n] : 0.0f;
      xs[i][n] = v;
      xtab[((size_t)a * C + i) * 8 + n] = v;
    }
    phi_column(cube_offset(at.o[1], i, g.h, at.X[1]), at.sigma, NU, col, 1);
#pragma unroll
    for (int n = 0; n < 8; n++) ytab[((size_t)a * C + i) * 8 + n] = n < NP ? (float)col[n] : 0.0f;
  }
  __syncwarp();
  if constexpr (MODE != kSimtMode) {
    constexpr TcMode TM = (TcMode)MODE;
    constexpr int K = TcK<TM>::K;
    const int gq = lane >> 2, tq = lane & 3;
    uint32_t* out = bfrag + ((size_t)a * kWarp + lane) * (kMaxCube / 8) * 4;
    for (int s = 0; s * K < C; s++) {
      // k -> x of the A loads: FP32 rows x = 2t, 2t+1 (+8, +9); BF16 rows x = t, t+4 (+8, +12)
      float b[4];
      if constexpr (K == 8) {
        b[0] = xs[8 * s + (SB == 4 ? 2 * tq : tq)][gq];
        b[1] = xs[8 * s + (SB == 4 ? 2 * tq + 1 : tq + 4)][gq];
        b[2] = b[3] = 0.0f;
      } else {
        b[0] = xs[16 * s + (SB == 4 ? 2 * tq : tq)][gq];
        b[1] = xs[16 * s + (SB == 4 ? 2 * tq + 1 : tq + 4)][gq];
        b[2] = xs[16 * s + (SB == 4 ? 2 * tq + 8 : tq + 8)][gq];
        b[3] = xs[16 * s + (SB == 4 ? 2 * tq + 9 : tq + 12)][gq];
      }
      const BFrag<TM> f = make_bfrag<TM>(b);
      reinterpret_cast<uint4*>(out)[s] = make_uint4(f.hi[0], f.hi[1], f.lo[0], f.lo[1]);
    }
  }
}

// --------------------------------------------------------------------------------- plane sweep
// Bytes of one ring stage: a row of nx x points, rounded up to 1024 so that every stage starts on a
// 1024-byte boundary, which the 128-byte swizzle pattern of the TMA (and swz) is anchored to.
template <int SB>
__host__ __device__ __forceinline__ uint32_t plane_stage_bytes(int nx) {
  return ((uint32_t)nx * plane_row_bytes<SB>() + 1023u) & ~1023u;
}

// Per (warp, slot) shared area, filled when a segment starts: the atom's B fragments (tensor forms:
// [k-step][lane] with 2 words -- hi -- or 4 words -- hi, lo -- for the split forms; up to 4 k-steps for
// a 32-point cube) or its x table (CUDA-core form, [C][8]), then its y table [C][8].  The per-row work
// then reads shared memory only.
constexpr int kPlaneMaxCube = 32;
constexpr int kPlaneSmemBudget = 227 * 1024;

template <int MODE>
struct SlotLayout {
  static constexpr bool kSplit = MODE == (int)TcMode::X3TF32 || MODE == (int)TcMode::SPLIT16;
  static constexpr int kWords = kSplit ? 4 : 2;        // B-fragment words per (k-step, lane)
  static constexpr int kFrag = 4 * 32 * kWords * 4;    // 1 or 2 KB (the CUDA-core x table: 1 KB)
  static constexpr int kBytes = kFrag + 32 * 8 * 4;
};

template <int MODE, int SB>
struct PlaneSmem {
  // everything but the ring, including the alignment slack of the ring
  static constexpr size_t fixed() {
    return 1024 + 2 * kPlaneMaxStages * sizeof(unsigned long long)   // full / empty barriers
           + (size_t)kPlaneWarps * 8 * kT1Stride * sizeof(float)      // T1 transpose buffers
           + (size_t)kPlaneWarps * kPlaneSlots * SlotLayout<MODE>::kBytes  // slot tables
           + (size_t)kPlaneWarps * kPlaneSlots * 32;                  // slot records
  }
  static size_t bytes(int nx, int stages) { return fixed() + (size_t)stages * plane_stage_bytes<SB>(nx); }
};

template <int NU, int MODE, int SB>
__global__ void __launch_bounds__(kPlaneThreads, 1)
    k_project_plane(const __grid_constant__ CUtensorMap map, GridDev g, const int4* __restrict__ items,
                    const int* __restrict__ slot_ptr, const PlaneSeg* __restrict__ segs,
                    const uint32_t* __restrict__ bfrag, const float* __restrict__ xtab,
                    const float* __restrict__ ytab, int stages, int nbt, float* t2p, int* status,
                    long long wait_cycles, int stop_rows) {
  using BS = Basis<NU>;
  constexpr int NP = BS::NP, P = BS::P;
  constexpr int S = kPlaneSlots;
  constexpr bool TC = MODE != kSimtMode;
  constexpr TcMode TM = TC ? (TcMode)MODE : TcMode::TF32;
  constexpr int K = TcK<TM>::K;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = pl_smem(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const int Nx = g.n[0], Ny = g.n[1], C = g.cube, B = g.nbands;
  const uint32_t rowbytes = (uint32_t)Nx * plane_row_bytes<SB>();  // bytes one TMA row load delivers
  const uint32_t stagebytes = plane_stage_bytes<SB>(Nx);
  const uint32_t ring = base;
  const uint32_t bar_full = ring + (uint32_t)stages * stagebytes;
  const uint32_t bar_empty = bar_full + kPlaneMaxStages * 8;
  const uint32_t t1buf = bar_empty + kPlaneMaxStages * 8;
  using SL = SlotLayout<MODE>;
  const uint32_t slots = t1buf + kPlaneWarps * 8 * kT1Stride * 4;
  const uint32_t recs = slots + kPlaneWarps * S * SL::kBytes;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // band tiles of one plane run next to each other: they share DRAM pages and the plan entries
  const int item_id = (int)blockIdx.x / nbt, bt = (int)blockIdx.x - item_id * nbt;
  const int4 item = items[item_id];  // z, ylo, yhi, first slot-list index of the item
  const int z = item.x, ylo = item.y, R = item.z - item.y;
  const int b0 = bt * kWarp;

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; s++) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, kPlaneWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();

  if (warp == kPlaneWarps) {
    // ---------------------------------------------------------------- producer: TMA row loads
    if (lane == 0) {
      int issued = 0;
      bool ok = true;
      // stop_rows < R only under fault injection: the rows after it are never issued, so the consumers'
      // bounded waits for them expire
      const int Rp = min(R, stop_rows);
      for (int r = 0, st = 0, k = 0; r < Rp; r++) {  // st = r % stages, k = r / stages
        if (r > 0 && ++st == stages) {
          st = 0;
          k++;
        }
        if (!mbar_wait(bar_empty + 8 * st, (uint32_t)((k & 1) ^ 1), wait_cycles)) {
          ok = false;
          break;
        }
        mbar_expect_tx(bar_full + 8 * st, rowbytes);
        tma_load_row(ring + (uint32_t)st * stagebytes, &map, b0, (z * Ny + ylo + r) * Nx, bar_full + 8 * st);
        issued = r + 1;
      }
      if (!ok || Rp < R) {
        if (!ok) atomicOr(status, kStatusTimeout);
        // let the copies already issued land before the CTA's shared memory is released (they complete
        // whatever the consumers do, so this wait keeps the default limit)
        for (int r = max(0, issued - stages); r < issued; r++)
          (void)mbar_wait(bar_full + 8 * (r % stages), (uint32_t)((r / stages) & 1), kDefaultWaitCycles);
      }
    }
    return;
  }

  // ------------------------------------------------------------------ consumers
  const int gq = lane >> 2, tq = lane & 3;
  const int b = b0 + lane;
  const bool bok = b < B;
  const int list0 = item.w + warp * S;
  // per slot: rows [ys, ye) of the current segment in registers; the segment cursor and list end in
  // the slot record (words 4, 5), next to x0, iy - y, t2i and flags (words 0..3)
  int ys[S], ye[S];
#pragma unroll
  for (int s = 0; s < S; s++) {
    const int c0 = slot_ptr[list0 + s], c1 = slot_ptr[list0 + s + 1];
    ys[s] = c0 < c1 ? segs[c0].ys : 0x7fffffff;
    ye[s] = c0 < c1 ? segs[c0].ye : 0x7fffffff;
    if (lane == 0) {
      int* rec = reinterpret_cast<int*>(smem_raw + (recs - raw) + (warp * S + s) * 32);
      rec[4] = c0;
      rec[5] = c1;
    }
  }
  __syncwarp();
  float t2[S][P];
#pragma unroll
  for (int s = 0; s < S; s++)
#pragma unroll
    for (int p = 0; p < P; p++) t2[s][p] = 0.0f;
  const uint32_t myt1 = t1buf + (uint32_t)warp * 8 * kT1Stride * 4;
  float* t1w = reinterpret_cast<float*>(smem_raw + (myt1 - raw));

  for (int r = 0, st = 0, k = 0; r < R; r++) {  // st = r % stages, k = r / stages
    if (r > 0 && ++st == stages) {
      st = 0;
      k++;
    }
    const int y = ylo + r;
    // the warp leaves together: a lane whose wait ran out takes the others with it, so no lane is left
    // behind at a warp barrier of the row
    if (!__all_sync(0xffffffffu, mbar_wait(bar_full + 8 * st, (uint32_t)(k & 1), wait_cycles))) {
      if (lane == 0) atomicOr(status, kStatusTimeout);
      break;
    }
    const uint32_t row = ring + (uint32_t)st * stagebytes;
#pragma unroll
    for (int s = 0; s < S; s++) {
      if (ys[s] <= y) {  // warp-uniform: the slot's current segment covers this row
        const uint32_t sa = slots + (uint32_t)(warp * S + s) * SL::kBytes;  // tables of this slot
        const uint32_t ra = recs + (uint32_t)(warp * S + s) * 32;           // slot record
        int* rec = reinterpret_cast<int*>(smem_raw + (ra - raw));
        if (y == ys[s]) {
          // segment start: stage the atom's tables, record its offsets, load or clear the sums
          const PlaneSeg sg = segs[rec[4]];
          if constexpr (TC) {
            const uint4* src = reinterpret_cast<const uint4*>(bfrag + ((size_t)sg.atom * kWarp + lane) * (kMaxCube / 8) * 4);
            for (int ks = 0; ks * K < C; ks++) {
              const uint4 w = __ldg(src + ks);
              if constexpr (SL::kSplit)
                asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};\n" ::"r"(sa + (uint32_t)(ks * 32 + lane) * 16),
                             "r"(w.x), "r"(w.y), "r"(w.z), "r"(w.w));
              else
                asm volatile("st.shared.v2.u32 [%0], {%1,%2};\n" ::"r"(sa + (uint32_t)(ks * 32 + lane) * 8), "r"(w.x),
                             "r"(w.y));
            }
          } else if (lane < C) {
            const float4* src = reinterpret_cast<const float4*>(xtab + ((size_t)sg.atom * C + lane) * 8);
            const float4 f0 = __ldg(src), f1 = __ldg(src + 1);
            float4* dst = reinterpret_cast<float4*>(smem_raw + (sa - raw) + lane * 32);
            dst[0] = f0;
            dst[1] = f1;
          }
          if (lane < C) {
            const float4* src = reinterpret_cast<const float4*>(ytab + ((size_t)sg.atom * C + lane) * 8);
            const float4 f0 = __ldg(src), f1 = __ldg(src + 1);
            float4* dst = reinterpret_cast<float4*>(smem_raw + (sa - raw) + SL::kFrag + lane * 32);
            dst[0] = f0;
            dst[1] = f1;
          }
          if (lane == 0) {
            // bit 2 of the flags: the cube's x points are one contiguous run of the row (no wrap, no clip)
            const bool lin = sg.x0 >= 0 && sg.x0 + C <= Nx;
            *reinterpret_cast<int4*>(smem_raw + (ra - raw)) =
                make_int4(sg.x0, sg.iy0 - sg.ys, sg.t2i, sg.flags | (lin ? 4 : 0));
          }
          const size_t t2off = (size_t)sg.t2i * P * B + b;
#pragma unroll
          for (int p = 0; p < P; p++) t2[s][p] = (sg.flags == 2 && bok) ? t2p[t2off + (size_t)p * B] : 0.0f;
          __syncwarp();
        }
        const int4 rc = *reinterpret_cast<const int4*>(smem_raw + (ra - raw));
        const int x0 = rc.x, iy = y + rc.y;
        // ---- x-pass (a3): t1[n] for this lane's band
        float t1[NP];
        if constexpr (!TC) {
#pragma unroll
          for (int n = 0; n < NP; n++) t1[n] = 0.0f;
          for (int i = 0; i < C; i++) {
            const int x = plane_x(x0, i, Nx, g.periodic);
            const float v = SB == 4 ? lds32(row + swz(x, lane >> 2) + (uint32_t)(lane & 3) * 4)
                                    : lds_bf16(row + (uint32_t)x * 64u + (uint32_t)lane * 2u);
            const float4 f0 = lds128(sa + (uint32_t)i * 32), f1 = lds128(sa + (uint32_t)i * 32 + 16);
            const float f[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
#pragma unroll
            for (int n = 0; n < NP; n++) t1[n] = fmaf(v, f[n], t1[n]);
          }
        } else {
          float d[2][4], dl[2][4];
#pragma unroll
          for (int m = 0; m < 2; m++)
#pragma unroll
            for (int j = 0; j < 4; j++) d[m][j] = dl[m][j] = 0.0f;
          const bool lin = (rc.w & 4) != 0;
          // contiguous cube: x advances by 8 per TF32 k-step (1024 bytes, same swizzle phase), so the
          // A loads are fixed offsets from two per-lane base addresses
          const uint32_t pa = SB == 4 ? row + swz(x0 + 2 * tq, gq) : row + bfo(x0 + tq, gq);
          const uint32_t pb = SB == 4 ? row + swz(x0 + 2 * tq + 1, gq) : row + bfo(x0 + tq + 4, gq);
#pragma unroll 2
          for (int ks = 0; ks < kPlaneMaxCube / K; ks++) {
            if (ks * K < C) {
              uint4 bw = make_uint4(0u, 0u, 0u, 0u);
              if constexpr (SL::kSplit)
                asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];\n"
                             : "=r"(bw.x), "=r"(bw.y), "=r"(bw.z), "=r"(bw.w)
                             : "r"(sa + (uint32_t)(ks * 32 + lane) * 16));
              else
                asm volatile("ld.shared.v2.u32 {%0,%1}, [%2];\n"
                             : "=r"(bw.x), "=r"(bw.y)
                             : "r"(sa + (uint32_t)(ks * 32 + lane) * 8));
              BFrag<TM> bfr;
              bfr.hi[0] = bw.x;
              bfr.hi[1] = bw.y;
              bfr.lo[0] = bw.z;
              bfr.lo[1] = bw.w;
              if constexpr (K == 8) {
                float4 va, vb;
                if constexpr (SB == 4) {
                  if (lin) {
                    va = lds128(pa + ks * 1024);
                    vb = lds128(pb + ks * 1024);
                  } else {
                    const int xa = plane_x(x0, 8 * ks + 2 * tq, Nx, g.periodic);
                    const int xb = plane_x(x0, 8 * ks + 2 * tq + 1, Nx, g.periodic);
                    va = lds128(row + swz(xa, gq));
                    vb = lds128(row + swz(xb, gq));
                  }
                } else {
                  if (lin) {
                    va = lds_bf16x4(pa + ks * 512);
                    vb = lds_bf16x4(pb + ks * 512);
                  } else {
                    va = lds_bf16x4(row + bfo(plane_x(x0, 8 * ks + tq, Nx, g.periodic), gq));
                    vb = lds_bf16x4(row + bfo(plane_x(x0, 8 * ks + tq + 4, Nx, g.periodic), gq));
                  }
                }
                const float a0[4] = {va.x, va.y, vb.x, vb.y};
                const float a1[4] = {va.z, va.w, vb.z, vb.w};
                tc_product<TM>(d[0], dl[0], a0, bfr);
                tc_product<TM>(d[1], dl[1], a1, bfr);
              } else {
                float4 v0, v1, v2, v3;
                if constexpr (SB == 4) {
                  if (lin) {
                    v0 = lds128(pa + ks * 2048);
                    v1 = lds128(pb + ks * 2048);
                    v2 = lds128(pa + ks * 2048 + 1024);
                    v3 = lds128(pb + ks * 2048 + 1024);
                  } else {
                    const int xq0 = plane_x(x0, 16 * ks + 2 * tq, Nx, g.periodic);
                    const int xq1 = plane_x(x0, 16 * ks + 2 * tq + 1, Nx, g.periodic);
                    const int xq2 = plane_x(x0, 16 * ks + 2 * tq + 8, Nx, g.periodic);
                    const int xq3 = plane_x(x0, 16 * ks + 2 * tq + 9, Nx, g.periodic);
                    v0 = lds128(row + swz(xq0, gq));
                    v1 = lds128(row + swz(xq1, gq));
                    v2 = lds128(row + swz(xq2, gq));
                    v3 = lds128(row + swz(xq3, gq));
                  }
                } else {
                  if (lin) {
                    v0 = lds_bf16x4(pa + ks * 1024);
                    v1 = lds_bf16x4(pb + ks * 1024);
                    v2 = lds_bf16x4(pa + ks * 1024 + 512);
                    v3 = lds_bf16x4(pb + ks * 1024 + 512);
                  } else {
                    v0 = lds_bf16x4(row + bfo(plane_x(x0, 16 * ks + tq, Nx, g.periodic), gq));
                    v1 = lds_bf16x4(row + bfo(plane_x(x0, 16 * ks + tq + 4, Nx, g.periodic), gq));
                    v2 = lds_bf16x4(row + bfo(plane_x(x0, 16 * ks + tq + 8, Nx, g.periodic), gq));
                    v3 = lds_bf16x4(row + bfo(plane_x(x0, 16 * ks + tq + 12, Nx, g.periodic), gq));
                  }
                }
                const float a0[8] = {v0.x, v1.x, v0.y, v1.y, v2.x, v3.x, v2.y, v3.y};
                const float a1[8] = {v0.z, v1.z, v0.w, v1.w, v2.z, v3.z, v2.w, v3.w};
                tc_product<TM>(d[0], dl[0], a0, bfr);
                tc_product<TM>(d[1], dl[1], a1, bfr);
              }
            }
          }
          // lane (g, t) holds T1 of bands 4g..4g+3 at n = 2t, 2t+1; transpose to one band per lane
          if constexpr (TM == TcMode::X3TF32 || TM == TcMode::SPLIT16) {
            const float ls = tc_lo_scale<TM>();
#pragma unroll
            for (int m = 0; m < 2; m++)
#pragma unroll
              for (int j = 0; j < 4; j++) d[m][j] = fmaf(ls, dl[m][j], d[m][j]);
          }
          const float4 w0 = make_float4(d[0][0], d[0][2], d[1][0], d[1][2]);
          const float4 w1 = make_float4(d[0][1], d[0][3], d[1][1], d[1][3]);
          *reinterpret_cast<float4*>(t1w + (2 * tq) * kT1Stride + 4 * gq) = w0;
          *reinterpret_cast<float4*>(t1w + (2 * tq + 1) * kT1Stride + 4 * gq) = w1;
          __syncwarp();
#pragma unroll
          for (int n = 0; n < NP; n++) t1[n] = t1w[n * kT1Stride + lane];
          __syncwarp();
        }
        // ---- y-pass (a4)
        const uint32_t ya = sa + SL::kFrag + (uint32_t)iy * 32;
        const float4 y0 = lds128(ya), y1 = lds128(ya + 16);
        const float wy[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
        for (int ny = 0; ny < NP; ny++)
#pragma unroll
          for (int nx = 0; nx + ny <= NU; nx++)
            t2[s][BS::pair(nx, ny)] = fmaf(t1[nx], wy[ny], t2[s][BS::pair(nx, ny)]);
        if (y == ye[s] - 1) {
          if (bok) {
            const size_t t2off = (size_t)rc.z * P * B + b;
#pragma unroll
            for (int p = 0; p < P; p++) t2p[t2off + (size_t)p * B] = t2[s][p];
          }
          const int c0 = rec[4] + 1, c1 = rec[5];
          ys[s] = c0 < c1 ? segs[c0].ys : 0x7fffffff;
          ye[s] = c0 < c1 ? segs[c0].ye : 0x7fffffff;
          __syncwarp();  // every lane has read the cursor; the slot's tables may be restaged next
          if (lane == 0) rec[4] = c0;
          __syncwarp();
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(bar_empty + 8 * st);
  }
}

// --------------------------------------------------------------------------------- z-pass
template <int NU>
__global__ void __launch_bounds__(kWarp) k_plane_zpass(GridDev g, const AtomDev* __restrict__ atoms,
                                                       const float* __restrict__ t2p, float* __restrict__ coeff) {
  using BS = Basis<NU>;
  constexpr int NP = BS::NP, P = BS::P, N = BS::N;
  __shared__ float zt[NP][kMaxCube];
  const int a = blockIdx.x, lane = threadIdx.x, C = g.cube, B = g.nbands;
  const int b = blockIdx.y * kWarp + lane;
  const AtomDev at = atoms[a];
  for (int i = lane; i < C; i += kWarp) phi_column(cube_offset(at.o[2], i, g.h, at.X[2]), at.sigma, NU, &zt[0][i], kMaxCube);
  __syncwarp();
  // rows of the cube inside the grid (not periodic); without any, no T2 was written for this atom
  bool yrows = true;
  if (!g.periodic) yrows = at.o[1] < g.n[1] && at.o[1] + C > 0;
  float acc[N];
#pragma unroll
  for (int k = 0; k < N; k++) acc[k] = 0.0f;
  if (yrows && b < B) {
    for (int iz = 0; iz < C; iz++) {
      if (cube_index(at.o[2], iz, g.n[2], g.periodic) < 0) continue;
      const float* src = t2p + ((size_t)a * C + iz) * P * B + b;
      float t2[P];
#pragma unroll
      for (int p = 0; p < P; p++) t2[p] = src[(size_t)p * B];
      int k = 0;
#pragma unroll
      for (int nz = 0; nz < NP; nz++) {
        const float w = zt[nz][iz];
#pragma unroll
        for (int ny = 0; ny + nz <= NU; ny++)
#pragma unroll
          for (int nx = 0; nx + ny + nz <= NU; nx++) {
            acc[k] = fmaf(t2[BS::pair(nx, ny)], w, acc[k]);
            k++;
          }
      }
    }
  }
  if (b < B) {
    const float h3 = (float)(g.h * g.h * g.h);
#pragma unroll
    for (int k = 0; k < N; k++) coeff[((size_t)a * N + k) * B + b] = acc[k] * h3;
  }
}

// --------------------------------------------------------------------------------- host side
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

template <int MODE, int SB>
int plane_stages(int nx) {
  const int budget = kPlaneSmemBudget - (int)PlaneSmem<MODE, SB>::fixed();
  return std::min(kPlaneMaxStages, std::max(2, budget / (int)plane_stage_bytes<SB>(nx)));
}

template <int NU, int MODE, int SB>
cudaError_t plane_run(const PlaneLaunch& p) {
  const int A = p.natoms, nbt = (p.g.nbands + kWarp - 1) / kWarp;
  k_plane_tables<NU, MODE, SB><<<A, kWarp, 0, p.stream>>>(p.g, p.atoms, p.xtab, p.ytab, p.bfrag);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)p.g.nbands, (cuuint64_t)p.g.n[0] * p.g.n[1] * p.g.n[2]};
  const cuuint64_t strides[1] = {(cuuint64_t)p.g.nbands * SB};
  const cuuint32_t box[2] = {32u, (cuuint32_t)p.g.n[0]};
  const cuuint32_t estr[2] = {1u, 1u};
  auto enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  if (enc(&map, SB == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
          const_cast<void*>(p.psi), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          SB == 4 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  if (p.nitems > 0) {
    const int stages = plane_stages<MODE, SB>(p.g.n[0]);
    const size_t smem = PlaneSmem<MODE, SB>::bytes(p.g.n[0], stages);
    auto kern = k_project_plane<NU, MODE, SB>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)p.nitems * nbt, kPlaneThreads, smem, p.stream>>>(map, p.g, p.items, p.slot_ptr, p.segs, p.bfrag,
                                                                      p.xtab, p.ytab, stages, nbt, p.t2p, p.status,
                                                                      p.wait_cycles, p.stop_rows);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (p.t2_only) return cudaSuccess;
  k_plane_zpass<NU><<<dim3(A, nbt), kWarp, 0, p.stream>>>(p.g, p.atoms, p.t2p, p.coeff);
  return cudaGetLastError();
}

template <int NU, int SB>
cudaError_t plane_mode_sb(const PlaneLaunch& p, sho_prec prec) {
  switch (prec) {
    case SHO_P_FP32: return plane_run<NU, kSimtMode, SB>(p);
    case SHO_P_TF32: return plane_run<NU, (int)TcMode::TF32, SB>(p);
    case SHO_P_3XTF32: return plane_run<NU, (int)TcMode::X3TF32, SB>(p);
    case SHO_P_BF16: return plane_run<NU, (int)TcMode::BF16, SB>(p);
    case SHO_P_SPLIT_FP16: return plane_run<NU, (int)TcMode::SPLIT16, SB>(p);
    default: return cudaErrorInvalidValue;
  }
}

template <int NU>
cudaError_t plane_mode(const PlaneLaunch& p, sho_prec prec) {
  return p.psi_dtype == SHO_BF16 ? plane_mode_sb<NU, 2>(p, prec) : plane_mode_sb<NU, 4>(p, prec);
}

}  // namespace

bool plane_ok(const sho_grid* grid, const void* psi, sho_dtype psi_dt, int nbands, int numax, int cube,
              sho_prec prec) {
  if ((psi_dt != SHO_F32 && psi_dt != SHO_BF16) || !fp32_stream_ok(psi, psi_dt, nbands)) return false;
  if (prec != SHO_P_FP32 && !is_tc(prec)) return false;
  if (numax > kTcMaxNumax || cube % 16 != 0 || cube > kPlaneMaxCube) return false;
  if (grid->n[0] > 256 || (long long)grid->n[0] * grid->n[1] * grid->n[2] >= (1ll << 31)) return false;
  if (grid->periodic && cube > grid->n[0]) return false;
  return encode_fn() != nullptr;
}

// Row segments of every (atom, plane) and their assignment to (warp, slot) registers, per plane and
// round.  Segments of one slot are disjoint in y; a wrapped atom (periodic) has a tail [0, e) and a
// head [s, Ny) in the same warp: the tail's partial T2 is written first and the head continues from
// it, so each T2[a][iz] is written once complete.  Segments that find no free slot go to another
// round (another CTA sweeping the same plane).
void plan_planes(const sho_grid* grid, const std::vector<AtomDev>& at, int cube, PlanePlan& plan) {
  const int nx = grid->n[0], ny = grid->n[1], nz = grid->n[2];
  const bool per = grid->periodic != 0;
  const int W = kPlaneWarps, S = kPlaneSlots;
  // A head segment starts ny - cube rows after its tail ended.  With at least kPlaneMaxStages rows in
  // between, the ring's barriers order the tail's T2 stores before the head's loads (the tail's warp
  // released the row buffer that the head's row later reused); otherwise both go to one warp, whose
  // program order suffices.
  const bool same_warp = ny - cube < kPlaneMaxStages;
  plan.items.clear();
  plan.slot_ptr.assign(1, 0);
  plan.segs.clear();
  std::vector<std::vector<PlaneSeg>> byz((size_t)nz);
  for (size_t a = 0; a < at.size(); a++) {
    const int oy = at[a].o[1], oz = at[a].o[2];
    int x0 = at[a].o[0];
    if (per) {
      x0 %= nx;
      if (x0 < 0) x0 += nx;
    }
    for (int iz = 0; iz < cube; iz++) {
      int z = oz + iz;
      if (per) {
        z %= nz;
        if (z < 0) z += nz;
      } else if (z < 0 || z >= nz) {
        continue;
      }
      PlaneSeg sg;
      sg.atom = (int)a;
      sg.iz = iz;
      sg.x0 = x0;
      sg.t2i = (int)a * cube + iz;
      if (!per) {
        const int s0 = std::max(oy, 0), e0 = std::min(oy + cube, ny);
        if (s0 >= e0) continue;
        sg.ys = s0;
        sg.ye = e0;
        sg.iy0 = s0 - oy;
        sg.flags = 0;
        byz[(size_t)z].push_back(sg);
      } else {
        int s0 = oy % ny;
        if (s0 < 0) s0 += ny;
        if (s0 + cube <= ny) {
          sg.ys = s0;
          sg.ye = s0 + cube;
          sg.iy0 = 0;
          sg.flags = 0;
          byz[(size_t)z].push_back(sg);
        } else {
          PlaneSeg tail = sg, head = sg;
          tail.ys = 0;
          tail.ye = s0 + cube - ny;
          tail.iy0 = ny - s0;
          tail.flags = 1;
          head.ys = s0;
          head.ye = ny;
          head.iy0 = 0;
          head.flags = 2;
          byz[(size_t)z].push_back(tail);
          byz[(size_t)z].push_back(head);
        }
      }
    }
  }
  std::vector<int> free_at((size_t)W * S), cum((size_t)W);
  std::vector<std::vector<PlaneSeg>> lists((size_t)W * S);
  for (int z = 0; z < nz; z++) {
    std::vector<PlaneSeg> pend = byz[(size_t)z];
    std::stable_sort(pend.begin(), pend.end(), [](const PlaneSeg& l, const PlaneSeg& r) {
      return l.ys != r.ys ? l.ys < r.ys : (l.flags != r.flags ? l.flags < r.flags : l.atom < r.atom);
    });
    while (!pend.empty()) {
      std::fill(free_at.begin(), free_at.end(), 0);
      std::fill(cum.begin(), cum.end(), 0);
      for (auto& l : lists) l.clear();
      std::vector<int> tail_slot(at.size(), -1);  // slot of an atom's tail in this round
      std::vector<char> defer(at.size(), 0);      // atom's wrapped pair moves to the next round
      std::vector<PlaneSeg> next;
      for (const PlaneSeg& sg : pend) {
        if (defer[(size_t)sg.atom]) {
          next.push_back(sg);
          continue;
        }
        // least busy warp at the segment's first row, then the least rows assigned so far: keeps the
        // warps' total work even, so none holds the row ring back for long
        int best = -1, best_load = 1 << 30, best_cum = 1 << 30;
        for (int w = 0; w < W; w++) {
          if (same_warp && sg.flags == 2 && tail_slot[(size_t)sg.atom] >= 0 && tail_slot[(size_t)sg.atom] / S != w)
            continue;
          int load = 0, freeslot = -1;
          for (int s = 0; s < S; s++) {
            if (free_at[(size_t)w * S + s] > sg.ys)
              load++;
            else if (freeslot < 0)
              freeslot = w * S + s;
          }
          if (freeslot >= 0 && (load < best_load || (load == best_load && cum[(size_t)w] < best_cum))) {
            best_load = load;
            best_cum = cum[(size_t)w];
            best = freeslot;
          }
        }
        if (best < 0) {
          if (sg.flags == 2 && tail_slot[(size_t)sg.atom] >= 0) {
            // undo the tail: both halves move on together
            auto& l = lists[(size_t)tail_slot[(size_t)sg.atom]];
            for (size_t i = 0; i < l.size(); i++)
              if (l[i].atom == sg.atom && l[i].flags == 1) {
                next.push_back(l[i]);
                l.erase(l.begin() + (long)i);
                break;
              }
          }
          if (sg.flags == 1) defer[(size_t)sg.atom] = 1;
          next.push_back(sg);
          continue;
        }
        lists[(size_t)best].push_back(sg);
        free_at[(size_t)best] = sg.ye;
        cum[(size_t)(best / S)] += sg.ye - sg.ys;
        if (sg.flags == 1) tail_slot[(size_t)sg.atom] = best;
      }
      bool placed = false;
      for (const auto& l : lists) placed = placed || !l.empty();
      if (!placed) {
        // Every placement of this round was undone (a head found no slot in its tail's warp): sweep
        // the first pending segment alone, with its other half (if wrapped) in the same warp.
        std::vector<PlaneSeg> rest;
        const int a0 = next.front().atom;
        int s = 0;
        for (const PlaneSeg& sg : next) {
          if (sg.atom == a0 && s < S) {
            lists[(size_t)s++].push_back(sg);
          } else {
            rest.push_back(sg);
          }
        }
        next.swap(rest);
      }
      int ylo = ny, yhi = 0;
      for (const auto& l : lists)
        for (const PlaneSeg& sg : l) {
          ylo = std::min(ylo, sg.ys);
          yhi = std::max(yhi, sg.ye);
        }
      if (yhi > ylo) {
        plan.items.push_back(make_int4(z, ylo, yhi, (int)plan.slot_ptr.size() - 1));
        for (const auto& l : lists) {
          for (const PlaneSeg& sg : l) plan.segs.push_back(sg);
          plan.slot_ptr.push_back((int)plan.segs.size());
        }
      }
      std::stable_sort(next.begin(), next.end(), [](const PlaneSeg& l, const PlaneSeg& r) {
        return l.ys != r.ys ? l.ys < r.ys : (l.flags != r.flags ? l.flags < r.flags : l.atom < r.atom);
      });
      pend.swap(next);
    }
  }
}

// Check a plan against its definition: every (atom, plane, grid row) of every cube exactly once, the
// segments of one slot ordered and disjoint, items of one plane contiguous, rows inside [ylo, yhi), and a
// wrapped atom's two halves in one warp when the grid is too small for the ring to order them.
// Returns 0 or the number of the first violated rule.
int plane_plan_check(const sho_grid* grid, const std::vector<AtomDev>& at, int cube, const PlanePlan& plan) {
  const int ny = grid->n[1], nz = grid->n[2];
  const bool per = grid->periodic != 0;
  const int W = kPlaneWarps, S = kPlaneSlots;
  const bool same_warp = ny - cube < kPlaneMaxStages;
  std::vector<int> count((size_t)at.size() * cube * ny, 0);  // (atom, iz, y) -> times covered
  int last_z = -1;
  std::vector<char> seen_z((size_t)nz, 0);
  for (size_t it = 0; it < plan.items.size(); it++) {
    const int4 item = plan.items[it];
    if (item.x < 0 || item.x >= nz) return 1;
    if (item.x != last_z) {
      if (seen_z[(size_t)item.x]) return 2;  // items of a plane are contiguous
      seen_z[(size_t)item.x] = 1;
      last_z = item.x;
    }
    std::vector<int> tail_warp(at.size(), -1), head_warp(at.size(), -1);
    for (int w = 0; w < W; w++)
      for (int s2 = 0; s2 < S; s2++) {
        const int li = item.w + w * S + s2;
        int prev_end = -1;
        for (int q = plan.slot_ptr[(size_t)li]; q < plan.slot_ptr[(size_t)li + 1]; q++) {
          const PlaneSeg& sg = plan.segs[(size_t)q];
          if (sg.ys < item.y || sg.ye > item.z || sg.ys >= sg.ye) return 3;
          if (sg.ys < prev_end) return 4;  // overlap within a slot
          prev_end = sg.ye;
          const AtomDev& a = at[(size_t)sg.atom];
          int z = a.o[2] + sg.iz;
          if (per) z = ((z % nz) + nz) % nz;
          if (z != item.x || sg.t2i != sg.atom * cube + sg.iz) return 5;
          for (int y = sg.ys; y < sg.ye; y++) {
            int iy = y - a.o[1];
            if (per) iy = ((iy % ny) + ny) % ny;
            if (iy != sg.iy0 + (y - sg.ys) || iy < 0 || iy >= cube) return 6;
            count[((size_t)sg.atom * cube + sg.iz) * ny + y]++;
          }
          if (sg.flags == 1) tail_warp[(size_t)sg.atom] = w;
          if (sg.flags == 2) head_warp[(size_t)sg.atom] = w;
        }
      }
    for (size_t a = 0; a < at.size(); a++) {
      if ((tail_warp[a] >= 0) != (head_warp[a] >= 0)) return 7;  // both halves in the same sweep
      if (same_warp && tail_warp[a] >= 0 && tail_warp[a] != head_warp[a]) return 8;
    }
  }
  for (size_t a = 0; a < at.size(); a++)
    for (int iz = 0; iz < cube; iz++) {
      int z = at[a].o[2] + iz;
      const bool zin = per || (z >= 0 && z < nz);
      for (int y = 0; y < ny; y++) {
        int iy = y - at[a].o[1];
        if (per) iy = ((iy % ny) + ny) % ny;
        const int want = (zin && iy >= 0 && iy < cube) ? 1 : 0;
        if (count[((size_t)a * cube + iz) * ny + y] != want) return 9;
      }
    }
  return 0;
}

cudaError_t launch_project_plane(const PlaneLaunch& p, sho_prec prec) {
  switch (p.numax) {
    case 0: return plane_mode<0>(p, prec);
    case 1: return plane_mode<1>(p, prec);
    case 2: return plane_mode<2>(p, prec);
    case 3: return plane_mode<3>(p, prec);
    case 4: return plane_mode<4>(p, prec);
    case 5: return plane_mode<5>(p, prec);
    case 6: return plane_mode<6>(p, prec);
    case 7: return plane_mode<7>(p, prec);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sho
