// sho_ozaki_project.cu -- FP64-accurate projection (SHO_P_FF64) with the x-pass on the fifth-generation
// tensor cores, by exact digit slicing of psi and of the x functions.
//
//   T1_a[iz][iy][b][nx] = sum_ix psi[j(ix, iy, iz)][b] phi^a_nx(ix)        (Sec. 3.2 step 1; eq. TuckerTensor)
//
// The x-pass of a cube row is a product of a (bands x points) and a (points x states) matrix.  As in the
// tensor-core expansion (sho_ozaki.cu; Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59, 2012, in
// fixed-point form):
//   * per (row, band, half row of 16 points) a power of two F = 2^e above max |psi| of those points, per
//     atom a power of two G_a above max |phi^a|;
//   * psi / F = sum_{i=1..6} d_i and phi^a_nx(ix) / G_a = sum_{j=1..6} e_j, signed integers times 2^(-8 i),
//     2^(-8 j) (round-to-nearest digits from the float pair of psi; at most 256 in magnitude);
//   * the products d_i e_j of each level L = i + j = 2 .. 8 go to one accumulator per level, where the
//     sums over the digit pairs and the 16 points stay integers below 2^24 and so are exact; levels above
//     8 are dropped (below 2^-56 F G_a per product);
//   * T1[nx] = G_a (F_0 S_0[nx] + F_1 S_1[nx]) with S_h the half row's level sums, summed as float pairs;
//     the y-pass then runs as float-float dot steps and each finished plane's sums go to the FP64
//     workspace of the z-pass kernel (k_project_ff_zpass), exactly as in the float-float projection.
// The operands are BF16 (digits of at most 8 significant bits -- integers up to 256 -- are exact in
// BF16).  The MMA sums over the psi digits as well as the points: for psi digit i the B operand stacks
// the x functions' digit j = L - i of every level L = 2..8 (64 rows: level x state, zero where L - i is
// not a digit), so that
//   D[band][(L, n)] += sum_k d_i[band][k] e_{L-i}[n][k]
// gathers the level-L products of all digit pairs in one accumulator column (at most 6 x 16 products of
// at most 2^16 per level: exact integers); M = 128 bands, N = 64, K = 16 points: 6 MMAs per half row.
// Opt-in (sho_set_project_kernel): measured about 20 % slower than the float-float kernel on GB300, its
// digit warps the bound.
//
// Persistent kernel, one CTA per SM over work items (atom, 128-band tile, cube plane) in contiguous
// ranges, 32 rows per item, with three warp roles that meet on mbarriers only:
//   * eight digit warps, thread = (band, half row): the row's 16 psi values (the next row's loaded ahead),
//     the frame, six digit slices written as the A operands of the half row's stage (three stages, free
//     once their MMAs are done), then arrivals on the stage's operand barrier and on the row's frame
//     barrier (four frame and accumulator slots, free once row gr - 4 is read back);
//   * one MMA thread: the atom's stacked digit table staged once per atom by a bulk copy (after every MMA
//     reading the previous one is done), then per half row 12 MMAs into the row's level accumulators in
//     tensor memory (four rows in flight, 512 columns), committed to the stage's barrier and, after the
//     row, to the row's barrier;
//   * four read-back warps, one thread per band: the row's level sums and frames, T1 as float pairs, the
//     y-pass, and at each plane's end its sums to the workspace.
// Deterministic: fixed order, exact leading levels, each item computed by one CTA.  Every wait is bounded;
// the first one that runs out stops every role (a shared flag), the kernel records kStatusTimeout, waits
// (bounded) for its own copies and MMAs, frees tensor memory and returns.
#include <algorithm>

#include <cuda_bf16.h>

#include "sho_device.cuh"
#include "sho_ff.cuh"
#include "sho_oz.cuh"
#include "sho_umma.cuh"

namespace sho {

constexpr int kOpBands = 128;                          // bands per item (the MMA M), one read-back thread each
constexpr int kOpN = 64;                               // MMA N: 7 levels x 8 states (levels 2..8)
constexpr int kOpHalf = 16;                            // cube points per half row (the K of one operand set)
constexpr int kOpDigits = 6;                           // digits per operand value
constexpr int kOpDigitThreads = 2 * kOpBands;          // thread = (band, half row)
constexpr int kOpThreads = kOpDigitThreads + kOpBands + 32;  // + read-back warps + MMA warp: 416
constexpr int kOpMmaWarp = (kOpDigitThreads + kOpBands) / 32;  // 12
constexpr uint32_t kOpAKc = kOpBands * 16;             // one K column of A (128 bands x 8 points, BF16): 2 KB
constexpr uint32_t kOpASlice = 2 * kOpAKc;             // one digit of one half row: 4 KB
constexpr uint32_t kOpAStage = kOpDigits * kOpASlice;  // the six digit slices of one half row: 24 KB
constexpr int kOpStages = 4;                            // half-row operand stages in flight
constexpr uint32_t kOpBKc = kOpN * 16;                 // one K column of B (64 rows x 8 points): 1 KB
constexpr uint32_t kOpBSlice = 4 * kOpBKc;             // one psi digit's stacked table, 32 points: 4 KB
constexpr uint32_t kOpBBytes = kOpDigits * kOpBSlice;  // stacked digit table of one atom: 24 KB
constexpr int kOpSlotCols = 2 * kOpN;                  // one row: an accumulator set per half row: 128
constexpr int kOpRows = 4;                             // rows whose accumulators and frames are in flight
constexpr int kOpCols = kOpRows * kOpSlotCols;         // 512

struct OpSmem {
  static constexpr size_t off_b = kOpStages * (size_t)kOpAStage;           // after four A stages (96 KB)
  static constexpr size_t off_e = off_b + kOpBBytes;                        // frames [4 rows][2 halves][128]
  static constexpr size_t off_bar = (off_e + kOpRows * 2 * kOpBands * 4 + 127) & ~(size_t)127;
  static constexpr size_t bytes = off_bar + 256;  // barriers, tensor-memory slot, abort flag
};
static_assert(OpSmem::bytes <= 227 * 1024, "one CTA per SM");

// ------------------------------------------------------------------------------------- tables
// Block a (128 threads): G_a = 2^e with max |phi_x| < 2^e; the digits e_j (j = 1..6) of phi_x / G_a; for
// each psi digit i the stacked B operand [8 point columns][64 rows (L - 2) 8 + n][4 points] holding e_{L-i}
// of state n (zero where L - i is not in 1..6, above numax and beyond the cube); and the y functions as
// float pairs [NP][C].  Every digit step is exact in FP64.
template <int NU>
__global__ void __launch_bounds__(128) k_op_tables(GridDev g, const AtomDev* __restrict__ atoms,
                                                   __nv_bfloat16* __restrict__ btab, float* __restrict__ gpow,
                                                   float2* __restrict__ tyff) {
  constexpr int NP = NU + 1;
  __shared__ double px[NP][32];
  __shared__ float dg[kOpDigits][8][32];  // e_j [digit][state][point]
  __shared__ double red[4];
  const int a = blockIdx.x, tid = threadIdx.x, C = g.cube;
  const AtomDev at = atoms[a];
  if (tid < 32) {
    double col[NP];
    if (tid < C) {
      phi_column(cube_offset(at.o[0], tid, g.h, at.X[0]), at.sigma, NU, col, 1);
    } else {
#pragma unroll
      for (int n = 0; n < NP; n++) col[n] = 0.0;
    }
#pragma unroll
    for (int n = 0; n < NP; n++) px[n][tid] = col[n];
  } else if (tid >= 64 && tid - 64 < C) {
    const int i = tid - 64;
    double col[NP];
    phi_column(cube_offset(at.o[1], i, g.h, at.X[1]), at.sigma, NU, col, 1);
#pragma unroll
    for (int n = 0; n < NP; n++) {
      const ff f = ff_from_double_exact(col[n]);
      tyff[((size_t)a * NP + n) * C + i] = make_float2(f.hi, f.lo);
    }
  }
  __syncthreads();
  double m = 0.0;
  for (int i = tid; i < NP * 32; i += 128) m = fmax(m, fabs(px[i / 32][i % 32]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) red[tid >> 5] = m;
  __syncthreads();
  m = fmax(fmax(red[0], red[1]), fmax(red[2], red[3]));
  int e = 0;
  if (m > 0.0) (void)frexp(m, &e);  // m < 2^e
  const double G = m > 0.0 ? ldexp(1.0, e) : 1.0;
  if (tid == 0) gpow[a] = (float)G;
  const double ginv = 1.0 / G;
  for (int idx = tid; idx < 8 * 32; idx += 128) {
    const int n = idx / 32, i = idx % 32;
    double v = n < NP ? px[n][i] * ginv : 0.0;  // |v| < 1
    double sc = 1.0, isc = 1.0;
#pragma unroll
    for (int j = 0; j < kOpDigits; j++) {
      sc *= 256.0;
      isc *= 0.00390625;
      const double d = rint(v * sc) * isc;
      v -= d;
      dg[j][n][i] = (float)d;  // at most 256 (then 128) times 2^(-8 (j + 1))
    }
  }
  __syncthreads();
  __nv_bfloat16* dst = btab + (size_t)a * (kOpBBytes / 2);
  for (int idx = tid; idx < kOpDigits * kOpN * 32; idx += 128) {
    const int di = idx / (kOpN * 32), r = (idx / 32) % kOpN, k = idx % 32;  // psi digit i = di + 1
    const int L = r / 8 + 2, n = r % 8, j = L - (di + 1);                    // x digit j (1-based)
    const float v = (r < 56 && j >= 1 && j <= kOpDigits) ? dg[j - 1][n][k] : 0.0f;
    // digits of at most 8 significant bits: exact in BF16
    dst[di * (kOpBSlice / 2) + (k / 8) * (kOpBKc / 2) + r * 8 + (k % 8)] = __float2bfloat16_rn(v);
  }
}

// ------------------------------------------------------------------------------------- projection
template <int NU>
__global__ void __launch_bounds__(kOpThreads, 1)  // 13 warps: at most 128 registers (16 K per SM sub-partition)
    k_project_ozaki(GridDev g, const double* __restrict__ psi, const AtomDev* __restrict__ atoms, int natoms,
                    const __nv_bfloat16* __restrict__ btab, const float* __restrict__ gpow,
                    const float2* __restrict__ tyff, double* __restrict__ t2g, int* __restrict__ status,
                    long long wait_cycles) {
  using BS = Basis<NU>;
  constexpr int NP = BS::NP, P = BS::P;
  static_assert(NP <= 8, "8 states per level column group");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int C = g.cube, Nx = g.n[0], Ny = g.n[1], Nz = g.n[2], B = g.nbands;
  const int nbt = (B + kOpBands - 1) / kOpBands;
  const long long nitems = (long long)natoms * nbt * C;
  const long long w0 = nitems * blockIdx.x / gridDim.x, w1 = nitems * (blockIdx.x + 1) / gridDim.x;
  const int nhalf = C > kOpHalf ? 2 : 1;
  const uint32_t sbase = um_smem(smem_raw);
  const uint32_t sB = sbase + (uint32_t)OpSmem::off_b;
  int* sexp = reinterpret_cast<int*>(smem_raw + OpSmem::off_e);  // [row slot][half][band]
  unsigned char* barp = smem_raw + OpSmem::off_bar;
  const uint32_t bar0 = um_smem(barp);
  // operand stages by half-row count modulo 3; accumulators and frames by row modulo 4
  constexpr uint32_t kFa = 0, kCa = kFa + 8 * kOpStages, kXf = kCa + 8 * kOpStages, kRd = kXf + 8 * kOpRows,
                     kAe = kRd + 8 * kOpRows, kBb = kAe + 8 * kOpRows, kDr = kBb + 8, kSlot = kDr + 8;
  static_assert(kSlot + 8 <= OpSmem::bytes - OpSmem::off_bar, "barrier area");
  auto fa = [&](int q) { return bar0 + kFa + 8 * q; };  // A operands of stage q written (128 arrivals)
  auto ca = [&](int q) { return bar0 + kCa + 8 * q; };  // MMAs reading stage q done (MMA commit)
  auto xf = [&](int r) { return bar0 + kXf + 8 * r; };  // frames of row slot r written (256)
  auto rd = [&](int r) { return bar0 + kRd + 8 * r; };  // MMAs of row slot r done (MMA commit)
  auto ae = [&](int r) { return bar0 + kAe + 8 * r; };  // accumulators and frames of row slot r read (128)
  const uint32_t bb = bar0 + kBb;                       // digit table staged (bulk copy)
  const uint32_t dr = bar0 + kDr;                       // drain: every MMA issued so far done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(barp + kSlot);
  volatile int* s_abort = reinterpret_cast<volatile int*>(barp + kSlot + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    *s_abort = 0;
    for (int q = 0; q < kOpStages; q++) {
      um_mbar_init_n(fa(q), kOpBands);
      um_mbar_init(ca(q));
    }
    for (int r = 0; r < kOpRows; r++) {
      um_mbar_init_n(xf(r), kOpDigitThreads);
      um_mbar_init(rd(r));
      um_mbar_init_n(ae(r), kOpBands);
    }
    um_mbar_init(bb);
    um_mbar_init(dr);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) tmem_alloc(um_smem(tmem_slot), kOpCols);
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  const uint32_t tmem = *tmem_slot;

  // a wait that gives up when another thread's wait ran out, or after `wait_cycles` (then it says so)
  auto wait = [&](uint32_t bar, uint32_t parity) {
    if (um_mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!um_mbar_try(bar, parity)) {
      if (*s_abort) return false;
      if (clock64() - t0 > wait_cycles) {
        *s_abort = 1;
        return false;
      }
    }
    return true;
  };
  // work item w: atom, band tile, cube plane
  auto item = [&](long long w, int& a, int& bt, int& iz) {
    a = (int)(w / ((long long)nbt * C));
    const int r = (int)(w - (long long)a * nbt * C);
    bt = r / C;
    iz = r - bt * C;
  };

  if (warp == kOpMmaWarp) {
    // ---- MMA thread
    if (lane == 0) {
      constexpr uint32_t idesc = umma_idesc(kUmmaBF16, kOpBands, kOpN);
      const uint64_t ad0 = umma_desc(sbase, kOpAKc, 128), bd0 = umma_desc(sB, kOpBKc, 128);
      int gr = 0, cur = -1;
      uint32_t bbp = 0, drp = 0;
      bool any = false, ok = true;
      for (long long w = w0; w < w1 && ok; w++) {
        int a, bt, iz;
        item(w, a, bt, iz);
        if (a != cur) {
          // every MMA reading the previous atom's table done, then this atom's table staged
          if (any) {
            umma_commit(dr);
            if (!wait(dr, drp)) break;
            drp ^= 1u;
          }
          fence_async_smem();
          um_expect_tx(bb, kOpBBytes);
          um_bulk(sB, btab + (size_t)a * (kOpBBytes / 2), kOpBBytes, bb);
          if (!wait(bb, bbp)) {
            (void)um_mbar_wait(bb, bbp, kDefaultWaitCycles);  // the copy completes before the CTA exits
            break;
          }
          bbp ^= 1u;
          cur = a;
        }
        for (int iy = 0; iy < C && ok; iy++, gr++) {
          const int rs = gr & (kOpRows - 1);
          // the row slot's accumulators read back (row gr - 4)
          if (gr >= kOpRows && !wait(ae(rs), (uint32_t)(((gr - kOpRows) / kOpRows) & 1))) { ok = false; break; }
          // both half rows' operands written, then the row's MMAs, the two halves' accumulator sets
          // interleaved
          for (int h = 0; h < nhalf && ok; h++) {
            const int st = gr * nhalf + h;
            if (!wait(fa(st % kOpStages), (uint32_t)((st / kOpStages) & 1))) ok = false;
          }
          if (!ok) break;
          tc05_fence_after();
          const int st0 = gr * nhalf;
          const uint64_t ad_0 = ad0 + (uint64_t)(((st0 % kOpStages) * kOpAStage) >> 4);
          const uint64_t ad_1 = ad0 + (uint64_t)((((st0 + 1) % kOpStages) * kOpAStage) >> 4);
          const uint32_t drow = tmem + (uint32_t)(rs * kOpSlotCols);
#pragma unroll
          for (int i = 0; i < kOpDigits; i++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
              if (h >= nhalf) continue;
              umma_f16(drow + (uint32_t)(h * kOpN), (h ? ad_1 : ad_0) + (uint64_t)((i * kOpASlice) >> 4),
                       bd0 + (uint64_t)((i * kOpBSlice + 2 * h * kOpBKc) >> 4), idesc,
                       i > 0);  // the first digit starts each accumulator set
            }
          for (int h = 0; h < nhalf; h++) umma_commit(ca((st0 + h) % kOpStages));
          if (!ok) break;
          umma_commit(rd(rs));
          any = true;
        }
      }
      if (any) {  // every MMA issued completes before the tensor memory is released
        umma_commit(dr);
        (void)um_mbar_wait(dr, drp, kDefaultWaitCycles);
      }
    }
    __syncwarp();
  } else if (tid < kOpDigitThreads) {
    // ---- digit threads, thread = (band, half row): per row the 16 psi values, their frame and six digit
    // slices as the A operands of the half row's stage, once the stage's earlier MMAs are done and the
    // row slot's frames (row gr - 4) are read back
    const int bl = tid & (kOpBands - 1), hh = tid >> 7;
    const bool active = hh < nhalf;  // a second half row exists
    int gr = 0, cur = -1;
    int jx[kOpHalf];
    bool range_bad = false;
    double pv[kOpHalf], pn[kOpHalf];
    for (long long w = w0; w < w1; w++) {
      int a, bt, iz;
      item(w, a, bt, iz);
      const AtomDev at = atoms[a];
      if (a != cur) {
#pragma unroll
        for (int k = 0; k < kOpHalf; k++) {
          const int ix = hh * kOpHalf + k;
          jx[k] = ix < C ? cube_index(at.o[0], ix, Nx, g.periodic) : -1;
        }
        cur = a;
      }
      const int b = bt * kOpBands + bl;
      const bool bvalid = b < B && active;
      const int jz = cube_index(at.o[2], iz, Nz, g.periodic);
      auto load_row = [&](int iy, double (&v)[kOpHalf]) {
        const int jy = cube_index(at.o[1], iy, Ny, g.periodic);
        const bool rok = bvalid && jz >= 0 && jy >= 0;
        const double* row = psi + (((size_t)(rok ? jz : 0) * Ny + (rok ? jy : 0)) * Nx) * (size_t)B + b;
#pragma unroll
        for (int k = 0; k < kOpHalf; k++) v[k] = (rok && jx[k] >= 0) ? row[(size_t)jx[k] * B] : 0.0;
      };
      load_row(0, pv);
      bool ok = true;
      for (int iy = 0; iy < C; iy++, gr++) {
        const int rs = gr & (kOpRows - 1);
        const int st = gr * nhalf + hh, q = st % kOpStages;
        if (iy + 1 < C) load_row(iy + 1, pn);  // in flight during this row
        // stage free: the MMAs of half row st - 3 done; frame slot free: row gr - 4 read back
        if ((active && st >= kOpStages && !wait(ca(q), (uint32_t)(((st - kOpStages) / kOpStages) & 1))) ||
            (gr >= kOpRows && !wait(ae(rs), (uint32_t)(((gr - kOpRows) / kOpRows) & 1)))) {
          ok = false;
          break;
        }
        // the frame: a power of two above max |psi| of the 16 points, from the largest high word (the
        // magnitudes of doubles order as their bit patterns)
        unsigned int mh = 0u;
#pragma unroll
        for (int k = 0; k < kOpHalf; k++) {
          range_bad |= ff_out_of_range(pv[k]);
          mh = max(mh, (unsigned int)((unsigned long long)__double_as_longlong(pv[k]) >> 32) & 0x7fffffffu);
        }
        int e = (int)(mh >> 20) - 1023 + 1;  // |psi| < 2^e
        e = max(-124, min(e, 127));
        sexp[(rs * 2 + hh) * kOpBands + bl] = e;
        if (active) {
          const float s1 = oz_pow2(-(e >> 1)), s2 = oz_pow2(-(e - (e >> 1)));  // 2^-e in two factors
          unsigned char* arow = smem_raw + (size_t)q * kOpAStage + (size_t)bl * 16;
#pragma unroll
          for (int kc = 0; kc < 4; kc++) {  // groups of 4 points: half of an 8-point BF16 core-matrix row
            float dg[kOpDigits][4];
#pragma unroll
            for (int k4 = 0; k4 < 4; k4++) {
              const ff v = ff_from_double(pv[4 * kc + k4]);
              float rem = __fmul_rn(__fmul_rn(v.hi, s1), s2);  // |rem| < 1
              const float lo = __fmul_rn(__fmul_rn(v.lo, s1), s2);
              dg[0][k4] = oz_digit(rem, 0x1.8p+15f);  // grid 2^-8
              dg[1][k4] = oz_digit(rem, 0x1.8p+7f);   // grid 2^-16
              dg[2][k4] = oz_digit(rem, 0x1.8p-1f);   // grid 2^-24: what is left of hi lies below it
              rem = __fadd_rn(rem, lo);
              dg[3][k4] = oz_digit(rem, 0x1.8p-9f);   // grid 2^-32
              dg[4][k4] = oz_digit(rem, 0x1.8p-17f);  // grid 2^-40
              dg[5][k4] = oz_digit(rem, 0x1.8p-25f);  // grid 2^-48
            }
#pragma unroll
            for (int i = 0; i < kOpDigits; i++) {
              const __nv_bfloat162 lo2 = __floats2bfloat162_rn(dg[i][0], dg[i][1]);  // exact: 8-bit digits
              const __nv_bfloat162 hi2 = __floats2bfloat162_rn(dg[i][2], dg[i][3]);
              *reinterpret_cast<uint2*>(arow + i * kOpASlice + (kc >> 1) * kOpAKc + (kc & 1) * 8) =
                  make_uint2(*reinterpret_cast<const uint32_t*>(&lo2), *reinterpret_cast<const uint32_t*>(&hi2));
            }
          }
          fence_async_smem();  // the A slices become visible to the tensor core
          um_mbar_arrive(fa(q));
        }
        um_mbar_arrive(xf(rs));
#pragma unroll
        for (int k = 0; k < kOpHalf; k++) pv[k] = pn[k];
      }
      if (!ok) break;
    }
    if (__any_sync(0xffffffffu, range_bad) && lane == 0 && status) atomicOr(status, kStatusRange);
  } else {
    // ---- read-back threads, one per band (tensor-memory lanes 32 (warp - 8) ..): per row T1 from the
    // level sums and frames as float pairs, the float-float y-pass, and each plane's sums in FP64
    const int bl = tid - kOpDigitThreads;
    const uint32_t tlane = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    int gr = 0;
    for (long long w = w0; w < w1; w++) {
      int a, bt, iz;
      item(w, a, bt, iz);
      const int b = bt * kOpBands + bl;
      const bool bvalid = b < B;
      const float G = gpow[a];
      const float2* ty = tyff + (size_t)a * NP * C;
      float t2s[P], t2c[P];
#pragma unroll
      for (int p = 0; p < P; p++) t2s[p] = t2c[p] = 0.0f;
      bool ok = true;
      for (int iy = 0; iy < C; iy++, gr++) {
        const int rs = gr & (kOpRows - 1);
        if (!wait(xf(rs), (uint32_t)((gr / kOpRows) & 1)) || !wait(rd(rs), (uint32_t)((gr / kOpRows) & 1))) {
          ok = false;
          break;
        }
        tc05_fence_after();
        const uint32_t tcol = tlane + (uint32_t)(rs * kOpSlotCols);
        // T1[n] = G (2^e0 S0[n] + 2^e1 S1[n]) with S_h[n] = sum over levels 2..8 of column (L - 2) 8 + n,
        // the half rows read one after the other; each scale applied in two power-of-two factors
        float th[NP], tl[NP];
        ff t1[NP];
        for (int h = 0; h < nhalf; h++) {
          float sh[NP], sl[NP];  // levels 2..4 as a float pair, then the smaller levels added to the low part
          const uint32_t s0 = tcol + (uint32_t)(h * kOpN);
          {
            float v[32];  // levels 2..5
            tmem_ld8x4(s0, s0 + 8, s0 + 16, s0 + 24, v);
#pragma unroll
            for (int n = 0; n < NP; n++) {
              float c0, c1;
              oz_two_sum(v[n], v[8 + n], sh[n], c0);   // levels 2 and 3 (exact integers)
              oz_two_sum(sh[n], v[16 + n], sh[n], c1);  // level 4
              sl[n] = __fadd_rn(__fadd_rn(c0, c1), v[24 + n]);
            }
          }
          {
            float v[32];  // levels 6..8 and the zero columns
            tmem_ld8x4(s0 + 32, s0 + 40, s0 + 48, s0 + 56, v);
#pragma unroll
            for (int n = 0; n < NP; n++) sl[n] = __fadd_rn(sl[n], __fadd_rn(v[n], __fadd_rn(v[8 + n], v[16 + n])));
          }
          const int eh = sexp[(rs * 2 + h) * kOpBands + bl];
          const float ga = G * oz_pow2(eh >> 1), gb = oz_pow2(eh - (eh >> 1));
#pragma unroll
          for (int n = 0; n < NP; n++) {
            const float hs = __fmul_rn(__fmul_rn(sh[n], ga), gb);
            const float ls = __fmul_rn(__fmul_rn(sl[n], ga), gb);
            if (h == 0) {
              th[n] = hs;
              tl[n] = ls;
            } else {
              float hi, lo;
              oz_two_sum(th[n], hs, hi, lo);
              th[n] = hi;
              tl[n] = __fadd_rn(lo, __fadd_rn(tl[n], ls));
            }
          }
        }
        tc05_fence_before();
        um_mbar_arrive(ae(rs));  // the row slot's accumulators and frames may be refilled
#pragma unroll
        for (int n = 0; n < NP; n++) oz_two_sum(th[n], tl[n], t1[n].hi, t1[n].lo);  // the halves may cancel
        // y-pass (a4) as float-float dot steps
#pragma unroll
        for (int ny = 0; ny < NP; ny++) {
          const float2 wy = ty[ny * C + iy];
#pragma unroll
          for (int nx = 0; nx + ny <= NU; nx++)
            ff_dot_step(t2s[BS::pair(nx, ny)], t2c[BS::pair(nx, ny)], t1[nx], ff{wy.x, wy.y});
        }
      }
      if (!ok) break;
      // the finished plane's sums in FP64 for the z-pass (zero for a plane outside an open grid)
      if (bvalid) {
        double* out = t2g + ((size_t)a * C + iz) * P * B + b;
#pragma unroll
        for (int p = 0; p < P; p++) out[(size_t)p * B] = ff_to_double(t2s[p], t2c[p]);
      }
    }
  }
  __syncthreads();
  if (tid == 0 && *s_abort && status) atomicOr(status, kStatusTimeout);
  tc05_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kOpCols);
}

// ------------------------------------------------------------------------------------ launchers
// The tensor-core form covers numax <= 7 (8 states fit N = 16), cubes of at most 32 points, no spherical
// support, and one CTA's shared memory per SM.
bool ozaki_project_ok(const ProjectLaunch& p) {
  return p.op && p.numax <= 7 && p.g.cube <= 32 && p.g.r2max <= 0.0;
}

template <int NU>
static cudaError_t op_nu(const ProjectLaunch& p) {
  if constexpr (NU > 7) {
    return cudaErrorNotSupported;
  } else {
    const OpLayout L = op_layout(p.natoms, p.g.cube, p.numax);
    char* ws = static_cast<char*>(p.op);
    __nv_bfloat16* btab = reinterpret_cast<__nv_bfloat16*>(ws + L.btab);
    float* gpow = reinterpret_cast<float*>(ws + L.gpow);
    float2* tyff = reinterpret_cast<float2*>(ws + L.tyff);
    k_op_tables<NU><<<(unsigned)p.natoms, 128, 0, p.stream>>>(p.g, p.atoms, btab, gpow, tyff);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto kern = k_project_ozaki<NU>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OpSmem::bytes);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    if (fa.maxThreadsPerBlock < kOpThreads) return cudaErrorLaunchOutOfResources;  // registers of the build
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long nitems = (long long)p.natoms * ((p.g.nbands + kOpBands - 1) / kOpBands) * p.g.cube;
    const unsigned nblk = (unsigned)std::min<long long>(nitems, sms);
    kern<<<nblk, kOpThreads, OpSmem::bytes, p.stream>>>(p.g, static_cast<const double*>(p.psi), p.atoms, p.natoms,
                                                        btab, gpow, tyff, static_cast<double*>(p.t2), p.status,
                                                        p.wait_cycles);
    return cudaGetLastError();
  }
}

cudaError_t launch_project_ozaki(const ProjectLaunch& p) {
  switch (p.numax) {
    case 0: return op_nu<0>(p);
    case 1: return op_nu<1>(p);
    case 2: return op_nu<2>(p);
    case 3: return op_nu<3>(p);
    case 4: return op_nu<4>(p);
    case 5: return op_nu<5>(p);
    case 6: return op_nu<6>(p);
    case 7: return op_nu<7>(p);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace sho
