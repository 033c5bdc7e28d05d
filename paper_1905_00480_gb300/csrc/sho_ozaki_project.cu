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
//   * the products d_i e_j of level L = i + j = 2, 3, 4 go to one accumulator per level, where the sums
//     over the 16 points stay integers below 2^24 and so are exact; levels 5 .. 8 share a fourth one;
//     levels above 8 are dropped (below 2^-56 F G_a per product);
//   * T1[nx] = G_a (F_0 S_0[nx] + F_1 S_1[nx]) with S_h the half row's level sums, summed as float pairs;
//     the y-pass then runs as float-float dot steps and each finished plane's sums go to the FP64
//     workspace of the z-pass kernel (k_project_ff_zpass), exactly as in the float-float projection.
// The operands are TF32 (digits of at most 9 significant bits are exact in TF32), M = 128 bands, N = 16
// (the numax + 1 <= 8 states, zero-padded), K = 8 points per MMA, two K steps per half row.
//
// Persistent kernel, one CTA per SM over work items (atom, 128-band tile, cube plane) in contiguous
// ranges, 32 rows per item, with three warp roles that meet on mbarriers only:
//   * eight digit warps, thread = (band, half row): the row's 16 psi values (the next row's loaded ahead),
//     the frame, six digit slices written as the A operands of the row's slot (two slots by row parity,
//     free once the MMAs of row gr - 2 are done), then arrivals on the slot's operand barrier and on the
//     frame barrier of the row (four frame and accumulator slots, free once row gr - 4 is read back);
//   * one MMA thread: the atom's digit table staged once per atom by a bulk copy (after every MMA reading
//     the previous one is done), then per row 2 halves x 26 digit pairs x 2 K steps of M128 N16 K8 MMAs into
//     the row's level accumulators in tensor memory (four rows in flight, 512 columns), committed to
//     the row's barrier;
//   * four read-back warps, one thread per band: the row's accumulators and frames, T1 as float pairs,
//     the y-pass, and at each plane's end its sums to the workspace.
// Opt-in (sho_set_project_kernel): measured at twice the float-float kernel's time on GB300, bound by its
// MMA thread -- the 104 narrow MMAs of a row take about 75 cycles each while the digit warps wait.
// Deterministic: fixed order, exact leading levels, each item computed by one CTA.  Every wait is bounded;
// the first one that runs out stops every role (a shared flag), the kernel records kStatusTimeout, waits
// (bounded) for its own copies and MMAs, frees tensor memory and returns.
#include <algorithm>

#include "sho_device.cuh"
#include "sho_ff.cuh"
#include "sho_oz.cuh"
#include "sho_umma.cuh"

namespace sho {

constexpr int kOpBands = 128;                          // bands per item (the MMA M), one read-back thread each
constexpr int kOpN = 16;                               // MMA N: the states, zero-padded
constexpr int kOpHalf = 16;                            // cube points per half row (the K of one operand set)
constexpr int kOpDigits = 6;                           // digits per operand value
constexpr int kOpMaxLevel = 8;                         // digit pairs (i, j) with i + j <= 8 are multiplied
constexpr int kOpGroups = 4;                           // accumulators: levels 2, 3, 4 and 5..8
constexpr int kOpDigitThreads = 2 * kOpBands;          // thread = (band, half row)
constexpr int kOpThreads = kOpDigitThreads + kOpBands + 32;  // + read-back warps + MMA warp: 416
constexpr int kOpMmaWarp = (kOpDigitThreads + kOpBands) / 32;  // 12
constexpr uint32_t kOpAKc = kOpBands * 16;             // one K column of A (128 bands x 4 points, TF32): 2 KB
constexpr uint32_t kOpASlice = 4 * kOpAKc;             // one digit of one half row: 8 KB
constexpr uint32_t kOpASlot = 2 * kOpDigits * kOpASlice;  // both halves, six digits: 96 KB
constexpr uint32_t kOpBKc = kOpN * 16;                 // one K column of B (16 states x 4 points): 256 B
constexpr uint32_t kOpBSlice = 8 * kOpBKc;             // one digit, 32 points: 2 KB
constexpr uint32_t kOpBBytes = kOpDigits * kOpBSlice;  // digit table of one atom: 12 KB
constexpr int kOpSlotCols = 2 * kOpGroups * kOpN;      // tensor-memory columns of one row: 128
constexpr int kOpRows = 4;                             // rows whose accumulators and frames are in flight
constexpr int kOpCols = kOpRows * kOpSlotCols;         // 512

struct OpSmem {
  static constexpr size_t off_b = 2 * (size_t)kOpASlot;                     // after two A slots (192 KB)
  static constexpr size_t off_e = off_b + kOpBBytes;                        // frames [4 rows][2 halves][128]
  static constexpr size_t off_bar = (off_e + kOpRows * 2 * kOpBands * 4 + 127) & ~(size_t)127;
  static constexpr size_t bytes = off_bar + 256;  // barriers, tensor-memory slot, abort flag
};
static_assert(OpSmem::bytes <= 227 * 1024, "one CTA per SM");

// ------------------------------------------------------------------------------------- tables
// Block a (128 threads): G_a = 2^e with max |phi_x| < 2^e, the digit table of phi_x / G_a in the B layout
// [6 digits][8 point columns][16 states][4 points] (zero above numax and beyond the cube), and the y
// functions as float pairs [NP][C].  Every digit step is exact in FP64.
template <int NU>
__global__ void __launch_bounds__(128) k_op_tables(GridDev g, const AtomDev* __restrict__ atoms,
                                                   float* __restrict__ btab, float* __restrict__ gpow,
                                                   float2* __restrict__ tyff) {
  constexpr int NP = NU + 1;
  __shared__ double px[NP][32];
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
  float* dst = btab + (size_t)a * (kOpBBytes / 4);
  for (int idx = tid; idx < kOpN * 32; idx += 128) {
    const int n = idx / 32, i = idx % 32;
    double v = n < NP ? px[n][i] * ginv : 0.0;  // |v| < 1
    double sc = 1.0, isc = 1.0;
#pragma unroll
    for (int j = 0; j < kOpDigits; j++) {
      sc *= 256.0;
      isc *= 0.00390625;
      const double d = rint(v * sc) * isc;
      v -= d;
      dst[j * (kOpBSlice / 4) + (i / 4) * (kOpBKc / 4) + n * 4 + (i % 4)] = (float)d;
    }
  }
}

// ------------------------------------------------------------------------------------- projection
template <int NU>
__global__ void __launch_bounds__(kOpThreads, 1)
    k_project_ozaki(GridDev g, const double* __restrict__ psi, const AtomDev* __restrict__ atoms, int natoms,
                    const float* __restrict__ btab, const float* __restrict__ gpow, const float2* __restrict__ tyff,
                    double* __restrict__ t2g, int* __restrict__ status, long long wait_cycles) {
  using BS = Basis<NU>;
  constexpr int NP = BS::NP, P = BS::P;
  static_assert(NP <= 8, "the states fit one 8-column read-back");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int C = g.cube, Nx = g.n[0], Ny = g.n[1], Nz = g.n[2], B = g.nbands;
  const int nbt = (B + kOpBands - 1) / kOpBands;
  const long long nitems = (long long)natoms * nbt * C;
  const long long w0 = nitems * blockIdx.x / gridDim.x, w1 = nitems * (blockIdx.x + 1) / gridDim.x;
  const int nhalf = C > kOpHalf ? 2 : 1;
  const uint32_t sbase = um_smem(smem_raw);
  const uint32_t sB = sbase + (uint32_t)OpSmem::off_b;
  int* sexp = reinterpret_cast<int*>(smem_raw + OpSmem::off_e);  // [slot][half][band]
  unsigned char* barp = smem_raw + OpSmem::off_bar;
  const uint32_t bar0 = um_smem(barp);
  // A operand slots by row parity; accumulators and frames by row modulo 4
  auto fb = [&](int s) { return bar0 + 8 * s; };        // A operands of slot s written (256 arrivals)
  auto xf = [&](int r) { return bar0 + 16 + 8 * r; };   // frames of row slot r written (256)
  auto rd = [&](int r) { return bar0 + 48 + 8 * r; };   // MMAs of row slot r done (MMA commit)
  auto ae = [&](int r) { return bar0 + 80 + 8 * r; };   // accumulators and frames of row slot r read (128)
  const uint32_t bb = bar0 + 112;                       // digit table staged (bulk copy)
  const uint32_t dr = bar0 + 120;                       // drain: every MMA issued so far done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(barp + 128);
  volatile int* s_abort = reinterpret_cast<volatile int*>(barp + 132);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    *s_abort = 0;
    for (int s = 0; s < 2; s++) um_mbar_init_n(fb(s), kOpDigitThreads);
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
      constexpr uint32_t idesc = umma_idesc(kUmmaTF32, kOpBands, kOpN);
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
          um_bulk(sB, btab + (size_t)a * (kOpBBytes / 4), kOpBBytes, bb);
          if (!wait(bb, bbp)) {
            (void)um_mbar_wait(bb, bbp, kDefaultWaitCycles);  // the copy completes before the CTA exits
            break;
          }
          bbp ^= 1u;
          cur = a;
        }
        for (int iy = 0; iy < C; iy++, gr++) {
          const int slot = gr & 1, rs = gr & (kOpRows - 1);
          // the row slot's accumulators read back (row gr - 4), the A operands of row gr written
          if (gr >= kOpRows && !wait(ae(rs), (uint32_t)(((gr - kOpRows) >> 2) & 1))) { ok = false; break; }
          if (!wait(fb(slot), (uint32_t)((gr >> 1) & 1))) { ok = false; break; }
          tc05_fence_after();
          const uint64_t ad = ad0 + (uint64_t)((slot * kOpASlot) >> 4);
          for (int h = 0; h < nhalf; h++) {
            // consecutive MMAs share their A operand (one digit slice, one K step): pairs j for each (i, ks)
#pragma unroll
            for (int i = 1; i <= kOpDigits; i++)
#pragma unroll
              for (int ks = 0; ks < 2; ks++)
#pragma unroll
                for (int j = 1; j <= kOpDigits; j++) {
                  if (i + j > kOpMaxLevel) continue;
                  const int grp = (i + j < 5 ? i + j : 5) - 2;
                  const uint32_t dacc = tmem + (uint32_t)(rs * kOpSlotCols + (h * kOpGroups + grp) * kOpN);
                  // the first product of each level group in the row starts its accumulator
                  const bool acc = ks > 0 || !(i == 1 && j <= 4);
                  umma_tf32(dacc,
                            ad + (uint64_t)(((h * kOpDigits + i - 1) * kOpASlice + 2 * ks * kOpAKc) >> 4),
                            bd0 + (uint64_t)(((j - 1) * kOpBSlice + (4 * h + 2 * ks) * kOpBKc) >> 4), idesc, acc);
                }
          }
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
    // slices as the A operands of the row's slot, once the slot's MMAs and read-back of row gr - 2 are done
    const int bl = tid & (kOpBands - 1), hh = tid >> 7;
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
      const bool bvalid = b < B;
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
        const int slot = gr & 1, rs = gr & (kOpRows - 1);
        if (iy + 1 < C) load_row(iy + 1, pn);  // in flight during this row
        // A slot free: the MMAs of row gr - 2 done; frame slot free: row gr - 4 read back
        if ((gr >= 2 && !wait(rd((gr - 2) & (kOpRows - 1)), (uint32_t)(((gr - 2) >> 2) & 1))) ||
            (gr >= kOpRows && !wait(ae(rs), (uint32_t)(((gr - kOpRows) >> 2) & 1)))) {
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
        const float s1 = oz_pow2(-(e >> 1)), s2 = oz_pow2(-(e - (e >> 1)));  // 2^-e in two factors
        unsigned char* arow = smem_raw + (size_t)slot * kOpASlot + (size_t)hh * kOpDigits * kOpASlice + (size_t)bl * 16;
#pragma unroll
        for (int kc = 0; kc < 4; kc++) {
          float dg[kOpDigits][4];
#pragma unroll
          for (int q = 0; q < 4; q++) {
            const ff v = ff_from_double(pv[4 * kc + q]);
            float rem = __fmul_rn(__fmul_rn(v.hi, s1), s2);  // |rem| < 1
            const float lo = __fmul_rn(__fmul_rn(v.lo, s1), s2);
            dg[0][q] = oz_digit(rem, 0x1.8p+15f);  // grid 2^-8
            dg[1][q] = oz_digit(rem, 0x1.8p+7f);   // grid 2^-16
            dg[2][q] = oz_digit(rem, 0x1.8p-1f);   // grid 2^-24: what is left of hi lies below it
            rem = __fadd_rn(rem, lo);
            dg[3][q] = oz_digit(rem, 0x1.8p-9f);   // grid 2^-32
            dg[4][q] = oz_digit(rem, 0x1.8p-17f);  // grid 2^-40
            dg[5][q] = oz_digit(rem, 0x1.8p-25f);  // grid 2^-48
          }
#pragma unroll
          for (int i = 0; i < kOpDigits; i++)
            *reinterpret_cast<float4*>(arow + i * kOpASlice + kc * kOpAKc) =
                make_float4(dg[i][0], dg[i][1], dg[i][2], dg[i][3]);
        }
        fence_async_smem();  // the A slices become visible to the tensor core
        um_mbar_arrive(fb(slot));
        um_mbar_arrive(xf(rs));
#pragma unroll
        for (int k = 0; k < kOpHalf; k++) pv[k] = pn[k];
      }
      if (!ok) break;
    }
    if (__any_sync(0xffffffffu, range_bad) && lane == 0 && status) atomicOr(status, kStatusRange);
  } else {
    // ---- read-back threads, one per band (tensor-memory lanes 32 (warp - 8) ..): per row T1 from the
    // level accumulators and frames as float pairs, the float-float y-pass, and each plane's sums in FP64
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
        if (!wait(xf(rs), (uint32_t)((gr >> 2) & 1)) || !wait(rd(rs), (uint32_t)((gr >> 2) & 1))) {
          ok = false;
          break;
        }
        tc05_fence_after();
        const uint32_t tcol = tlane + (uint32_t)(rs * kOpSlotCols);
        const int e0 = sexp[(rs * 2 + 0) * kOpBands + bl], e1 = sexp[(rs * 2 + 1) * kOpBands + bl];
        // T1[n] = G (2^e0 S0[n] + 2^e1 S1[n]), the half rows read one after the other; each scale applied
        // in two power-of-two factors
        float th[NP], tl[NP];  // half row 0, scaled, as float pairs
        {
          float d[32];  // d[8 g + n]: level accumulator g of state n
          tmem_ld8x4(tcol, tcol + kOpN, tcol + 2 * kOpN, tcol + 3 * kOpN, d);
          const float ga = G * oz_pow2(e0 >> 1), gb = oz_pow2(e0 - (e0 >> 1));
#pragma unroll
          for (int n = 0; n < NP; n++) {
            float sh, c0, c1;
            oz_two_sum(d[n], d[8 + n], sh, c0);
            oz_two_sum(sh, d[16 + n], sh, c1);
            th[n] = __fmul_rn(__fmul_rn(sh, ga), gb);
            tl[n] = __fmul_rn(__fmul_rn(__fadd_rn(__fadd_rn(c0, c1), d[24 + n]), ga), gb);
          }
        }
        ff t1[NP];
        if (nhalf > 1) {
          float d[32];
          tmem_ld8x4(tcol + 4 * kOpN, tcol + 5 * kOpN, tcol + 6 * kOpN, tcol + 7 * kOpN, d);
          const float ga = G * oz_pow2(e1 >> 1), gb = oz_pow2(e1 - (e1 >> 1));
#pragma unroll
          for (int n = 0; n < NP; n++) {
            float sh, c0, c1;
            oz_two_sum(d[n], d[8 + n], sh, c0);
            oz_two_sum(sh, d[16 + n], sh, c1);
            const float h1 = __fmul_rn(__fmul_rn(sh, ga), gb);
            const float l1 = __fmul_rn(__fmul_rn(__fadd_rn(__fadd_rn(c0, c1), d[24 + n]), ga), gb);
            float hi, lo;
            oz_two_sum(th[n], h1, hi, lo);
            oz_two_sum(hi, __fadd_rn(lo, __fadd_rn(tl[n], l1)), t1[n].hi, t1[n].lo);  // the halves may cancel
          }
        } else {
#pragma unroll
          for (int n = 0; n < NP; n++) oz_two_sum(th[n], tl[n], t1[n].hi, t1[n].lo);
        }
        tc05_fence_before();
        um_mbar_arrive(ae(rs));  // the row slot's accumulators and frames may be refilled
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
    float* btab = reinterpret_cast<float*>(ws + L.btab);
    float* gpow = reinterpret_cast<float*>(ws + L.gpow);
    float2* tyff = reinterpret_cast<float2*>(ws + L.tyff);
    k_op_tables<NU><<<(unsigned)p.natoms, 128, 0, p.stream>>>(p.g, p.atoms, btab, gpow, tyff);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto kern = k_project_ozaki<NU>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OpSmem::bytes);
    if (e != cudaSuccess) return e;
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
