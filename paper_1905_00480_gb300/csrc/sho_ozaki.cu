// sho_ozaki.cu -- FP64-accurate expansion (SHO_P_FF64) with the x-pass on the fifth-generation tensor
// cores, by exact digit slicing of both operands.
//
//   psi[z][y][x][b] += sum_a sum_nx T1_a[y][b][nx] phi^a_nx(x)          (Sec. 3.2 step 3; eq. TuckerTensor)
//
// T1_a comes from the float-float y-pass of the FP64 z-pass result; the x-pass is, per grid row, a
// product of a (bands x states) and a (states x points) matrix summed over the atoms.  On GB300 the FP64
// pipe is slow and a float-float x-pass costs ten FP32 instructions per (atom, point, band, state), so
// here the x-pass runs on the tensor cores with the splitting of Ozaki, Ogita, Oishi and Rump ("Error-free
// transformations of matrix multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012), in the fixed-point form:
//   * per (row, band) a power of two F above every covering atom's max_nx |T1_a[nx]| G_a (bounded ahead of
//     the y-pass: an FP32 y-pass over all rows of each (atom, plane, band) with an error term), and per
//     atom a power of two G_a above max |phi^a|;
//   * T1_a[nx] G_a / F = sum_{i=1..6} d_i and phi^a_nx(x) / G_a = sum_{j=1..6} e_j, where d_i, e_j are
//     signed integers times 2^(-8 i), 2^(-8 j) (round-to-nearest digits; at most 256 in magnitude for the
//     first digit, 128 for the others, 256 for d_4 which also takes the low float of T1);
//   * every product d_i e_j is an integer of at most 2^16 times 2^(-8 (i + j)), exact in the tensor
//     core's FP32 products.  Products of level L = i + j = 2, 3, 4 go to one accumulator per level, where
//     their sums stay integers below 2^24 and so are exact (at most 204 / (numax + 1) atoms per tile);
//     levels 5 .. 8 share a fourth accumulator and round at 2^-24 of a term that is 2^-24 below the
//     leading one; levels above 8 are dropped (below 2^-56 F per product);
//   * the point's update is F (D_2 + D_3 + D_4 + D_5..8), summed as a float pair and added to psi in FP64.
// The operands are TF32 (digits of at most 9 significant bits are exact in TF32), K = 8 states.
//
// Persistent kernel, two CTAs per SM walking the tiles (one grid row x 32 x points x 128 bands) in a
// fixed stride, with the work of a tile split over four warp roles that meet on mbarriers only:
//   * a list warp writes each tile's record two tiles ahead: the plane's atoms whose cube meets the tile
//     (ascending), their y function values at the row and G_a exponents, the frame exponent of every band,
//     and the tile's psi prefetched to L2;
//   * four digit warps, one thread per band: per atom the float-float y-pass on the band's T2 slice (float
//     pairs, loaded one atom ahead), T1 cut into six digit slices written as the A operands of the atom's
//     slot (two slots by atom parity), then an arrival on the slot's operand barrier;
//   * one MMA thread: per atom the next atom's x digit window staged by bulk copies into a ring of three
//     (one atom ahead), then, once the A operands and the window are in, 26 digit-pair MMAs (M = 128 bands,
//     N = 32 points, K = 8) into the tile's four level accumulators in tensor memory, committed to the
//     slot's barrier; after the tile's last atom a commit marks its accumulators complete;
//   * four read-back warps, one thread per band: the tile's accumulators read from tensor memory, summed
//     as a float pair, scaled by the frame and added to psi in FP64.
// Two accumulator sets (2 x 4 x 32 = 256 columns) let the read-back of tile k run while the MMAs of tile
// k + 1 accumulate.  Deterministic: fixed atom order, exact integer sums in the leading levels, each tile
// computed by one CTA whatever the schedule.  Every wait is bounded; the first one that runs out stops
// every role (a shared flag), the kernel records kStatusTimeout, waits (bounded) for its own copies and
// MMAs, frees tensor memory and returns; tiles read back before that hold their update, the others none.
#include <algorithm>

#include "sho_device.cuh"
#include "sho_ff.cuh"
#include "sho_umma.cuh"
#include "sho_oz.cuh"

namespace sho {

constexpr int kOzX = 32;                             // x points per tile (the MMA N)
constexpr int kOzBands = 128;                        // bands per tile (the MMA M), one thread each
constexpr int kOzWarps = 10;                         // 4 digit warps, 4 read-back warps, a list warp, an MMA warp
constexpr int kOzAllThreads = kOzWarps * 32;
constexpr int kOzListWarp = 8, kOzMmaWarp = 9;
constexpr int kOzDigits = 6;                         // digits per operand value
constexpr int kOzMaxLevel = 8;                       // digit pairs (i, j) with i + j <= 8 are multiplied
constexpr int kOzGroups = 4;                         // accumulators: levels 2, 3, 4 and 5..8
constexpr int kOzBufCols = kOzGroups * kOzX;         // tensor-memory columns of one tile's accumulators: 128
constexpr int kOzCols = 2 * kOzBufCols;              // two tiles in flight: 256
constexpr int kOzTabRows = 96;                       // rows of a digit table: cube point ix = row - 32
constexpr uint32_t kOzA = kOzBands * 8 * 4;          // one A digit slice [128 bands][8 states] TF32: 4 KB
constexpr uint32_t kOzAChunk = kOzBands * 16;        // its states 4..7 (the second core matrix along K)
constexpr uint32_t kOzB = kOzX * 8 * 4;              // one B digit slice [32 points][8 states]: 1 KB
constexpr uint32_t kOzBChunk = kOzX * 16;            // its states 4..7
constexpr int kOzTabFloats = kOzDigits * 2 * kOzTabRows * 4;  // digit table of one atom
constexpr int kOzBBuf = 3;                           // digit-window buffers (staged one atom ahead)

// Atoms per tile that keep the levels 2..4 exact: the level-4 products (first digits up to 256, the others
// up to 128) are at most 2 * 2^15 + 2^14 per state and atom, so (numax + 1) states x atoms x 2.5 * 2^15 <= 2^24.
__host__ __device__ constexpr int oz_max_atoms(int numax) { return 2048 / (10 * (numax + 1)); }

template <int NU>
struct OzSmem {
  static constexpr int NP = NU + 1, P = Basis<NU>::P;
  static constexpr size_t kA = (size_t)kOzDigits * kOzA;  // A slices of one operand slot: 24 KB
  static constexpr size_t kBs = (size_t)kOzDigits * kOzB;  // one digit window: 6 KB
  // Per-tile list record (two, by tile parity): header (atom count, or -1 after the last tile; z, y, x0 of
  // the tile; first band), the frame exponent of each band [128], the listed atoms (atom, cube row, cube x
  // offset, cube plane) [max_plane], their y function values [max_plane][NP] float pairs and the exponents
  // of their G_a [max_plane].
  __host__ __device__ static size_t rec_bytes(int mp) {
    return ((size_t)32 + 4 * kOzBands + 16 * (size_t)mp + 8 * (size_t)NP * mp + 4 * (size_t)mp + 15) & ~(size_t)15;
  }
  __host__ __device__ static size_t off_b() { return 2 * kA; }
  __host__ __device__ static size_t off_rec(int mp, int u) { return 2 * kA + kOzBBuf * kBs + (size_t)u * rec_bytes(mp); }
  __host__ __device__ static size_t off_bar(int mp) { return (off_rec(mp, 2) + 127) & ~(size_t)127; }
  static size_t bytes(int mp) { return off_bar(mp) + 256; }  // barriers, tensor-memory slot, abort flag
};

// ------------------------------------------------------------------------------------- tables
// Blocks [0, A), one per atom: G_a = 2^e with max |phi_x| < 2^e, and the digit table of phi_x / G_a,
// [6 digits][2 chunks][96 rows][4 states] with row = ix + 32 and zeros outside the cube and above numax
// (from the FP64 tables [A][2][NP][C]).  The other blocks, one thread per (atom, plane, band): a bound of
// max_y max_nx |T1[nx](y)| from the float-pair T2 and y tables, T1 summed in FP32 from the leading floats
// plus 2^-20 sum |T2| |phi| for the dropped low parts and the FP32 rounding (at most (numax + 3) 2^-24 of
// that sum), rounded up.
template <int NU>
__global__ void __launch_bounds__(128) k_oz_tables(int natoms, int cube, int nbands, const double* __restrict__ tables,
                                                   const float2* __restrict__ t2, const float2* __restrict__ tyff,
                                                   float* __restrict__ dtab, float* __restrict__ gpow,
                                                   float* __restrict__ tmax) {
  using BS = Basis<NU>;
  constexpr int NP = NU + 1, P = BS::P;
  const int tid = threadIdx.x, C = cube;
  if ((int)blockIdx.x >= natoms) {
    const long long i = (long long)(blockIdx.x - natoms) * 128 + tid;
    if (i >= (long long)natoms * C * nbands) return;
    const long long az = i / nbands, b = i - az * nbands;
    const int a = (int)(az / C);
    float t[P];
#pragma unroll
    for (int p = 0; p < P; p++) t[p] = t2[(az * P + p) * nbands + b].x;
    const float2* ty = tyff + (size_t)a * NP * C;
    float m = 0.0f;
    for (int iy = 0; iy < C; iy++) {
      float w[NP];
#pragma unroll
      for (int n = 0; n < NP; n++) w[n] = __ldg(&ty[n * C + iy].x);
#pragma unroll
      for (int nx = 0; nx < NP; nx++) {
        float s = 0.0f, e = 0.0f;
#pragma unroll
        for (int ny = 0; nx + ny <= NU; ny++) {
          s = fmaf(t[BS::pair(nx, ny)], w[ny], s);
          e = fmaf(fabsf(t[BS::pair(nx, ny)]), fabsf(w[ny]), e);
        }
        m = fmaxf(m, fmaf(e, 0x1p-20f, fabsf(s)));
      }
    }
    tmax[i] = m * (1.0f + 0x1p-20f);
    return;
  }
  __shared__ double red[4];
  const int a = blockIdx.x;
  const double* tx = tables + (size_t)a * 2 * NP * C;
  double m = 0.0;
  for (int i = tid; i < NP * C; i += 128) m = fmax(m, fabs(tx[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) red[tid >> 5] = m;
  __syncthreads();
  m = fmax(fmax(red[0], red[1]), fmax(red[2], red[3]));
  int e = 0;
  if (m > 0.0) (void)frexp(m, &e);  // m < 2^e
  const double G = m > 0.0 ? ldexp(1.0, e) : 1.0;
  if (tid == 0) gpow[a] = (float)G;
  // one (chunk, row, state) entry per iteration, its six digits in one pass: v = phi / G (exact: a power of
  // two), d_j = rint(v 2^(8j)) 2^(-8j), v -= d_j; every step is exact in FP64
  float* dt = dtab + (size_t)a * kOzTabFloats;
  const double ginv = 1.0 / G;
  for (int idx = tid; idx < 2 * kOzTabRows * 4; idx += 128) {
    const int q = idx & 3, row = (idx >> 2) % kOzTabRows, c = idx / (4 * kOzTabRows);
    const int n = 4 * c + q, ix = row - 32;
    double v = (n < NP && ix >= 0 && ix < C) ? tx[(size_t)n * C + ix] * ginv : 0.0;  // |v| < 1
    double sc = 1.0, isc = 1.0;
#pragma unroll
    for (int j = 0; j < kOzDigits; j++) {
      sc *= 256.0;
      isc *= 0.00390625;
      const double d = rint(v * sc) * isc;
      v -= d;
      dt[(size_t)j * 2 * kOzTabRows * 4 + idx] = (float)d;  // at most 256 (then 128) times 2^(-8 (j + 1))
    }
  }
}

// ------------------------------------------------------------------------------------- expansion
// BLOCH: complex coefficients and psi of a Bloch wave (Sec. 2.5), (re, im) pairs as two real bands in
// neighbouring lanes; each (atom, tile) T1 turns by the phase of the translation of the tile's points
// (one run: the tile segment does not cross the cell boundary) before its digit slicing, and the frames
// bound the turned values (the sum of the pair's bounds).
template <int NU, bool BLOCH = false>
__global__ void __launch_bounds__(kOzAllThreads, 2)
    k_expand_ozaki(GridDev g, const AtomDev* __restrict__ atoms, const int* __restrict__ plane_ptr,
                   const int* __restrict__ plane_atoms, int max_plane, const float2* __restrict__ tyff,
                   const float2* __restrict__ t2, const float* __restrict__ dtab, const float* __restrict__ gpow,
                   const float* __restrict__ tmax, double* __restrict__ psi, int* __restrict__ status,
                   long long wait_cycles, int stop_stage, const BlochPh* __restrict__ bph) {
  using BS = Basis<NU>;
  using SM = OzSmem<NU>;
  constexpr int NP = SM::NP, P = SM::P;
  static_assert(NP <= 8, "a digit slice holds at most 8 states");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int C = g.cube, Nx = g.n[0], Ny = g.n[1], Nz = g.n[2], B = g.nbands;
  const int mp = max_plane;
  const uint32_t sbase = um_smem(smem_raw);
  const uint32_t sB = sbase + (uint32_t)SM::off_b();
  unsigned char* barp = smem_raw + SM::off_bar(mp);
  const uint32_t bar0 = um_smem(barp);
  auto mf = [&](int u) { return bar0 + 8 * u; };        // list record u written (32 arrivals)
  auto me = [&](int u) { return bar0 + 16 + 8 * u; };   // list record u read by the read-back threads (128)
  auto af = [&](int u) { return bar0 + 32 + 8 * u; };   // accumulators u complete (MMA commit)
  auto ae = [&](int u) { return bar0 + 48 + 8 * u; };   // accumulators u read back (128 arrivals)
  auto fb = [&](int s) { return bar0 + 64 + 8 * s; };   // A operands of slot s written (128 arrivals)
  auto cb = [&](int s) { return bar0 + 80 + 8 * s; };   // MMAs from slot s done (MMA commit)
  auto bb = [&](int q) { return bar0 + 96 + 8 * q; };   // digit window q staged (bulk copies)
  const uint32_t dr = bar0 + 120;                       // drain: every MMA of this CTA done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(barp + 128);
  volatile int* s_abort = reinterpret_cast<volatile int*>(barp + 132);
  auto rec = [&](int u) { return smem_raw + SM::off_rec(mp, u); };
  auto rec_hdr = [&](int u) { return reinterpret_cast<int*>(rec(u)); };
  auto rec_ef = [&](int u) { return reinterpret_cast<int*>(rec(u) + 32); };
  auto rec_list = [&](int u) { return reinterpret_cast<int4*>(rec(u) + 32 + 4 * kOzBands); };
  auto rec_y = [&](int u) { return reinterpret_cast<float2*>(rec(u) + 32 + 4 * kOzBands + 16 * (size_t)mp); };
  auto rec_gexp = [&](int u) {
    return reinterpret_cast<int*>(rec(u) + 32 + 4 * kOzBands + 16 * (size_t)mp + 8 * (size_t)NP * mp);
  };
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nseg = (Nx + kOzX - 1) / kOzX, nbt = (B + kOzBands - 1) / kOzBands;
  const int ntiles = nseg * Ny * Nz;  // one grid row x 32 x points each, for every band tile

  if (tid == 0) {
    *s_abort = 0;
    for (int u = 0; u < 2; u++) {
      um_mbar_init_n(mf(u), 32);
      um_mbar_init_n(me(u), kOzBands);
      um_mbar_init(af(u));
      um_mbar_init_n(ae(u), kOzBands);
      um_mbar_init_n(fb(u), kOzBands);
      um_mbar_init(cb(u));
    }
    for (int q = 0; q < kOzBBuf; q++) um_mbar_init(bb(q));
    um_mbar_init(dr);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) tmem_alloc(um_smem(tmem_slot), kOzCols);
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

  if (warp == kOzListWarp) {
    // ---- list warp: the record of each of this CTA's tiles that a cube meets, two tiles ahead of the
    // read-back: its atoms (ascending), their y values at the tile's row and G_a exponents, the frame
    // exponent of every band, and the tile's psi to L2
    int cursor = blockIdx.x;
    for (int k = 0;; k++) {
      const int u = k & 1;
      // record u is free once the read-back of tile k - 2 has taken what it needs
      const bool ok = k < 2 || wait(me(u), (uint32_t)(((k - 2) >> 1) & 1));
      if (!__all_sync(0xffffffffu, ok)) break;
      int4* sl = rec_list(u);
      int nl = 0, z = 0, y = 0, xs = 0, bt = 0;
      while (cursor < ntiles * nbt) {
        const int t = cursor % ntiles;
        bt = cursor / ntiles;
        cursor += gridDim.x;
        const int seg = t % nseg, yz = t / nseg;
        y = yz % Ny;
        z = yz / Ny;
        xs = seg * kOzX;
        const int q0 = plane_ptr[z], q1 = plane_ptr[z + 1];
        nl = 0;
        for (int base = q0; base < q1; base += 32) {
          const int q = base + lane;
          int4 r = make_int4(-1, 0, 0, 0);
          bool m = false;
          if (q < q1) {
            const int a = plane_atoms[q];
            const AtomDev at = atoms[a];
            int dy = y - at.o[1], dx = xs - at.o[0], dz = z - at.o[2];
            if (g.periodic) {
              dy %= Ny;
              if (dy < 0) dy += Ny;
              dx %= Nx;
              if (dx < 0) dx += Nx;
              dz %= Nz;
              if (dz < 0) dz += Nz;
              m = dy < C && (dx < C || dx + kOzX > Nx);
              if (dx >= C) dx -= Nx;  // the cube starts inside the tile (one run: Nx >= C + 32)
            } else {
              m = dy >= 0 && dy < C && dx < C && dx + kOzX > 0;
            }
            r = make_int4(a, dy, dx, dz);
          }
          const unsigned bal = __ballot_sync(0xffffffffu, m);
          if (m) sl[nl + __popc(bal & ((1u << lane) - 1u))] = r;
          nl += __popc(bal);
        }
        if (nl > 0) break;
      }
      int* hdr = rec_hdr(u);
      if (nl == 0) {  // no tile left: the end marker
        if (lane == 0) hdr[0] = -1;
        __syncwarp();
        um_mbar_arrive(mf(u));
        break;
      }
      const int b0 = bt * kOzBands, nb = min(kOzBands, B - b0);
      __syncwarp();  // the list entries written above are read by every lane below
      float2* yl = rec_y(u);
      for (int i = lane; i < nl * NP; i += 32) {
        const int li = i / NP, n = i - li * NP;
        const int4 r = sl[li];
        yl[i] = tyff[((size_t)r.x * NP + n) * C + r.y];
      }
      int* ge = rec_gexp(u);
      for (int li = lane; li < nl; li += 32) ge[li] = (int)((__float_as_uint(gpow[sl[li].x]) >> 23) & 0xffu) - 127;
      {
        const double* pp = psi + (((size_t)z * Ny + y) * Nx + xs + lane) * (size_t)B + b0;
        if (xs + lane < Nx) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(pp), "r"((uint32_t)(nb * 8)) : "memory");
      }
      // the frame of each band: a power of two above every listed atom's bound |T1_a| G_a
      float xb[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 2
      for (int li = 0; li < nl; li++) {
        const int4 r = sl[li];
        const float ga = gpow[r.x];
        const float* tm = tmax + ((size_t)r.x * C + r.w) * B + b0;
#pragma unroll
        for (int c = 0; c < 4; c++) {
          const int bi = lane + 32 * c;
          if (bi < nb) xb[c] = fmaxf(xb[c], (BLOCH ? tm[bi] + tm[bi ^ 1] : tm[bi]) * ga);
        }
      }
      int* ef = rec_ef(u);
      bool range_bad = false;
#pragma unroll
      for (int c = 0; c < 4; c++) {
        int eF = 0;
        if (xb[c] > 0.0f) eF = (int)((__float_as_uint(xb[c] * (1.0f + 0x1p-20f)) >> 23) & 0xffu) - 127 + 1;  // xb < 2^eF
        range_bad |= eF > 127;  // the bound overflowed the float range
        ef[lane + 32 * c] = max(-124, min(eF, 127));
      }
      if (range_bad && status) atomicOr(status, kStatusRange);
      if (lane == 0) {
        hdr[0] = nl;
        hdr[1] = z;
        hdr[2] = y;
        hdr[3] = xs;
        hdr[4] = b0;
        hdr[5] = nb;
      }
      __syncwarp();
      um_mbar_arrive(mf(u));
    }
  } else if (warp == kOzMmaWarp) {
    // ---- MMA thread: per tile, once its accumulators are free (read back two tiles ago), per atom: the
    // next atom's digit window staged into the ring (one atom ahead; stop_stage < the tile's atom count
    // only under fault injection: windows from that atom on are never staged, so the wait runs out), the
    // A operands and this atom's window awaited, 26 digit-pair MMAs issued and committed to the slot
    if (lane == 0) {
      constexpr uint32_t idesc = umma_idesc(kUmmaTF32, kOzBands, kOzX);
      const uint64_t ad0 = umma_desc(sbase, kOzAChunk, 128), bd0 = umma_desc(sB, kOzBChunk, 128);
      int gi = 0;          // atoms of this CTA so far: slot gi & 1, window buffer gi % 3
      int staged = 0;      // windows staged (by CTA atom index)
      int consumed = 0;    // windows waited for
      bool any = false;    // an MMA was issued
      auto stage = [&](const int4 r, int ga) {
        const int q = ga % kOzBBuf;
        const uint32_t dst = sB + (uint32_t)(q * SM::kBs);
        const float* src = dtab + (size_t)r.x * kOzTabFloats + (size_t)(r.z + 32) * 4;  // rows r.z + 32 ..
        fence_async_smem();  // the buffer's earlier use (by the tensor core, completed) comes before the copies
        um_expect_tx(bb(q), (uint32_t)SM::kBs);
#pragma unroll
        for (int jc = 0; jc < 2 * kOzDigits; jc++)
          um_bulk(dst + (uint32_t)(jc * kOzBChunk), src + (size_t)jc * kOzTabRows * 4, kOzBChunk, bb(q));
        staged = ga + 1;
      };
      for (int k = 0;; k++) {
        const int u = k & 1;
        if (!wait(mf(u), (uint32_t)((k >> 1) & 1))) break;
        const int nl = rec_hdr(u)[0];
        if (nl < 0) break;
        if (k >= 2 && !wait(ae(u), (uint32_t)(((k - 2) >> 1) & 1))) break;
        tc05_fence_after();
        const int4* sl = rec_list(u);
        const uint32_t dacc = tmem + (uint32_t)(u * kOzBufCols);
        if (stop_stage > 0) stage(sl[0], gi);
        bool ok = true;
        for (int li = 0; li < nl && ok; li++) {
          const int ga = gi + li, slot = ga & 1, q = ga % kOzBBuf;
          // slot ga & 1 and window buffer (ga + 1) % 3 free: the MMAs of atom ga - 2 are done
          if (ga >= 2 && !wait(cb(slot), (uint32_t)(((ga - 2) >> 1) & 1))) { ok = false; break; }
          if (li + 1 < nl && li + 1 < stop_stage) stage(sl[li + 1], ga + 1);
          if (!wait(fb(slot), (uint32_t)((ga >> 1) & 1))) { ok = false; break; }
          if (!wait(bb(q), (uint32_t)((ga / kOzBBuf) & 1))) { ok = false; break; }
          consumed = ga + 1;
          tc05_fence_after();
          const uint64_t ad = ad0 + (uint64_t)((slot * SM::kA) >> 4), bd = bd0 + (uint64_t)((q * SM::kBs) >> 4);
#pragma unroll
          for (int i = 1; i <= kOzDigits; i++)
#pragma unroll
            for (int j = 1; j <= kOzDigits; j++) {
              if (i + j > kOzMaxLevel) continue;
              const int grp = (i + j < 5 ? i + j : 5) - 2;
              // the first product of each level group in the tile starts its accumulator
              const bool acc = li > 0 || !(i == 1 && j <= 4);
              umma_tf32(dacc + (uint32_t)(grp * kOzX), ad + (uint64_t)(((i - 1) * kOzA) >> 4),
                        bd + (uint64_t)(((j - 1) * kOzB) >> 4), idesc, acc);
            }
          umma_commit(cb(slot));
          any = true;
        }
        if (!ok) break;
        umma_commit(af(u));  // the tile's accumulators are complete once its MMAs are
        gi += nl;
      }
      // windows staged and not waited for (at most two) complete whatever else happens; every MMA issued
      // completes before the tensor memory is released
      for (int q = consumed; q < staged; q++)
        (void)um_mbar_wait(bb(q % kOzBBuf), (uint32_t)((q / kOzBBuf) & 1), kDefaultWaitCycles);
      if (any) {
        umma_commit(dr);
        (void)um_mbar_wait(dr, 0, kDefaultWaitCycles);
      }
    }
    __syncwarp();
  } else if (warp < 4) {
    // ---- digit threads, one per band: per atom the float-float y-pass of the tile row and its six digit
    // slices as the A operands of the atom's slot, once the slot's MMAs of atom gi - 2 are done
    const int bl = tid;
    int gi = 0;
    float2 tv[P];  // T2 of the current atom for this thread's band (float pairs), loaded one atom ahead
    for (int k = 0;; k++) {
      const int u = k & 1;
      if (!wait(mf(u), (uint32_t)((k >> 1) & 1))) break;
      const int* hdr = rec_hdr(u);
      const int nl = hdr[0];
      if (nl < 0) break;
      const int b0 = hdr[4], nb = hdr[5];
      const bool bvalid = bl < nb;
      const int b = b0 + bl;
      const int eF = rec_ef(u)[bl];
      const int4* sl = rec_list(u);
      const float2* yl = rec_y(u);
      const int* ge = rec_gexp(u);
      auto load_t2 = [&](int li) {
        if (!bvalid) return;
        const int4 r = sl[li];
        const float2* src = t2 + ((size_t)r.x * C + r.w) * P * B + b;
#pragma unroll
        for (int p = 0; p < P; p++) tv[p] = src[(size_t)p * B];
      };
      load_t2(0);
      bool ok = true;
      for (int li = 0; li < nl; li++) {
        const int ga = gi + li, slot = ga & 1;
        // the whole warp leaves together (the Bloch turn below exchanges values between lanes)
        const bool free_slot = ga < 2 || wait(cb(slot), (uint32_t)(((ga - 2) >> 1) & 1));
        if (!__all_sync(0xffffffffu, free_slot)) {
          ok = false;
          break;
        }
        float ys[NP], yc[NP];
#pragma unroll
        for (int n = 0; n < NP; n++) ys[n] = yc[n] = 0.0f;
        if (bvalid) {
          const float2* yv = yl + li * NP;
#pragma unroll
          for (int ny = 0; ny < NP; ny++) {
            const float2 w = yv[ny];
#pragma unroll
            for (int nx = 0; nx + ny <= NU; nx++)
              ff_dot_step(ys[nx], yc[nx], ff{tv[BS::pair(nx, ny)].x, tv[BS::pair(nx, ny)].y}, ff{w.x, w.y});
          }
        }
        if (li + 1 < nl) load_t2(li + 1);  // in flight during the digits and the next wait
        if constexpr (BLOCH) {
          // T1 turned by the phase of the translation of the tile's points (every lane of the warp)
          const int4 r = sl[li];
          const BlochPh& bp = bph[r.x];
          const float4 ph = bp.ph[(max(r.z, 0) >= bp.w[0] ? 1 : 0) + (r.y >= bp.w[1] ? 2 : 0) + (r.w >= bp.w[2] ? 4 : 0)];
          if (!ff_is_one(ph)) {
#pragma unroll
            for (int n = 0; n < NP; n++) {
              const ff v = ff_rotate(ff_norm(ys[n], yc[n]), ph, lane);
              ys[n] = v.hi;
              yc[n] = v.lo;
            }
          }
        }
        // six digit slices of T1 G_a / F, written as the A operands (two chunks of four states)
        const int kk = ge[li] - eF;  // G_a / F = 2^kk
        const float sa = (kk < -126 || !bvalid) ? 0.0f : oz_pow2(min(kk, 127));
        unsigned char* arow = smem_raw + (size_t)slot * SM::kA + (size_t)bl * 16;
#pragma unroll
        for (int c = 0; c < 2; c++) {
          float dg[kOzDigits][4];
#pragma unroll
          for (int q = 0; q < 4; q++) {
            const int n = 4 * c + q;
            if (n < NP) {
              const ff tt = ff_norm(ys[n], yc[n]);
              float rem = __fmul_rn(tt.hi, sa);  // |rem| < 1
              const float lo = __fmul_rn(tt.lo, sa);
              dg[0][q] = oz_digit(rem, 0x1.8p+15f);  // grid 2^-8
              dg[1][q] = oz_digit(rem, 0x1.8p+7f);   // grid 2^-16
              dg[2][q] = oz_digit(rem, 0x1.8p-1f);   // grid 2^-24: what is left of hi lies below it
              rem = __fadd_rn(rem, lo);
              dg[3][q] = oz_digit(rem, 0x1.8p-9f);   // grid 2^-32
              dg[4][q] = oz_digit(rem, 0x1.8p-17f);  // grid 2^-40
              dg[5][q] = oz_digit(rem, 0x1.8p-25f);  // grid 2^-48
            } else {
#pragma unroll
              for (int i = 0; i < kOzDigits; i++) dg[i][q] = 0.0f;
            }
          }
#pragma unroll
          for (int i = 0; i < kOzDigits; i++)
            *reinterpret_cast<float4*>(arow + i * kOzA + c * kOzAChunk) = make_float4(dg[i][0], dg[i][1], dg[i][2], dg[i][3]);
        }
        fence_async_smem();  // the A slices become visible to the tensor core
        um_mbar_arrive(fb(slot));
      }
      if (!ok) break;
      gi += nl;
    }
  } else {
    // ---- read-back threads, one per band (tensor-memory lanes 32 (warp - 4) ..): per tile, the four
    // level accumulators of the 32 points summed as a float pair, scaled by the frame and added to psi in
    // FP64; then the accumulators are free for tile k + 2
    const int bl = tid - 128;
    const uint32_t tlane = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    for (int k = 0;; k++) {
      const int u = k & 1;
      if (!wait(mf(u), (uint32_t)((k >> 1) & 1))) break;
      const int* hdr = rec_hdr(u);
      const int nl = hdr[0];
      if (nl < 0) break;
      const int z = hdr[1], y = hdr[2], xs = hdr[3], b0 = hdr[4], nb = hdr[5];
      const float F = oz_pow2(rec_ef(u)[bl]);
      const bool wr = bl < nb;
      const int xend = min(kOzX, Nx - xs);
      double* rowp = psi + (((size_t)z * Ny + y) * Nx + xs) * (size_t)B + b0 + bl;
      double pv[8];  // the current batch of 8 points, the next batch's loads issued before its adds
#pragma unroll
      for (int x = 0; x < 8; x++) pv[x] = (wr && x < xend) ? rowp[(size_t)x * B] : 0.0;
      if (!wait(af(u), (uint32_t)((k >> 1) & 1))) break;
      um_mbar_arrive(me(u));  // the record is no longer needed: the list warp may refill it
      tc05_fence_after();
      const uint32_t tcol = tlane + (uint32_t)(u * kOzBufCols);
#pragma unroll 1
      for (int x0 = 0; x0 < kOzX; x0 += 8) {
        float d[32];  // d[8 g + x]: level accumulator g of point x0 + x
        tmem_ld8x4(tcol + (uint32_t)x0, tcol + (uint32_t)(kOzX + x0), tcol + (uint32_t)(2 * kOzX + x0),
                   tcol + (uint32_t)(3 * kOzX + x0), d);
        double pn[8];
#pragma unroll
        for (int x = 0; x < 8; x++) pn[x] = (wr && x0 + 8 + x < xend) ? rowp[(size_t)(x0 + 8 + x) * B] : 0.0;
        if (wr) {
#pragma unroll
          for (int x = 0; x < 8; x++) {
            if (x0 + x < xend) {
              float s, e1, e2;
              oz_two_sum(d[x], d[8 + x], s, e1);
              oz_two_sum(s, d[16 + x], s, e2);
              const float c = __fadd_rn(__fadd_rn(e1, e2), d[24 + x]);
              rowp[(size_t)(x0 + x) * B] = pv[x] + ff_to_double(__fmul_rn(s, F), __fmul_rn(c, F));
            }
          }
        }
#pragma unroll
        for (int x = 0; x < 8; x++) pv[x] = pn[x];
      }
      tc05_fence_before();
      um_mbar_arrive(ae(u));
    }
  }
  __syncthreads();
  if (tid == 0 && *s_abort && status) atomicOr(status, kStatusTimeout);
  tc05_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kOzCols);
}

// The kernel's MMA schedule on host digits: A [6][128][8] and B [6][32][8] (digit values), D [4][128][32]
// the four level accumulators (test of the operand layouts and of the exactness of the level sums).
__global__ void __launch_bounds__(128) k_oz_selftest(const float* __restrict__ A, const float* __restrict__ Bm,
                                                     float* __restrict__ D, int* __restrict__ status) {
  __shared__ __align__(1024) unsigned char sm[kOzDigits * kOzA + kOzDigits * kOzB];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < kOzDigits * kOzBands * 8; i += 128) {
    const int s = i / (kOzBands * 8), m = (i / 8) % kOzBands, k = i % 8;
    *reinterpret_cast<float*>(sm + s * kOzA + (k / 4) * kOzAChunk + m * 16 + (k % 4) * 4) = A[i];
  }
  for (int i = tid; i < kOzDigits * kOzX * 8; i += 128) {
    const int s = i / (kOzX * 8), n = (i / 8) % kOzX, k = i % 8;
    *reinterpret_cast<float*>(sm + kOzDigits * kOzA + s * kOzB + (k / 4) * kOzBChunk + n * 16 + (k % 4) * 4) = Bm[i];
  }
  if (warp == 0) tmem_alloc(um_smem(&tslot), kOzGroups * kOzX);
  if (tid == 0) {
    um_mbar_init(um_smem(&bar));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  fence_async_smem();
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  const uint32_t tmem = tslot;
  const uint32_t tlane = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
  for (int c = 0; c < kOzGroups; c++) tmem_zero32(tlane + (uint32_t)(32 * c));
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  if (tid == 0) {
    constexpr uint32_t idesc = umma_idesc(kUmmaTF32, kOzBands, kOzX);
    const uint32_t sa = um_smem(sm), sb = sa + kOzDigits * kOzA;
    for (int i = 1; i <= kOzDigits; i++)
      for (int j = 1; j <= kOzDigits; j++) {
        if (i + j > kOzMaxLevel) continue;
        const int grp = (i + j < 5 ? i + j : 5) - 2;
        umma_tf32(tmem + (uint32_t)(grp * kOzX), umma_desc(sa + (uint32_t)((i - 1) * kOzA), kOzAChunk, 128),
                  umma_desc(sb + (uint32_t)((j - 1) * kOzB), kOzBChunk, 128), idesc, true);
      }
    umma_commit(um_smem(&bar));
  }
  const bool done = um_mbar_wait(um_smem(&bar), 0, 2000000000ll);
  if (!done && tid == 0) atomicOr(status, kStatusTimeout);
  if (!done) (void)um_mbar_wait(um_smem(&bar), 0, kDefaultWaitCycles);
  tc05_fence_after();
  for (int c = 0; c < kOzGroups; c++) {
    float v[32];
    tmem_ld32(tlane + (uint32_t)(32 * c), v);
#pragma unroll
    for (int x = 0; x < 32; x++) D[((size_t)c * kOzBands + 32 * warp + lane) * kOzX + x] = done ? v[x] : 0.0f;
  }
  tc05_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kOzGroups * kOzX);
}

// ------------------------------------------------------------------------------------ launchers
template <int NU>
static cudaError_t ozaki_nu(const ExpandLaunch& p, const void* tyff) {
  if constexpr (NU > 7) {
    return cudaErrorNotSupported;
  } else {
    const OzLayout L = oz_layout(p.natoms, p.g.cube, p.g.nbands);
    char* ws = static_cast<char*>(p.oz);
    float* dtab = reinterpret_cast<float*>(ws + L.dtab);
    float* gpow = reinterpret_cast<float*>(ws + L.gpow);
    float* tmax = reinterpret_cast<float*>(ws + L.tmax);
    const long long nbound = (long long)p.natoms * p.g.cube * p.g.nbands;
    k_oz_tables<NU><<<(unsigned)(p.natoms + (nbound + 127) / 128), 128, 0, p.stream>>>(
        p.natoms, p.g.cube, p.g.nbands, static_cast<const double*>(p.tables), static_cast<const float2*>(p.t2),
        static_cast<const float2*>(tyff), dtab, gpow, tmax);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = OzSmem<NU>::bytes(p.max_plane);
    auto kern = p.bloch ? k_expand_ozaki<NU, true> : k_expand_ozaki<NU, false>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // persistent: two CTAs per SM walk the tiles (grid row x 32 points x 128 bands) in a fixed stride
    const long long ntiles = (long long)((p.g.n[0] + kOzX - 1) / kOzX) * p.g.n[1] * p.g.n[2] *
                             ((p.g.nbands + kOzBands - 1) / kOzBands);
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const unsigned nblk = (unsigned)std::min<long long>(ntiles, 2LL * sms);
    kern<<<nblk, kOzAllThreads, smem, p.stream>>>(
        p.g, p.atoms, p.plane_ptr, p.plane_atoms, p.max_plane, static_cast<const float2*>(tyff),
        static_cast<const float2*>(p.t2),
        dtab, gpow, tmax, static_cast<double*>(p.psi), p.status, p.wait_cycles, p.stop_stage, p.bloch);
    return cudaGetLastError();
  }
}

// The tensor-core form covers numax <= 7 (K = 8 states), cubes of at most 32 points (even), one run of
// cube points per tile row (a periodic grid of at least cube + 32 points along x), no spherical support,
// an even band count (16-byte rows of float pairs), at most oz_max_atoms(numax) atoms per plane, and the
// shared memory of one CTA.
bool ozaki_expand_ok(const ExpandLaunch& p) {
  if (!p.oz || p.numax > 7 || p.g.r2max > 0.0) return false;
  if (p.g.cube > 32 || (p.g.cube & 1) || (p.g.nbands & 1)) return false;
  if (p.g.periodic && p.g.n[0] < p.g.cube + kOzX) return false;
  if (p.max_plane > oz_max_atoms(p.numax)) return false;
  size_t smem = 0;
  switch (p.numax) {
    case 0: smem = OzSmem<0>::bytes(p.max_plane); break;
    case 1: smem = OzSmem<1>::bytes(p.max_plane); break;
    case 2: smem = OzSmem<2>::bytes(p.max_plane); break;
    case 3: smem = OzSmem<3>::bytes(p.max_plane); break;
    case 4: smem = OzSmem<4>::bytes(p.max_plane); break;
    case 5: smem = OzSmem<5>::bytes(p.max_plane); break;
    case 6: smem = OzSmem<6>::bytes(p.max_plane); break;
    default: smem = OzSmem<7>::bytes(p.max_plane); break;
  }
  return smem <= 227 * 1024;
}

cudaError_t launch_expand_ozaki(const ExpandLaunch& p, const void* tyff) {
  switch (p.numax) {
    case 0: return ozaki_nu<0>(p, tyff);
    case 1: return ozaki_nu<1>(p, tyff);
    case 2: return ozaki_nu<2>(p, tyff);
    case 3: return ozaki_nu<3>(p, tyff);
    case 4: return ozaki_nu<4>(p, tyff);
    case 5: return ozaki_nu<5>(p, tyff);
    case 6: return ozaki_nu<6>(p, tyff);
    case 7: return ozaki_nu<7>(p, tyff);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace sho

using namespace sho;

extern "C" int sho_selftest_ozaki(const float* A, const float* Bm, float* D) {
  if (!A || !Bm || !D) return SHO_ERR_ARG;
  const size_t na = (size_t)kOzDigits * kOzBands * 8, nbm = (size_t)kOzDigits * kOzX * 8;
  const size_t nd = (size_t)kOzGroups * kOzBands * kOzX;
  float *dA = nullptr, *dB = nullptr, *dD = nullptr;
  int* dst = nullptr;
  int st = SHO_OK;
  if (cudaMalloc(&dA, sizeof(float) * na) != cudaSuccess || cudaMalloc(&dB, sizeof(float) * nbm) != cudaSuccess ||
      cudaMalloc(&dD, sizeof(float) * nd) != cudaSuccess || cudaMalloc(&dst, sizeof(int)) != cudaSuccess) {
    st = SHO_ERR_OOM;
  } else if (cudaMemcpy(dA, A, sizeof(float) * na, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(dB, Bm, sizeof(float) * nbm, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemset(dst, 0, sizeof(int)) != cudaSuccess) {
    st = SHO_ERR_CUDA;
  } else {
    k_oz_selftest<<<1, 128>>>(dA, dB, dD, dst);
    int flag = 0;
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(D, dD, sizeof(float) * nd, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&flag, dst, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = SHO_ERR_CUDA;
    else if (flag)
      st = SHO_ERR_TIMEOUT;
  }
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dD);
  cudaFree(dst);
  cudaGetLastError();
  return st;
}
