// sho_umma_expand.cu -- FP32-class expansion with the x-pass on the fifth-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory), for the TF32, BF16, 3xTF32 and split-FP16 forms.
//
//   psi[z][y][x][b] += sum_a sum_nx T1_a[y][b][nx] phi_nx(x - X_a),   T1 from the y-pass of the z-pass
//   result T2 (Sec. 3.2 step 3, passes in the order z, y, x; eq. TuckerTensor, Sec. 3.4)
//
// A CTA owns a tile of one z plane: 8 grid rows (4 for the split forms) x 32 x points x 128 bands.  The
// tile's update lives in tensor memory for the whole atom loop: one accumulator per row (two for split
// FP16) of 128 lanes (bands) x 32 columns (x points).  For each atom whose cube meets the tile
// (ascending order):
//   * its band-tiled T2 slice (128 bands x pairs), y table and x table (both point-major) are staged in
//     shared memory by three bulk TMA copies issued by one thread, one atom ahead, completing on the
//     buffer's mbarrier;
//   * 256 threads run the y-pass (thread = band, half the rows each) and write T1 of every row as an MMA
//     A operand, [128 bands][8 states] TF32 (or [128][16] BF16 / FP16, states 8..15 zero), K-major
//     without swizzle, as a hi and a lo part for the split forms; the atom's x functions on the tile's 32
//     points become the B operand [32][8] (hi and lo);
//   * one thread issues the MMAs of every row, M=128, N=32: D[row] += A[row] B^T, and for the split forms
//     the two cross products A_hi B_lo + A_lo B_hi (into D[row] for 3xTF32, into a second accumulator
//     read back times 2^-11 for split FP16, Markidis et al. 2018; Ootomo & Yokota 2022), and commits them
//     to the operand slot's mbarrier; the next atom's y-pass writes the other slot meanwhile.
// At the end each warp reads its quarter of the lanes (tcgen05.ld) and adds the tile to psi in global
// memory once.  Atoms are added in ascending order: deterministic.  Every wait is bounded; on expiry the
// kernel records kStatusTimeout, waits (bounded) for its own MMAs and copies, frees tensor memory and
// returns.
#include "sho_tc.cuh"
#include "sho_umma.cuh"

namespace sho {

constexpr int kUmX = 32;         // x points per tile (the MMA N)
constexpr int kUmBands = 128;    // bands per tile (the MMA M)
constexpr int kUmThreads = 256;
constexpr int kUmKBytes = 32;    // bytes per operand row: 8 TF32 or 16 BF16 values

// Operand forms of the tensor-memory expansion (UM): TF32, BF16, and the split forms that restore about
// 22 operand bits with three products per row, 3xTF32 (hi and lo parts in TF32, all three products into
// one accumulator) and split FP16 (x = hi + 2^-11 lo', the hi*hi product into one accumulator and the
// two cross products into a second one, read back as main + 2^-11 cross).  The split forms keep a hi and
// a lo part of every operand and work on tiles of 4 rows, so an operand slot stays 32 KB.
constexpr int kUmTF32 = 0, kUmBF16 = 1, kUm3xTF32 = 2, kUmSplit16 = 3;
constexpr uint32_t kUmmaF16 = 0;  // instruction-descriptor operand type FP16 (kind::f16)
template <int UM>
struct UmMode {
  static constexpr bool split = UM >= kUm3xTF32;
  static constexpr bool h16 = UM == kUmBF16 || UM == kUmSplit16;  // 16-bit operands (K = 16, states 8..15 zero)
  static constexpr int rows = split ? 4 : 8;                     // grid rows per tile
  static constexpr int parts = split ? 2 : 1;                    // hi (and lo) operand parts
  static constexpr int nacc = UM == kUmSplit16 ? 2 : 1;          // accumulators per row
  static constexpr int cols = rows * kUmX * nacc;                // tensor-memory columns: 256 or 128
  static constexpr uint32_t ab = h16 ? (UM == kUmBF16 ? kUmmaBF16 : kUmmaF16) : kUmmaTF32;
};

template <int NU, int UM>
struct UmSmem {
  using MD = UmMode<UM>;
  static constexpr int NP = NU + 1, P = Basis<NU>::P, PP = tiled_pairs(P), NPX = (NP + 3) & ~3;
  static constexpr size_t kPart = (size_t)MD::rows * kUmBands * kUmKBytes;  // one operand part of A
  static constexpr size_t kA = MD::parts * kPart;                           // one A slot: 32 KB
  static constexpr size_t kBPart = (size_t)kUmX * kUmKBytes;
  static constexpr size_t kB = MD::parts * kBPart;                           // one B slot: 1 or 2 KB
  // staging buffer: T2 [128][PP] floats, y table [C][NPX], x table [C][NPX] (point-major)
  __host__ __device__ static size_t stage_floats(int cube) {
    return (size_t)kUmBands * PP + 2 * (size_t)cube * NPX;
  }
  __host__ __device__ static size_t off_b() { return 2 * kA; }
  __host__ __device__ static size_t off_stage() { return 2 * kA + 2 * kB; }
  __host__ __device__ static size_t off_bar(int cube) { return off_stage() + 2 * stage_floats(cube) * 4; }
  static size_t bytes(int cube, int max_plane) {
    return off_bar(cube) + 128 + (size_t)(max_plane + 1) * sizeof(int4);
  }
};

// The hi (and lo) operand values of x in the form's type, as the 32-bit words written to shared memory:
// TF32 bit patterns, or 16-bit values (BF16 / FP16) for pair packing.
template <int UM>
__device__ __forceinline__ void um_parts(float x, float& hi, float& lo) {
  if constexpr (UM == kUm3xTF32) {
    hi = __uint_as_float(tf32_bits(x));
    lo = __uint_as_float(tf32_bits(x - hi));
  } else if constexpr (UM == kUmSplit16) {
    f16_split(x, hi, lo);
  } else {
    hi = x;
    lo = 0.0f;
  }
}

// Four (TF32 forms: one 16-byte chunk of 4 states) or eight (16-bit forms) values as one K-major row piece.
template <int UM>
__device__ __forceinline__ uint4 um_pack4(const float* v) {
  if constexpr (UmMode<UM>::h16) {
    if constexpr (UM == kUmBF16)
      return make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    else
      return make_uint4(pack_f16(v[0], v[1]), pack_f16(v[2], v[3]), pack_f16(v[4], v[5]), pack_f16(v[6], v[7]));
  } else {
    return make_uint4(tf32_bits(v[0]), tf32_bits(v[1]), tf32_bits(v[2]), tf32_bits(v[3]));
  }
}

template <int NU, typename TP, int UM>
__global__ void __launch_bounds__(kUmThreads, 2)
    k_expand_umma(GridDev g, const AtomDev* __restrict__ atoms, const int* __restrict__ plane_ptr,
                  const int* __restrict__ plane_atoms, const float* __restrict__ tym,
                  const float* __restrict__ txm, const float* __restrict__ t2, TP* __restrict__ psi,
                  int* __restrict__ status, long long wait_cycles) {
  using BS = Basis<NU>;
  using SM = UmSmem<NU, UM>;
  using MD = UmMode<UM>;
  constexpr int NP = SM::NP, P = SM::P, PP = SM::PP, NPX = SM::NPX;
  constexpr int R = MD::rows;
  static_assert(NP <= 8, "one MMA covers at most 8 states");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int C = g.cube, Nx = g.n[0], Ny = g.n[1], Nz = g.n[2], B = g.nbands;
  const uint32_t sbase = um_smem(smem_raw);
  const uint32_t sA = sbase, sB = sbase + (uint32_t)SM::off_b();
  float* stage = reinterpret_cast<float*>(smem_raw + SM::off_stage());
  const size_t stf = SM::stage_floats(C);
  unsigned char* barp = smem_raw + SM::off_bar(C);
  const uint32_t bar0 = um_smem(barp);                      // commit barriers of operand slots 0 and 1
  const uint32_t fbar0 = bar0 + 16;                         // staging barriers of buffers 0 and 1
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(barp + 32);
  int* s_misc = reinterpret_cast<int*>(barp + 48);          // [0] list length, [1..8] warp counts
  int4* slist = reinterpret_cast<int4*>(barp + 128);        // after s_misc[0..8] (bytes 48..83)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const int nseg = (Nx + kUmX - 1) / kUmX, nyb = (Ny + R - 1) / R;
  int bid = blockIdx.x;
  const int seg = bid % nseg;
  bid /= nseg;
  const int yb = bid % nyb;
  const int z = bid / nyb;
  const int xs = seg * kUmX;
  const int nbt32 = (B + 31) / 32;                 // 32-band tiles of the band-tiled T2
  const int bt0 = blockIdx.y * 4;                  // first of this CTA's four
  const int ntile = min(4, nbt32 - bt0);
  const int q0 = plane_ptr[z], q1 = plane_ptr[z + 1];

  // atoms of the plane whose cube meets the tile, ascending (offsets as in the block gather)
  if (tid == 0) s_misc[0] = 0;
  __syncthreads();
  for (int base = q0; base < q1; base += kUmThreads) {
    const int q = base + tid;
    int4 r = make_int4(-1, 0, 0, 0);
    bool m = false;
    if (q < q1) {
      const int a = plane_atoms[q];
      const AtomDev at = atoms[a];
      int dy = yb * R - at.o[1], dx = xs - at.o[0], dz = z - at.o[2];
      if (g.periodic) {
        dy %= Ny;
        if (dy < 0) dy += Ny;
        dx %= Nx;
        if (dx < 0) dx += Nx;
        dz %= Nz;
        if (dz < 0) dz += Nz;
        m = (dy < C || dy + R > Ny) && (dx < C || dx + kUmX > Nx);
      } else {
        m = dy < C && dy + R > 0 && dx < C && dx + kUmX > 0;
      }
      r = make_int4(a, dy, dx, dz);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, m);
    if (lane == 0) s_misc[1 + warp] = __popc(bal);
    __syncthreads();
    int off = s_misc[0];
    for (int w = 0; w < warp; w++) off += s_misc[1 + w];
    if (m) slist[off + __popc(bal & ((1u << lane) - 1u))] = r;
    __syncthreads();
    if (tid == 0)
      for (int w = 0; w < kUmThreads / 32; w++) s_misc[0] += s_misc[1 + w];
    __syncthreads();
  }
  const int nlist = s_misc[0];
  if (nlist == 0) return;  // no cube meets the tile: psi is unchanged

  // tensor memory for the row accumulators, zeroed; commit barriers; the 16-bit operands' zero halves
  if (warp == 0) tmem_alloc(um_smem(tmem_slot), MD::cols);
  if (tid == 0) {
    um_mbar_init(bar0);
    um_mbar_init(bar0 + 8);
    um_mbar_init(fbar0);
    um_mbar_init(fbar0 + 8);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if constexpr (MD::h16) {
    // states 8..15 of every A and B row stay zero: the second 16 bytes of each row, in every part
    constexpr int arows = 2 * MD::parts * R * kUmBands;  // (slot, part, row, band)
    for (int i = tid; i < arows; i += kUmThreads)
      *reinterpret_cast<uint4*>(smem_raw + (size_t)(i / (R * kUmBands)) * SM::kPart +
                                umma_kmajor_offset(i % (R * kUmBands), 16, kUmKBytes)) = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < 2 * MD::parts * kUmX; i += kUmThreads)
      *reinterpret_cast<uint4*>(smem_raw + SM::off_b() + (size_t)(i / kUmX) * SM::kBPart +
                                umma_kmajor_offset(i % kUmX, 16, kUmKBytes)) = make_uint4(0, 0, 0, 0);
  }
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int quarter = warp & 3;                    // tensor-memory lanes 32 quarter .. of this warp
  const uint32_t tlane = tmem + ((uint32_t)(32 * quarter) << 16);
#pragma unroll
  for (int c = 0; c < MD::cols / 64; c++) tmem_zero32(tlane + (uint32_t)((warp >> 2) * (MD::cols / 2) + 32 * c));

  // stage atom li into staging buffer sb: three bulk copies by one thread, completing on the buffer's barrier
  auto stage_atom = [&](int li, int sb) {
    if (tid != 0) return;
    const int4 r = slist[li];
    const int a = r.x, iz = r.w;
    const uint32_t dst = um_smem(stage + (size_t)sb * stf), bar = fbar0 + 8 * sb;
    const uint32_t bt2 = (uint32_t)(ntile * 32 * PP * 4), btab = (uint32_t)(C * NPX * 4);
    fence_async_smem();  // the buffer's earlier readers (generic proxy) are ordered before the copies
    um_expect_tx(bar, bt2 + 2 * btab);
    um_bulk(dst, t2 + (((size_t)a * C + iz) * nbt32 + bt0) * 32 * PP, bt2, bar);
    um_bulk(dst + kUmBands * PP * 4, tym + (size_t)a * C * NPX, btab, bar);             // y table [C][NPX]
    um_bulk(dst + (kUmBands * PP + C * NPX) * 4, txm + (size_t)a * C * NPX, btab, bar); // x table [C][NPX]
  };

  const int bl = tid & 127, rh = tid >> 7;         // this thread's band and row half (rows R/2 rh .. )
  const bool bvalid = bt0 * 32 + bl < B && bl < ntile * 32;
  constexpr uint32_t idesc = umma_idesc(MD::ab, kUmBands, kUmX);
  bool ok = true;
  int issued = 0;    // atoms whose MMAs have been issued and committed (the same count in every thread)
  int pending = -1;  // atom whose staging copies may still be in flight when the loop stops early

  // the tile's psi rows go to L2 now, so the read-modify-write at the end finds them there
  {
    const int row = tid >> 5, x = tid & 31, y = yb * R + row;
    if (row < R && y < Ny && xs + x < Nx) {
      const TP* p = psi + (((size_t)z * Ny + y) * Nx + xs + x) * (size_t)B + (size_t)bt0 * 32;
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"((uint32_t)(ntile * 32 * sizeof(TP)))
                   : "memory");
    }
  }

  // MMAs of atom li are issued after the block barrier that opens iteration li + 1 (one barrier per atom):
  // per row hi*hi into the row's accumulator, and for the split forms hi*lo + lo*hi into the same one
  // (3xTF32) or into the row's cross accumulator (split FP16)
  auto mma = [&](uint32_t d, uint64_t ad, uint64_t bd) {
    if constexpr (MD::h16)
      umma_f16(d, ad, bd, idesc, true);
    else
      umma_tf32(d, ad, bd, idesc, true);
  };
  auto issue = [&](int li) {
    const int slot = li & 1;
    tc05_fence_after();
    const uint32_t b0a = sB + (uint32_t)(slot * SM::kB);
    const uint64_t bh = umma_desc(b0a, 128, 8 * kUmKBytes);
#pragma unroll
    for (int row = 0; row < R; row++) {
      const uint32_t a0a = sA + (uint32_t)(slot * SM::kA + row * kUmBands * kUmKBytes);
      const uint64_t ah = umma_desc(a0a, 128, 8 * kUmKBytes);
      mma(tmem + (uint32_t)(row * kUmX), ah, bh);
      if constexpr (MD::split) {
        const uint64_t al = umma_desc(a0a + (uint32_t)SM::kPart, 128, 8 * kUmKBytes);
        const uint64_t bl2 = umma_desc(b0a + (uint32_t)SM::kBPart, 128, 8 * kUmKBytes);
        const uint32_t dc = tmem + (uint32_t)(((MD::nacc == 2 ? R : 0) + row) * kUmX);
        mma(dc, ah, bl2);
        mma(dc, al, bh);
      }
    }
    umma_commit(bar0 + 8 * slot);
  };

  stage_atom(0, 0);
  for (int li = 0; li < nlist; li++) {
    const int slot = li & 1;
    // atom li's staging buffer (its (li >> 1)-th fill) has landed
    if (!um_mbar_wait(fbar0 + 8 * slot, (uint32_t)((li >> 1) & 1), wait_cycles)) ok = false;
    tc05_fence_before();
    // atom li staged; the operands of atom li - 1 are written and its staging buffer is free; a wait
    // that ran out in any thread ends the loop for all
    if (!__syncthreads_and(ok)) {
      pending = li;
      break;
    }
    if (li >= 1) {
      if (tid == 0) issue(li - 1);
      issued = li;
    }
    if (li + 1 < nlist) stage_atom(li + 1, slot ^ 1);
    // operand slot `slot` was last read by the MMAs of atom li - 2
    if (li >= 2 && !um_mbar_wait(bar0 + 8 * slot, (uint32_t)(((li - 2) >> 1) & 1), wait_cycles)) ok = false;
    const int4 r = slist[li];
    const float* st = stage + (size_t)slot * stf;
    const float* tys = st + kUmBands * PP;   // [C][NPX]
    const float* txs = tys + C * NPX;         // [C][NPX]
    // y-pass for R / 2 rows of this band, written as A rows (K-major, 32 bytes per band and part)
    float t2r[P];
    {
      const float4* row4 = reinterpret_cast<const float4*>(st + (size_t)bl * PP);
#pragma unroll
      for (int p4 = 0; p4 < (P + 3) / 4; p4++) {
        const float4 v = bvalid ? row4[p4] : make_float4(0.f, 0.f, 0.f, 0.f);
        if (4 * p4 + 0 < P) t2r[4 * p4 + 0] = v.x;
        if (4 * p4 + 1 < P) t2r[4 * p4 + 1] = v.y;
        if (4 * p4 + 2 < P) t2r[4 * p4 + 2] = v.z;
        if (4 * p4 + 3 < P) t2r[4 * p4 + 3] = v.w;
      }
    }
    unsigned char* arow = smem_raw + (size_t)slot * SM::kA;
#pragma unroll
    for (int rr = 0; rr < R / 2; rr++) {
      const int row = (R / 2) * rh + rr;
      int iy = r.y + row;
      if (g.periodic && iy >= Ny) iy -= Ny;
      const bool yin = iy >= 0 && iy < C && yb * R + row < Ny;
      float t1[8];
#pragma unroll
      for (int n = 0; n < 8; n++) t1[n] = 0.0f;
      if (yin) {
        float wy[NPX];
#pragma unroll
        for (int q = 0; q < NPX / 4; q++) {
          const float4 w4 = reinterpret_cast<const float4*>(tys + iy * NPX)[q];
          wy[4 * q] = w4.x;
          wy[4 * q + 1] = w4.y;
          wy[4 * q + 2] = w4.z;
          wy[4 * q + 3] = w4.w;
        }
#pragma unroll
        for (int ny = 0; ny < NP; ny++)
#pragma unroll
          for (int nx = 0; nx + ny <= NU; nx++) t1[nx] = fmaf(t2r[BS::pair(nx, ny)], wy[ny], t1[nx]);
      }
      unsigned char* dst = arow + (size_t)row * kUmBands * kUmKBytes + umma_kmajor_offset(bl, 0, kUmKBytes);
      float hi[8], lo[8];
#pragma unroll
      for (int n = 0; n < 8; n++) um_parts<UM>(t1[n], hi[n], lo[n]);
#pragma unroll
      for (int part = 0; part < MD::parts; part++) {
        const float* v = part ? lo : hi;
        unsigned char* d = dst + (size_t)part * SM::kPart;
        *reinterpret_cast<uint4*>(d) = um_pack4<UM>(v);
        if constexpr (!MD::h16)
          *reinterpret_cast<uint4*>(d + 128) = um_pack4<UM>(v + 4);  // K bytes 16..31: the next core matrix
      }
    }
    // B: the atom's x functions on the tile's points, [32 x][8 states], zero outside the cube
    {
      const int x = tid >> 3, n = tid & 7;
      int ix = r.z + x;
      if (g.periodic && ix >= Nx) ix -= Nx;
      const float v = (ix >= 0 && ix < C && n < NP && xs + x < Nx) ? txs[ix * NPX + n] : 0.0f;
      float vp[2];
      um_parts<UM>(v, vp[0], vp[1]);
#pragma unroll
      for (int part = 0; part < MD::parts; part++) {
        unsigned char* bs = smem_raw + SM::off_b() + (size_t)slot * SM::kB + (size_t)part * SM::kBPart;
        if constexpr (UM == kUmBF16) {
          *reinterpret_cast<__nv_bfloat16*>(bs + umma_kmajor_offset(x, 2 * n, kUmKBytes)) = __float2bfloat16_rn(vp[part]);
        } else if constexpr (MD::h16) {
          *reinterpret_cast<__half*>(bs + umma_kmajor_offset(x, 2 * n, kUmKBytes)) = __float2half_rn(vp[part]);
        } else {
          *reinterpret_cast<uint32_t*>(bs + umma_kmajor_offset(x, 4 * n, kUmKBytes)) = tf32_bits(vp[part]);
        }
      }
    }
    fence_async_smem();  // the operands written above become visible to the tensor core
  }
  // the last atom's operands: one more barrier, then its MMAs
  tc05_fence_before();
  ok = __syncthreads_and(ok);  // the same verdict in every thread
  if (ok && issued == nlist - 1) {
    if (tid == 0) issue(nlist - 1);
    issued = nlist;
  }
  // the last commit covers every MMA issued before it
  const int last = issued - 1;
  bool done = ok && last >= 0 && um_mbar_wait(bar0 + 8 * (last & 1), (uint32_t)((last >> 1) & 1), wait_cycles);
  done = __syncthreads_and(done);
  if (pending >= 0) {
    // the copies staging atom `pending` may still be in flight: they complete whatever else happens, so
    // wait for them with the default limit before the CTA's shared memory is released
    (void)um_mbar_wait(fbar0 + 8 * (pending & 1), (uint32_t)((pending >> 1) & 1), kDefaultWaitCycles);
  }
  if (!done) {
    if (tid == 0) atomicOr(status, kStatusTimeout);
    // the MMAs issued so far still complete; give them the default limit before tensor memory is freed
    if (last >= 0) (void)um_mbar_wait(bar0 + 8 * (last & 1), (uint32_t)((last >> 1) & 1), kDefaultWaitCycles);
  }
  tc05_fence_after();
  if (done) {
    // warp w: lanes 32 (w % 4) .. (bands), rows (R / 2) (w / 4) .. (R / 2) (w / 4 + 1) - 1
    const int b = bt0 * 32 + 32 * quarter + lane;
    const bool bok = b < B && 32 * quarter < ntile * 32;
#pragma unroll 1
    for (int rr = 0; rr < R / 2; rr++) {
      const int row = (R / 2) * (warp >> 2) + rr;
      const int y = yb * R + row;
      float v[32];
      tmem_ld32(tlane + (uint32_t)(row * kUmX), v);
      if constexpr (MD::nacc == 2) {  // split FP16: main + 2^-11 cross
        float vc[32];
        tmem_ld32(tlane + (uint32_t)((R + row) * kUmX), vc);
#pragma unroll
        for (int x = 0; x < 32; x++) v[x] = fmaf(vc[x], 0x1p-11f, v[x]);
      }
      if (y < Ny && bok) {
        TP* rp = psi + ((size_t)z * Ny + y) * (size_t)Nx * B + b;
        const int xend = min(kUmX, Nx - xs);
        float old[32];
#pragma unroll
        for (int x = 0; x < 32; x++) old[x] = x < xend ? to_real(rp[(size_t)(xs + x) * B], 0.0f) : 0.0f;
#pragma unroll
        for (int x = 0; x < 32; x++)
          if (x < xend) rp[(size_t)(xs + x) * B] = store_cast(old[x] + v[x], (TP*)nullptr);
      }
    }
  }
  tc05_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, MD::cols);
}

// One tcgen05 MMA, M = 128, N = 32, of host operands (test of the operand layouts and descriptors).
template <bool BF>
__global__ void __launch_bounds__(128) k_umma_selftest(const float* __restrict__ A, const float* __restrict__ Bm,
                                                       float* __restrict__ D, int* __restrict__ status) {
  __shared__ __align__(1024) unsigned char sm[kUmBands * kUmKBytes + kUmX * kUmKBytes];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ uint32_t tslot;
  constexpr int K = BF ? 16 : 8;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < kUmBands * K; i += 128) {
    const int r = i / K, k = i % K;
    if constexpr (BF)
      *reinterpret_cast<__nv_bfloat16*>(sm + umma_kmajor_offset(r, 2 * k, kUmKBytes)) = __float2bfloat16_rn(A[i]);
    else
      *reinterpret_cast<uint32_t*>(sm + umma_kmajor_offset(r, 4 * k, kUmKBytes)) = tf32_bits(A[i]);
  }
  for (int i = tid; i < kUmX * K; i += 128) {
    const int r = i / K, k = i % K;
    unsigned char* bs = sm + kUmBands * kUmKBytes;
    if constexpr (BF)
      *reinterpret_cast<__nv_bfloat16*>(bs + umma_kmajor_offset(r, 2 * k, kUmKBytes)) = __float2bfloat16_rn(Bm[i]);
    else
      *reinterpret_cast<uint32_t*>(bs + umma_kmajor_offset(r, 4 * k, kUmKBytes)) = tf32_bits(Bm[i]);
  }
  if (warp == 0) tmem_alloc(um_smem(&tslot), 32);
  if (tid == 0) {
    um_mbar_init(um_smem(&bar));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  fence_async_smem();
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  const uint32_t tmem = tslot;
  if (tid == 0) {
    constexpr uint32_t idesc = umma_idesc(BF ? kUmmaBF16 : kUmmaTF32, kUmBands, kUmX);
    const uint64_t adesc = umma_desc(um_smem(sm), 128, 8 * kUmKBytes);
    const uint64_t bdesc = umma_desc(um_smem(sm + kUmBands * kUmKBytes), 128, 8 * kUmKBytes);
    if constexpr (BF)
      umma_f16(tmem, adesc, bdesc, idesc, false);
    else
      umma_tf32(tmem, adesc, bdesc, idesc, false);
    umma_commit(um_smem(&bar));
  }
  const bool done = um_mbar_wait(um_smem(&bar), 0, 2000000000ll);
  if (!done && tid == 0) atomicOr(status, kStatusTimeout);
  if (!done) (void)um_mbar_wait(um_smem(&bar), 0, kDefaultWaitCycles);
  tc05_fence_after();
  float v[32];
  tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16), v);
#pragma unroll
  for (int x = 0; x < 32; x++) D[(32 * warp + lane) * kUmX + x] = done ? v[x] : 0.0f;
  tc05_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 32);
}

// ------------------------------------------------------------------------------------ launchers
template <int NU, typename TP, int UM>
static cudaError_t umma_run(const ExpandLaunch& p) {
  const size_t smem = UmSmem<NU, UM>::bytes(p.g.cube, p.max_plane);
  if (smem > 227 * 1024) return cudaErrorNotSupported;
  auto kern = k_expand_umma<NU, TP, UM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  constexpr int R = UmMode<UM>::rows;
  const int nseg = (p.g.n[0] + kUmX - 1) / kUmX, nyb = (p.g.n[1] + R - 1) / R;
  const unsigned nblk = (unsigned)nseg * nyb * p.g.n[2];
  kern<<<dim3(nblk, (p.g.nbands + kUmBands - 1) / kUmBands), kUmThreads, smem, p.stream>>>(
      p.g, p.atoms, p.plane_ptr, p.plane_atoms, static_cast<const float*>(p.tables_ymajor),
      static_cast<const float*>(p.tables_xmajor), static_cast<const float*>(p.t2), static_cast<TP*>(p.psi), p.status,
      p.wait_cycles);
  return cudaGetLastError();
}

template <int NU, typename TP>
static cudaError_t umma_mode(const ExpandLaunch& p, sho_prec prec) {
  switch (prec) {
    case SHO_P_TF32: return umma_run<NU, TP, kUmTF32>(p);
    case SHO_P_BF16: return umma_run<NU, TP, kUmBF16>(p);
    case SHO_P_3XTF32: return umma_run<NU, TP, kUm3xTF32>(p);
    case SHO_P_SPLIT_FP16: return umma_run<NU, TP, kUmSplit16>(p);
    default: return cudaErrorNotSupported;
  }
}

template <int NU>
static cudaError_t umma_nu(const ExpandLaunch& p, sho_prec prec) {
  if constexpr (NU > 7) {
    return cudaErrorNotSupported;
  } else {
    // the y table y-major goes after the x-major x table in the same workspace region (the region holds
    // txm_bytes_per_point(numax) >= 8 NPX bytes per atom and cube point)
    ExpandLaunch q = p;
    q.tables_ymajor = static_cast<float*>(p.tables_xmajor) + (size_t)p.natoms * p.g.cube * ((NU + 4) & ~3);
    cudaError_t e = launch_expand_zpass_f32_tiled(q);
    if (e != cudaSuccess) return e;
    if (p.psi_dtype == SHO_F32) return umma_mode<NU, float>(q, prec);
    return umma_mode<NU, __nv_bfloat16>(q, prec);
  }
}

bool umma_expand_ok(const ExpandLaunch& p, sho_prec prec) {
  if (prec != SHO_P_TF32 && prec != SHO_P_BF16 && prec != SHO_P_3XTF32 && prec != SHO_P_SPLIT_FP16) return false;
  if (p.numax > 7 || (p.psi_dtype != SHO_F32 && p.psi_dtype != SHO_BF16)) return false;
  if (p.g.r2max > 0.0) return false;
  return UmSmem<7, kUmTF32>::bytes(p.g.cube, p.max_plane) <= 227 * 1024;
}

cudaError_t launch_expand_umma(const ExpandLaunch& p, sho_prec prec) {
  switch (p.numax) {
    case 0: return umma_nu<0>(p, prec);
    case 1: return umma_nu<1>(p, prec);
    case 2: return umma_nu<2>(p, prec);
    case 3: return umma_nu<3>(p, prec);
    case 4: return umma_nu<4>(p, prec);
    case 5: return umma_nu<5>(p, prec);
    case 6: return umma_nu<6>(p, prec);
    case 7: return umma_nu<7>(p, prec);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace sho

using namespace sho;

extern "C" int sho_selftest_umma(int bf16, const float* A, const float* Bm, float* D) {
  if (!A || !Bm || !D) return SHO_ERR_ARG;
  const int K = bf16 ? 16 : 8;
  float *dA = nullptr, *dB = nullptr, *dD = nullptr;
  int* dst = nullptr;
  int st = SHO_OK;
  if (cudaMalloc(&dA, sizeof(float) * kUmBands * K) != cudaSuccess ||
      cudaMalloc(&dB, sizeof(float) * kUmX * K) != cudaSuccess ||
      cudaMalloc(&dD, sizeof(float) * kUmBands * kUmX) != cudaSuccess || cudaMalloc(&dst, sizeof(int)) != cudaSuccess) {
    st = SHO_ERR_OOM;
  } else if (cudaMemcpy(dA, A, sizeof(float) * kUmBands * K, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(dB, Bm, sizeof(float) * kUmX * K, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemset(dst, 0, sizeof(int)) != cudaSuccess) {
    st = SHO_ERR_CUDA;
  } else {
    if (bf16)
      k_umma_selftest<true><<<1, 128>>>(dA, dB, dD, dst);
    else
      k_umma_selftest<false><<<1, 128>>>(dA, dB, dD, dst);
    int flag = 0;
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(D, dD, sizeof(float) * kUmBands * kUmX, cudaMemcpyDeviceToHost) != cudaSuccess ||
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
