// sho_fp32.cu -- bandwidth-oriented kernels of the FP32-class forms (FP32 CUDA cores and the
// tensor-core forms) for band counts whose rows are 16-byte aligned.
//
// Projection (k_project_pipe): one warp per (atom, 32-band tile, z-slab) as in sho_project.cu, but the
// cube rows are streamed through a 4-stage cp.async ring in shared memory, so each warp keeps three
// rows (3 x 4 KB in FP32) in flight while it contracts the fourth.  The x-pass runs on CUDA cores
// (one lane per band) or as MMA tiles (bands x states); the y/z passes and the cluster reduction are
// those of the CUDA-core kernel.
//
// Expansion (k_expand_blk): a gather over tiles of 8 grid rows x 32 x points x 32 bands of one z plane
// (8 warps, one per row).  For each atom whose cube meets the tile, the z-pass slice T2[a][z][32][PP]
// (band-tiled) and the atom's x/y tables are staged once in shared memory (cp.async, in groups of one
// or two atoms staged two groups ahead) and shared by the 8 row-warps; each warp runs the y-pass from
// shared memory and accumulates the x-pass into a register tile of its row (32 x points per lane on
// CUDA cores, or the MMA accumulator fragments).  Atoms are added in ascending order and each psi
// element is read and written once: deterministic, no atomics.
#include <cooperative_groups.h>

#include "sho_tc.cuh"

namespace cg = cooperative_groups;

namespace sho {

constexpr int kSimt = -1;     // MODE value of the CUDA-core x-pass
constexpr int kStages = 4;    // cp.async ring depth of the projection

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

template <typename TP>
struct RowLayout {
  // bytes of one x point (32 bands) in the shared ring, padded so the MMA fragment reads and the
  // lane-per-band reads are free of bank conflicts
  static constexpr int kStride = sizeof(TP) == 4 ? 160 : 80;
  static constexpr int kChunksPerX = 32 * (int)sizeof(TP) / 16;  // 16-byte copies per x point
};

// ------------------------------------------------------------------------------- projection
template <int NU, typename TP, int MODE>
struct PipeSmem {
  static constexpr int NP = NU + 1, NPX = (NP + 3) & ~3, N = Basis<NU>::N;
  // numax <= 7: the z-pass accumulators live in registers and the ring doubles as the buffer of the
  // final cluster reduction; larger bases keep them in shared memory.
  static constexpr bool ACCR = NU <= 7;
  __host__ __device__ static size_t ring_bytes(int cube) {
    const size_t ring = (size_t)kStages * cube * RowLayout<TP>::kStride;
    const size_t red = (size_t)N * kWarp * 4;
    return ACCR ? (ring > red ? ring : red) : ring;
  }
  static size_t bytes(int cube) {
    size_t t = ring_bytes(cube);                                          // ring (+ reduction buffer)
    t += (size_t)cube * NPX * 4 + 2 * (size_t)NP * cube * 4;              // tables
    t += 8 * 36 * 4;                                                      // transpose buffer
    if (!ACCR) t += (size_t)N * kWarp * 4;                                // partial coefficients
    t = (t + 15) & ~(size_t)15;
    t += (size_t)cube * 8;                                                // x offsets
    t += (size_t)2 * cube * 4;                                            // y and z grid indices
    return t;
  }
};

// v times the unit complex number ph (leading floats of its float pairs) for complex data held by lane
// pairs, the real part in the even lane and the imaginary part in the odd one (every lane calls it).
__device__ __forceinline__ float f32_rotate(float v, const float4 ph, int lane) {
  const float u = __shfl_xor_sync(0xffffffffu, v, 1);
  return fmaf(v, ph.x, ((lane & 1) ? u : -u) * ph.z);
}

// BLOCH (SIMT form, float psi): complex psi of a Bloch wave (Sec. 2.5), its (re, im) pairs as two real
// bands in neighbouring lanes; the x-pass sum turns by the x translation's phase where the cube row
// crosses the cell boundary, and each row's x-pass result by the phase of its translation, so that the
// y- and z-passes stay real (as in the FP64-accurate form).
template <int NU, typename TP, int MODE, bool BLOCH = false>
__global__ void __launch_bounds__(kWarp) k_project_pipe(GridDev g, const TP* __restrict__ psi,
                                                        const AtomDev* __restrict__ atoms,
                                                        const int* __restrict__ order, int zsplit,
                                                        float* __restrict__ coeff, const BlochPh* __restrict__ bph) {
  using BS = Basis<NU>;
  using SM = PipeSmem<NU, TP, MODE>;
  constexpr int NP = BS::NP, P = BS::P, N = BS::N, NPX = SM::NPX;
  constexpr int RS = RowLayout<TP>::kStride, CPX = RowLayout<TP>::kChunksPerX;
  constexpr int RSE = RS / (int)sizeof(TP);  // ring row stride in elements
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int C = g.cube;
  constexpr bool ACCR = SM::ACCR;
  unsigned char* ring = smem_raw;
  const size_t ringb = SM::ring_bytes(C);
  float* phx = reinterpret_cast<float*>(ring + ringb);                     // [C][NPX]
  float* phy = phx + (size_t)C * NPX;                                      // [NP][C]
  float* phz = phy + (size_t)NP * C;                                       // [NP][C]
  float* t1s = phz + (size_t)NP * C;                                       // [8][36]
  float* acc = ACCR ? reinterpret_cast<float*>(ring) : t1s + 8 * 36;       // [N][32]
  size_t off = ringb + ((size_t)C * NPX + 2 * (size_t)NP * C + 8 * 36 + (ACCR ? 0 : (size_t)N * kWarp)) * 4;
  off = (off + 15) & ~(size_t)15;
  long long* xoff = reinterpret_cast<long long*>(smem_raw + off);          // [C] element offset of x point
  int* yidx = reinterpret_cast<int*>(xoff + C);                            // [C] grid row of cube row
  int* zidx = yidx + C;                                                    // [C] grid plane of cube plane

  const int lane = threadIdx.x, gq = lane >> 2, tq = lane & 3;
  // atoms in the plan's spatial order, so CTAs running together read overlapping cubes
  const int a = order ? order[blockIdx.y] : (int)blockIdx.y;
  const int B = g.nbands;
  const int b0 = blockIdx.z * kWarp;
  const bool bok = b0 + lane < B;
  const AtomDev at = atoms[a];

  for (int i = lane; i < C; i += kWarp) {
    double col[NP];
    phi_column(cube_offset(at.o[0], i, g.h, at.X[0]), at.sigma, NU, col, 1);
#pragma unroll
    for (int n = 0; n < NPX; n++) phx[i * NPX + n] = n < NP ? (float)col[n] : 0.0f;
    phi_column(cube_offset(at.o[1], i, g.h, at.X[1]), at.sigma, NU, phy + i, C);
    phi_column(cube_offset(at.o[2], i, g.h, at.X[2]), at.sigma, NU, phz + i, C);
    const int jx = cube_index(at.o[0], i, g.n[0], g.periodic);
    xoff[i] = jx < 0 ? -1ll : (long long)jx * B;
    yidx[i] = cube_index(at.o[1], i, g.n[1], g.periodic);
    zidx[i] = cube_index(at.o[2], i, g.n[2], g.periodic);
  }
  float accr[ACCR ? N : 1];
  if constexpr (ACCR) {
#pragma unroll
    for (int k = 0; k < N; k++) accr[k] = 0.0f;
  } else {
    for (int i = lane; i < N * kWarp; i += kWarp) acc[i] = 0.0f;
  }
  __syncwarp();

  const int chunk = (C + zsplit - 1) / zsplit;
  const int iz0 = blockIdx.x * chunk, iz1 = min(C, iz0 + chunk);
  const int R = max(0, iz1 - iz0) * C;  // rows of this slab, iy fastest
  const long long rowlen = (long long)g.n[0] * B;
  const int valid_band_bytes = (B - b0) * (int)sizeof(TP);

  // Issue the copies of the next slab row r into its ring stage (nothing for clipped rows); rows are
  // issued in order, their cube plane and row kept as counters.
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
    const TP* row = psi + ((long long)jz * g.n[1] + jy) * rowlen + b0;
    unsigned char* st = ring + (size_t)(r % kStages) * C * RS;
    const int nchunks = C * CPX;
    for (int q = lane; q < nchunks; q += kWarp) {
      const int x = q / CPX, part = q - x * CPX;
      const long long o = xoff[x];
      int nb = valid_band_bytes - part * 16;
      nb = nb < 0 ? 0 : (nb > 16 ? 16 : nb);
      const void* src = (o >= 0 && nb > 0) ? (const void*)(reinterpret_cast<const unsigned char*>(row + o) + part * 16)
                                           : (const void*)psi;
      cp_async16(smem_u32(st + x * RS + part * 16), src, o >= 0 ? nb : 0);
    }
  };

  // B fragments of the tensor-core x-pass (fixed per atom)
  constexpr bool TC = MODE != kSimt;
  constexpr TcMode TM = TC ? (TcMode)MODE : TcMode::TF32;
  constexpr int K = TcK<TM>::K, NA = TcFrag<TM>::NA, NB = TcFrag<TM>::NB;
  constexpr int MAXSTEP = kMaxCube / K;
  BFrag<TM> bf[TC ? MAXSTEP : 1];
  if constexpr (TC) {
#pragma unroll
    for (int s = 0; s < MAXSTEP; s++) {
      if (s * K < C) {
        float bv[NB];
#pragma unroll
        for (int i = 0; i < NB; i++) {
          int k, n;
          b_coord<TM>(i, gq, tq, k, n);
          bv[i] = (n <= NU) ? phx[(s * K + k) * NPX + n] : 0.0f;
        }
        bf[s] = make_bfrag<TM>(bv);
      }
    }
  }

#pragma unroll
  for (int r = 0; r < kStages - 1; r++) {
    issue_next();
    cp_async_commit();
  }
  float t2[P];
#pragma unroll
  for (int p = 0; p < P; p++) t2[p] = 0.0f;

  for (int r = 0, iz = iz0, iy = 0; r < R; r++) {
    cp_async_wait<kStages - 2>();
    __syncwarp();
    issue_next();  // row r + kStages - 1
    cp_async_commit();
    if (zidx[iz] >= 0 && yidx[iy] >= 0) {
      const TP* st = reinterpret_cast<const TP*>(ring + (size_t)(r % kStages) * C * RS);
      float t1[NP];
      if constexpr (!TC) {
#pragma unroll
        for (int n = 0; n < NP; n++) t1[n] = 0.0f;
        auto xpass = [&](int x0, int x1) {
          for (int ix = x0; ix < x1; ix++) {
            const float v = to_real(st[ix * RSE + lane], 0.0f);
            const float4* f4 = reinterpret_cast<const float4*>(phx + ix * NPX);
#pragma unroll
            for (int q = 0; q < NPX / 4; q++) {
              const float4 f = f4[q];
              if (4 * q + 0 < NP) t1[4 * q + 0] = fmaf(v, f.x, t1[4 * q + 0]);
              if (4 * q + 1 < NP) t1[4 * q + 1] = fmaf(v, f.y, t1[4 * q + 1]);
              if (4 * q + 2 < NP) t1[4 * q + 2] = fmaf(v, f.z, t1[4 * q + 2]);
              if (4 * q + 3 < NP) t1[4 * q + 3] = fmaf(v, f.w, t1[4 * q + 3]);
            }
          }
        };
        if constexpr (BLOCH) {
          // points before the crossing w, the sum turned by ph(before) / ph(after), the points after it,
          // and the row's sum turned by the phase of its last run (y and z bits of this row and plane)
          const BlochPh& bp = bph[a];
          const int wx = min(bp.w[0], C);
          xpass(0, wx);
          if (wx < C) {
#pragma unroll
            for (int n = 0; n < NP; n++) t1[n] = f32_rotate(t1[n], bp.xstep, lane);
          }
          xpass(wx, C);
          const float4 ph = bp.ph[(wx < C ? 1 : 0) + (iy >= bp.w[1] ? 2 : 0) + (iz >= bp.w[2] ? 4 : 0)];
#pragma unroll
          for (int n = 0; n < NP; n++) t1[n] = f32_rotate(t1[n], ph, lane);
        } else {
          xpass(0, C);
        }
      } else {
        float d[2][4], dl[2][4];
#pragma unroll
        for (int m = 0; m < 2; m++)
#pragma unroll
          for (int j = 0; j < 4; j++) d[m][j] = dl[m][j] = 0.0f;
#pragma unroll
        for (int s = 0; s < MAXSTEP; s++) {
          if (s * K < C) {
#pragma unroll
            for (int m = 0; m < 2; m++) {
              float av[NA];
#pragma unroll
              for (int i = 0; i < NA; i++) {
                int mm, k;
                a_coord<TM>(i, gq, tq, mm, k);
                av[i] = to_real(st[(s * K + k) * RSE + 16 * m + mm], 0.0f);
              }
              tc_product<TM>(d[m], dl[m], av, bf[s]);
            }
          }
        }
        const float ls = tc_lo_scale<TM>();
#pragma unroll
        for (int m = 0; m < 2; m++) {
          t1s[(2 * tq) * 36 + 16 * m + gq] = d[m][0] + ls * dl[m][0];
          t1s[(2 * tq + 1) * 36 + 16 * m + gq] = d[m][1] + ls * dl[m][1];
          t1s[(2 * tq) * 36 + 16 * m + gq + 8] = d[m][2] + ls * dl[m][2];
          t1s[(2 * tq + 1) * 36 + 16 * m + gq + 8] = d[m][3] + ls * dl[m][3];
        }
        __syncwarp();
#pragma unroll
        for (int n = 0; n < NP; n++) t1[n] = t1s[n * 36 + lane];
      }
      // y-pass
#pragma unroll
      for (int ny = 0; ny < NP; ny++) {
        const float w = phy[ny * C + iy];
#pragma unroll
        for (int nx = 0; nx + ny <= NU; nx++) t2[BS::pair(nx, ny)] = fmaf(t1[nx], w, t2[BS::pair(nx, ny)]);
      }
    }
    __syncwarp();
    if (iy == C - 1) {
      // z-pass of the finished plane
      int k = 0;
#pragma unroll
      for (int nz = 0; nz < NP; nz++) {
        const float w = phz[nz * C + iz];
#pragma unroll
        for (int ny = 0; ny + nz <= NU; ny++)
#pragma unroll
          for (int nx = 0; nx + ny + nz <= NU; nx++) {
            if constexpr (ACCR)
              accr[k] = fmaf(t2[BS::pair(nx, ny)], w, accr[k]);
            else
              acc[k * kWarp + lane] = fmaf(t2[BS::pair(nx, ny)], w, acc[k * kWarp + lane]);
            k++;
          }
      }
#pragma unroll
      for (int p = 0; p < P; p++) t2[p] = 0.0f;
    }
    if (++iy == C) {
      iy = 0;
      iz++;
    }
  }
  cp_async_wait<0>();
  __syncwarp();
  if constexpr (ACCR) {
#pragma unroll
    for (int k = 0; k < N; k++) acc[k * kWarp + lane] = accr[k];
  }

  cg::cluster_group cl = cg::this_cluster();
  cl.sync();
  const int rank = (int)cl.block_rank();
  const float h3 = (float)(g.h * g.h * g.h);
  for (int k = rank; k < N; k += zsplit) {
    float sum = 0.0f;
    for (int q = 0; q < zsplit; q++) sum += cl.map_shared_rank(acc, q)[k * kWarp + lane];
    if (bok) coeff[((long long)a * N + k) * B + b0 + lane] = sum * h3;
  }
  cl.sync();
}

// ------------------------------------------------------------------------------- expansion
constexpr int kRowsPerBlk = 8;       // grid rows (warps) per CTA
// atoms staged and computed per block barrier: two for the CUDA-core x-pass (its per-atom work is
// short), one for the MMA forms (measured faster with the smaller staging footprint)
template <int MODE>
struct AtomsPerBarrier {
  static constexpr int value = MODE == kSimt ? 2 : 1;
};
constexpr int kXSeg = 32;            // x points per tile

// Expansion x-pass B fragments, per atom and cube x point: entry (ix, t) is the fragment that lane
// t = lane % 4 of a warp uses for grid point ix (column n = lane / 4 of an MMA tile), converted to the
// mode's operand type once per atom: 4 words (hi and lo parts) for the split forms, else 2.
template <TcMode TM>
struct XFrag {
  static constexpr int WORDS = (TM == TcMode::X3TF32 || TM == TcMode::SPLIT16) ? 4 : 2;
};

template <int NU, int MODE>
struct BlkSmem {
  static constexpr bool TC = MODE != kSimt;
  static constexpr int NP = NU + 1, P = Basis<NU>::P, NPX = (NP + 3) & ~3, PP = tiled_pairs(P);
  static constexpr int XW = TC ? XFrag<TC ? (TcMode)MODE : TcMode::TF32>::WORDS : 0;
  static constexpr int kAtomsPerBarrier = AtomsPerBarrier<MODE>::value;
  // x data of one atom: CUDA cores the x table [C][NPX] (x-major); tensor forms the B fragments
  // [C + 1][4] of XW words, row C all zero (the fragment of points outside the cube)
  __host__ __device__ static size_t xtab_floats(int cube) {
    return TC ? (size_t)(cube + 1) * 4 * XW : (size_t)NPX * cube;
  }
  // per buffer: T2 slice [32 bands][PP] + x data + y table [NP][C]
  __host__ __device__ static size_t buf_floats(int cube) {
    return (size_t)PP * 32 + xtab_floats(cube) + (size_t)NP * cube;
  }
  // 3 groups of kAtomsPerBarrier staging buffers + (tensor forms) per-warp T1 transposes + atom list
  static size_t bytes(int cube, int max_plane) {
    return (3 * kAtomsPerBarrier * buf_floats(cube) + (TC ? (size_t)kRowsPerBlk * 16 * 36 : 0)) * 4 +
           (size_t)(max_plane + 1) * sizeof(int4);
  }
};

// The B-fragment table of the tensor forms, [A][C][4] entries of XFrag::WORDS words, from the x-major
// x table [A][C][NPX] (one block per atom).
template <int NU, int MODE>
__global__ void k_expand_xfrag(int cube, const float* __restrict__ txm, uint32_t* __restrict__ xf) {
  constexpr TcMode TM = (TcMode)MODE;
  constexpr int NP = NU + 1, NPX = (NP + 3) & ~3, NB = TcFrag<TM>::NB, W = XFrag<TM>::WORDS;
  const int a = blockIdx.x;
  for (int i = threadIdx.x; i < cube * 4; i += blockDim.x) {
    const int ix = i >> 2, t = i & 3;
    float bv[NB];
#pragma unroll
    for (int e = 0; e < NB; e++) {
      int k, n;
      b_coord<TM>(e, 0, t, k, n);
      bv[e] = k < NP ? txm[((size_t)a * cube + ix) * NPX + k] : 0.0f;
    }
    const BFrag<TM> f = make_bfrag<TM>(bv);
    uint32_t* dst = xf + ((size_t)a * cube * 4 + i) * W;
    dst[0] = f.hi[0];
    dst[1] = f.hi[1];
    if constexpr (W == 4) {
      dst[2] = f.lo[0];
      dst[3] = f.lo[1];
    }
  }
}

// Tensor forms: at most 128 registers, two blocks of 8 warps per SM; the CUDA-core form on FP32 psi at
// most 64 (four blocks); on BF16 psi the compiler's choice (about 80 registers, three blocks).
// BLOCH (SIMT form, float psi): complex coefficients and psi of a Bloch wave, (re, im) pairs as two real
// bands in neighbouring lanes; each (atom, row) y-pass result turns by the phase of the translation of
// each tile point it updates (the point's cube index before or after the crossing w), so that the z-, y-
// and x-passes stay real.
template <int NU, typename TP, int MODE, bool BLOCH = false>
__global__ void __launch_bounds__(kRowsPerBlk * kWarp, MODE != kSimt ? 2 : sizeof(TP) == 4 ? 4 : 0) k_expand_blk(GridDev g, const AtomDev* __restrict__ atoms,
                                                                    const int* __restrict__ plane_ptr,
                                                                    const int* __restrict__ plane_atoms,
                                                                    const float* __restrict__ tables,
                                                                    const float* __restrict__ txm,
                                                                    const uint32_t* __restrict__ xf,
                                                                    const float* __restrict__ t2,
                                                                    TP* __restrict__ psi,
                                                                    const BlochPh* __restrict__ bph) {
  using BS = Basis<NU>;
  using SM = BlkSmem<NU, MODE>;
  constexpr bool TC = MODE != kSimt;
  constexpr int NP = BS::NP, NPX = SM::NPX, XW = SM::XW, PP = SM::PP;
  constexpr int kAtomsPerBarrier = SM::kAtomsPerBarrier;
  constexpr TcMode TM = TC ? (TcMode)MODE : TcMode::TF32;
  constexpr int K = TcK<TM>::K, NA = TcFrag<TM>::NA;
  static_assert(!TC || K >= NP, "one MMA K step covers the states");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int C = g.cube;
  const int Nx = g.n[0], Ny = g.n[1], Nz = g.n[2];
  const size_t bufsz = SM::buf_floats(C);
  const size_t xtab = SM::xtab_floats(C);
  float* bufs = reinterpret_cast<float*>(smem_raw);  // 3 x kAtomsPerBarrier x [T2 slice | x data | y table]
  float* t1all = bufs + 3 * kAtomsPerBarrier * bufsz;            // [warps][16][36] (tensor forms)
  int4* slist = reinterpret_cast<int4*>(t1all + (TC ? kRowsPerBlk * 16 * 36 : 0));  // atoms meeting the tile, ascending
  __shared__ int wcount[kRowsPerBlk];
  __shared__ int s_nlist;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
  float* t1s = t1all + warp * 16 * 36;

  const int nseg = (Nx + kXSeg - 1) / kXSeg, nyb = (Ny + kRowsPerBlk - 1) / kRowsPerBlk;
  int bid = blockIdx.x;
  const int seg = bid % nseg;
  bid /= nseg;
  const int yb = bid % nyb;
  const int z = bid / nyb;
  const int xs = seg * kXSeg;
  const int y = yb * kRowsPerBlk + warp;
  const bool yok = y < Ny;
  const int B = g.nbands;
  const int b0 = blockIdx.y * kWarp;
  const bool bok = b0 + lane < B;
  const int q0 = plane_ptr[z], q1 = plane_ptr[z + 1];

  // Offsets of atom a's cube against this tile, wrapped into [0, N) on a periodic grid: r.y = cube
  // row of the tile's first row, r.z = cube point of its first x point, r.w = cube plane of z.  True
  // when the cube meets the tile's rows and x segment.  Computed once per (tile, atom) here, so the
  // atom loop below does no integer division.
  auto locate = [&](const AtomDev& at, int4& r) {
    int dy = yb * kRowsPerBlk - at.o[1], dx = xs - at.o[0], dz = z - at.o[2];
    bool m;
    if (g.periodic) {
      dy %= Ny;
      if (dy < 0) dy += Ny;
      dx %= Nx;
      if (dx < 0) dx += Nx;
      dz %= Nz;
      if (dz < 0) dz += Nz;
      m = (dy < C || dy + kRowsPerBlk > Ny) && (dx < C || dx + kXSeg > Nx);
    } else {
      m = dy < C && dy + kRowsPerBlk > 0 && dx < C && dx + kXSeg > 0;
    }
    r = make_int4(0, dy, dx, dz);
    return m;
  };

  // Stage atom a's T2 slice (plane z) and tables into buffer `buf` (all threads).
  auto stage = [&](const int4 r, int buf) {
    const int a = r.x, iz = r.w;
    float* dst = bufs + (size_t)buf * bufsz;
    // band-tiled T2: the [32][PP] slice of (atom, plane, band tile) is contiguous
    const float* src_t2 = t2 + (((size_t)a * C + iz) * gridDim.y + blockIdx.y) * kWarp * PP;
    for (int q = tid; q < 8 * PP; q += kRowsPerBlk * kWarp) cp_async16(smem_u32(dst + q * 4), src_t2 + q * 4, 16);
    if constexpr (TC) {
      const uint32_t* src_f = xf + (size_t)a * C * 4 * XW;     // B fragments [C][4] (row C stays zero)
      for (int q = tid; q < C * XW; q += kRowsPerBlk * kWarp)
        cp_async16(smem_u32(dst + PP * 32 + q * 4), src_f + q * 4, 16);
    } else {
      const float* src_x = txm + (size_t)a * C * NPX;           // x table, x-major [C][NPX]
      for (int q = tid; q < C * NPX / 4; q += kRowsPerBlk * kWarp)
        cp_async16(smem_u32(dst + PP * 32 + q * 4), src_x + q * 4, 16);
    }
    const float* src_y = tables + (size_t)a * 2 * NP * C + (size_t)NP * C;  // y table [NP][C]
    for (int q = tid; q < NP * C / 4; q += kRowsPerBlk * kWarp)
      cp_async16(smem_u32(dst + PP * 32 + xtab + q * 4), src_y + q * 4, 16);
  };

  // register tile: 32 x points of this warp's row, 32 bands
  float accr[TC ? 32 : 32];
  TP* rowp = psi + ((size_t)z * Ny + (yok ? y : 0)) * (size_t)Nx * B + b0;
  if constexpr (!TC) {
#pragma unroll
    for (int x = 0; x < kXSeg; x++)
      accr[x] = (yok && bok && xs + x < Nx) ? to_real(rowp[(size_t)(xs + x) * B + lane], 0.0f) : 0.0f;
  } else {
    // accumulator fragments: tile j (x = 8j..8j+7), M tile m (bands 16m..16m+15), element e:
    // (band 16m + gq + 8(e>>1), x 8j + 2tq + (e&1))
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int m = 0; m < 2; m++)
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const int band = 16 * m + gq + 8 * (e >> 1), x = xs + 8 * j + 2 * tq + (e & 1);
          accr[(j * 2 + m) * 4 + e] =
              (yok && x < Nx && b0 + band < B) ? to_real(rowp[(size_t)x * B + band], 0.0f) : 0.0f;
        }
  }
  if constexpr (TC) {
    for (int i = lane; i < 16 * 36; i += kWarp) t1s[i] = 0.0f;
    // the zero fragment row (index C) of the staging buffers; staging never writes it
    for (int i = tid; i < 3 * kAtomsPerBarrier * 4 * XW; i += kRowsPerBlk * kWarp)
      bufs[(size_t)(i / (4 * XW)) * bufsz + PP * 32 + (size_t)C * 4 * XW + i % (4 * XW)] = 0.0f;
  }

  // The plane's atoms that meet this tile, tested in parallel and compacted in ascending order.
  if (tid == 0) s_nlist = 0;
  __syncthreads();
  for (int base = q0; base < q1; base += kRowsPerBlk * kWarp) {
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
      for (int w = 0; w < kRowsPerBlk; w++) s_nlist += wcount[w];
    __syncthreads();
  }
  const int nlist = s_nlist;

  // walk them in groups of kAtomsPerBarrier atoms, three groups of staging buffers, groups staged two
  // ahead: the one barrier per group also shows that every warp is done with group gi - 1, whose
  // buffers are refilled with group gi + 2
  const int ngroups = (nlist + kAtomsPerBarrier - 1) / kAtomsPerBarrier;
  auto stage_group = [&](int gi, int slot) {
    for (int k = 0; k < kAtomsPerBarrier; k++) {
      const int li = gi * kAtomsPerBarrier + k;
      if (li < nlist) stage(slist[li], slot * kAtomsPerBarrier + k);
    }
  };
  if (ngroups > 0) stage_group(0, 0);
  cp_async_commit();
  if (ngroups > 1) stage_group(1, 1);
  cp_async_commit();
  for (int gi = 0, slot = 0; gi < ngroups; gi++, slot = slot == 2 ? 0 : slot + 1) {
    cp_async_wait<1>();  // this thread's copies of group gi have landed
    __syncthreads();
    if (gi + 2 < ngroups) stage_group(gi + 2, slot == 0 ? 2 : slot - 1);
    cp_async_commit();
    for (int k = 0; k < kAtomsPerBarrier; k++) {
      const int li = gi * kAtomsPerBarrier + k;
      if (li >= nlist) break;
      const int4 r = slist[li];
      const int buf = slot * kAtomsPerBarrier + k;
      const float* t2s = bufs + (size_t)buf * bufsz;
      const float* txs = t2s + PP * 32;      // x table [C][NPX], or B fragments [C + 1][4][XW] words
      const float* tys = txs + xtab;         // [NP][C]
      int iy = r.y + warp;  // cube row of this warp's grid row
      if (g.periodic && iy >= Ny) iy -= Ny;
      if (yok && iy >= 0 && iy < C) {
        // y-pass: T1[nx] for this row, lane = band; the lane's [PP] row of pairs comes in 16-byte loads
        float t1[NP], wy[NP];
#pragma unroll
        for (int n = 0; n < NP; n++) {
          t1[n] = 0.0f;
          wy[n] = tys[n * C + iy];
        }
        const float4* row4 = reinterpret_cast<const float4*>(t2s + lane * PP);
#pragma unroll
        for (int ny = 0; ny < NP; ny++)
#pragma unroll
          for (int nx = 0; nx + ny <= NU; nx++) {
            const int p = BS::pair(nx, ny);
            const float4 v = row4[p >> 2];  // the 16-byte chunk holding pair p (one load per chunk after unrolling)
            const float tv = (p & 3) == 0 ? v.x : (p & 3) == 1 ? v.y : (p & 3) == 2 ? v.z : v.w;
            t1[nx] = fmaf(tv, wy[ny], t1[nx]);
          }
        const int dx = r.z;  // cube index of tile point x is dx + x (mod Nx when periodic)
        if constexpr (!TC) {
          // Bloch data: the y-pass result turned by the phases of both runs of the cube row (before and
          // after the crossing w); each point takes the one of its cube index
          float t1b[BLOCH ? NP : 1];
          int wx = C;
          if constexpr (BLOCH) {
            const BlochPh& bp = bph[r.x];
            wx = bp.w[0];
            const int yz = (iy >= bp.w[1] ? 2 : 0) + (r.w >= bp.w[2] ? 4 : 0);
            const float4 ph0 = bp.ph[yz], ph1 = bp.ph[1 + yz];
#pragma unroll
            for (int n = 0; n < NP; n++) {
              t1b[n] = f32_rotate(t1[n], ph1, lane);
              t1[n] = f32_rotate(t1[n], ph0, lane);
            }
          }
#pragma unroll
          for (int x = 0; x < kXSeg; x++) {
            int ix = dx + x;
            if (g.periodic && ix >= Nx) ix -= Nx;
            if (ix >= 0 && ix < C) {
              float s = accr[x];
              const float4* f4 = reinterpret_cast<const float4*>(txs + ix * NPX);
              float tt[NP];
#pragma unroll
              for (int n = 0; n < NP; n++) {
                if constexpr (BLOCH)
                  tt[n] = ix >= wx ? t1b[n] : t1[n];
                else
                  tt[n] = t1[n];
              }
#pragma unroll
              for (int q = 0; q < NPX / 4; q++) {
                const float4 f = f4[q];
                if (4 * q + 0 < NP) s = fmaf(tt[4 * q + 0], f.x, s);
                if (4 * q + 1 < NP) s = fmaf(tt[4 * q + 1], f.y, s);
                if (4 * q + 2 < NP) s = fmaf(tt[4 * q + 2], f.z, s);
                if (4 * q + 3 < NP) s = fmaf(tt[4 * q + 3], f.w, s);
              }
              accr[x] = s;
            }
          }
        } else {
#pragma unroll
          for (int n = 0; n < NP; n++) t1s[n * 36 + lane] = t1[n];
          __syncwarp();
          AFrag<TM> afr[2];  // converted once, used by the four x tiles
#pragma unroll
          for (int m = 0; m < 2; m++) {
            float av[NA];
#pragma unroll
            for (int i = 0; i < NA; i++) {
              int mm, k;
              a_coord<TM>(i, gq, tq, mm, k);
              av[i] = t1s[k * 36 + 16 * m + mm];
            }
            afr[m] = make_afrag<TM>(av);
          }
          __syncwarp();
          constexpr bool SPLIT = TM == TcMode::X3TF32 || TM == TcMode::SPLIT16;
          const uint32_t* xfs = reinterpret_cast<const uint32_t*>(txs);
#pragma unroll
          for (int j = 0; j < 4; j++) {
            // this lane's column n = gq of tile j is cube point ix; outside the cube the zero row C
            int ix = dx + 8 * j + gq;
            if (g.periodic && ix >= Nx) ix -= Nx;
            ix = (unsigned)ix < (unsigned)C ? ix : C;
            BFrag<TM> bfr;
            if constexpr (XW == 4) {
              const uint4 v = *reinterpret_cast<const uint4*>(xfs + (ix * 4 + tq) * 4);
              bfr.hi[0] = v.x;
              bfr.hi[1] = v.y;
              bfr.lo[0] = v.z;
              bfr.lo[1] = v.w;
            } else {
              const uint2 v = *reinterpret_cast<const uint2*>(xfs + (ix * 4 + tq) * 2);
              bfr.hi[0] = v.x;
              bfr.hi[1] = v.y;
              bfr.lo[0] = bfr.lo[1] = 0u;
            }
#pragma unroll
            for (int m = 0; m < 2; m++) {
              float(&d)[4] = *reinterpret_cast<float(*)[4]>(&accr[(j * 2 + m) * 4]);
              float dl[4] = {0.0f, 0.0f, 0.0f, 0.0f};
              tc_product_pre<TM>(d, dl, afr[m], bfr);
              if constexpr (SPLIT) {
                const float ls = tc_lo_scale<TM>();
#pragma unroll
                for (int e = 0; e < 4; e++) d[e] = fmaf(ls, dl[e], d[e]);
              }
            }
          }
        }
      }
    }
  }
  cp_async_wait<0>();

  if (!yok) return;
  if constexpr (!TC) {
    if (bok)
#pragma unroll
      for (int x = 0; x < kXSeg; x++)
        if (xs + x < Nx) rowp[(size_t)(xs + x) * B + lane] = store_cast(accr[x], (TP*)nullptr);
  } else {
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int m = 0; m < 2; m++)
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const int band = 16 * m + gq + 8 * (e >> 1), x = xs + 8 * j + 2 * tq + (e & 1);
          if (x < Nx && b0 + band < B) rowp[(size_t)x * B + band] = store_cast(accr[(j * 2 + m) * 4 + e], (TP*)nullptr);
        }
  }
}

// ------------------------------------------------------------------------------- launchers
template <int NU, typename TP, int MODE>
static cudaError_t pipe_project_t(const ProjectLaunch& p) {
  const size_t smem = PipeSmem<NU, TP, MODE>::bytes(p.g.cube);
  auto kern = k_project_pipe<NU, TP, MODE>;
  if constexpr (MODE == kSimt && sizeof(TP) == 4 && NU <= kBlochRealMaxNumax) {
    if (p.bloch) kern = k_project_pipe<NU, TP, MODE, true>;
  } else if (p.bloch) {
    return cudaErrorInvalidValue;  // Bloch data: the FP32 CUDA-core form with float psi only
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.zsplit, p.natoms, (p.g.nbands + kWarp - 1) / kWarp);
  cfg.blockDim = dim3(kWarp, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = p.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = p.zsplit;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, p.g, static_cast<const TP*>(p.psi), p.atoms, p.order, p.zsplit,
                            static_cast<float*>(p.coeff), p.bloch);
}

template <int NU, typename TP, int MODE>
static cudaError_t blk_expand_t(const ExpandLaunch& p) {
  cudaError_t e = launch_expand_zpass_f32_tiled(p);
  if (e != cudaSuccess) return e;
  const uint32_t* xf = nullptr;
  if constexpr (MODE != kSimt) {
    // B fragments after the x-major x table in the same workspace
    constexpr int NPX = BlkSmem<NU, MODE>::NPX;
    uint32_t* f = reinterpret_cast<uint32_t*>(static_cast<float*>(p.tables_xmajor) + (size_t)p.natoms * p.g.cube * NPX);
    k_expand_xfrag<NU, MODE><<<p.natoms, 128, 0, p.stream>>>(p.g.cube, static_cast<const float*>(p.tables_xmajor), f);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    xf = f;
  }
  const size_t smem = BlkSmem<NU, MODE>::bytes(p.g.cube, p.max_plane);
  auto kern = k_expand_blk<NU, TP, MODE>;
  if constexpr (MODE == kSimt && sizeof(TP) == 4 && NU <= kBlochRealMaxNumax) {
    if (p.bloch) kern = k_expand_blk<NU, TP, MODE, true>;
  } else if (p.bloch) {
    return cudaErrorInvalidValue;  // Bloch data: the FP32 CUDA-core form with float psi only
  }
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int nseg = (p.g.n[0] + kXSeg - 1) / kXSeg, nyb = (p.g.n[1] + kRowsPerBlk - 1) / kRowsPerBlk;
  const unsigned nblk = (unsigned)nseg * nyb * p.g.n[2];
  kern<<<dim3(nblk, (p.g.nbands + kWarp - 1) / kWarp), kRowsPerBlk * kWarp, smem, p.stream>>>(
      p.g, p.atoms, p.plane_ptr, p.plane_atoms, static_cast<const float*>(p.tables),
      static_cast<const float*>(p.tables_xmajor), xf, static_cast<const float*>(p.t2), static_cast<TP*>(p.psi), p.bloch);
  return cudaGetLastError();
}

template <int NU, int MODE>
static cudaError_t fp32_dispatch_dtype(int op, const ProjectLaunch* pp, const ExpandLaunch* pe) {
  const sho_dtype dt = op == 0 ? pp->psi_dtype : pe->psi_dtype;
  if (dt == SHO_F32) return op == 0 ? pipe_project_t<NU, float, MODE>(*pp) : blk_expand_t<NU, float, MODE>(*pe);
  if (dt == SHO_BF16)
    return op == 0 ? pipe_project_t<NU, __nv_bfloat16, MODE>(*pp) : blk_expand_t<NU, __nv_bfloat16, MODE>(*pe);
  return cudaErrorInvalidValue;
}

template <int NU>
static cudaError_t fp32_dispatch_mode(int op, sho_prec prec, const ProjectLaunch* pp, const ExpandLaunch* pe) {
  if constexpr (NU <= 7) {
    switch (prec) {
      case SHO_P_FP32: return fp32_dispatch_dtype<NU, kSimt>(op, pp, pe);
      case SHO_P_TF32: return fp32_dispatch_dtype<NU, (int)TcMode::TF32>(op, pp, pe);
      case SHO_P_3XTF32: return fp32_dispatch_dtype<NU, (int)TcMode::X3TF32>(op, pp, pe);
      case SHO_P_BF16: return fp32_dispatch_dtype<NU, (int)TcMode::BF16>(op, pp, pe);
      case SHO_P_SPLIT_FP16: return fp32_dispatch_dtype<NU, (int)TcMode::SPLIT16>(op, pp, pe);
      default: return cudaErrorInvalidValue;
    }
  } else {
    if (prec == SHO_P_FP32) return fp32_dispatch_dtype<NU, kSimt>(op, pp, pe);
    return cudaErrorInvalidValue;
  }
}

static cudaError_t fp32_dispatch(int op, int numax, sho_prec prec, const ProjectLaunch* pp, const ExpandLaunch* pe) {
  switch (numax) {
    case 0: return fp32_dispatch_mode<0>(op, prec, pp, pe);
    case 1: return fp32_dispatch_mode<1>(op, prec, pp, pe);
    case 2: return fp32_dispatch_mode<2>(op, prec, pp, pe);
    case 3: return fp32_dispatch_mode<3>(op, prec, pp, pe);
    case 4: return fp32_dispatch_mode<4>(op, prec, pp, pe);
    case 5: return fp32_dispatch_mode<5>(op, prec, pp, pe);
    case 6: return fp32_dispatch_mode<6>(op, prec, pp, pe);
    case 7: return fp32_dispatch_mode<7>(op, prec, pp, pe);
    case 8: return fp32_dispatch_mode<8>(op, prec, pp, pe);
    case 9: return fp32_dispatch_mode<9>(op, prec, pp, pe);
    case 10: return fp32_dispatch_mode<10>(op, prec, pp, pe);
    default: return cudaErrorInvalidValue;
  }
}

// The streaming kernels need 16-byte aligned rows of bands: B * sizeof(element) % 16 == 0 for psi
// (and B % 4 == 0 for the FP32 intermediates of the expansion), and 16-byte aligned base pointers.
bool fp32_stream_ok(const void* psi, sho_dtype dt, int nbands) {
  const int es = dt == SHO_BF16 ? 2 : 4;
  return ((uintptr_t)psi % 16 == 0) && ((nbands * es) % 16 == 0) && (nbands % 4 == 0);
}

cudaError_t launch_project_fp32(const ProjectLaunch& p, sho_prec prec) { return fp32_dispatch(0, p.numax, prec, &p, nullptr); }

cudaError_t launch_expand_fp32(const ExpandLaunch& p, sho_prec prec) {
  if (p.kernel != 1 && umma_expand_ok(p, prec)) return launch_expand_umma(p, prec);
  return fp32_dispatch(1, p.numax, prec, nullptr, &p);
}

}  // namespace sho
