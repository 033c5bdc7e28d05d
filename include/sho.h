/*
 * sho.h -- C ABI of the GB300 SHO projector library (libsho.so).
 *
 * Projection of real-space grid wave functions onto analytical SHO (3D Hermite-Gauss) projector
 * functions, and its adjoint, the expansion, after Baumeister & Tsukamoto, "Analytical PAW Projector
 * Functions for Reduced Bandwidth Requirements" (PASC'19).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  Grid       grid point j = (jx, jy, jz), 0 <= j_d < n[d], sits at r = h * j (lengths in Bohr).
 *             psi is stored psi[jz][jy][jx][b]: bands innermost (the paper vectorises over bands,
 *             Sec. 6), contiguous, element type given by a sho_dtype.
 *  Atoms      pos[a][3] (x, y, z) and sigma[a] are HOST arrays of double.  The cube of atom a has
 *             edge `cube` points; its origin per axis is o_d = floor(pos[a][d] / h) - cube/2 + 1 and
 *             cube point i_d maps to grid index (o_d + i_d) mod n[d] (periodic) or is dropped when
 *             outside [0, n[d]) (not periodic).  The functions are evaluated at the unwrapped offset
 *             u_d = (o_d + i_d) h - pos[a][d].
 *  Functions  phi_n(u) = (sigma sqrt(pi) 2^n n!)^(-1/2) H_n(u/sigma) exp(-u^2 / 2 sigma^2)
 *             (eq. 1HO-eigenstate, Sec. 2.2, normalised; the paper leaves the factor out and folds it
 *             into the atomic matrix, Sec. 3.7), three of them multiplied per state
 *             (eq. SHO-factorizable-basis).
 *  Basis      all (nx, ny, nz) with nx + ny + nz <= numax (eq. SHO-basis, Sec. 2.5), N =
 *             (numax+1)(numax+2)(numax+3)/6 states (eq. SHO_basis_size), enumerated nz outer,
 *             ny middle, nx inner.  Coefficients are stored coeff[a][k][b], bands innermost.
 *  Memory     every array pointer except pos/sigma is a DEVICE pointer (cudaMalloc / torch); the
 *             caller owns all buffers and the library never frees or retains them after the call's
 *             work has completed on `stream`.
 *  Streams    `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls are
 *             asynchronous: they enqueue work and return.  A handle orders its own calls (each call
 *             waits for the handle's previous call), so one handle may be used from several streams,
 *             but not from several host threads at once.
 *  Errors     every call returns SHO_OK (0) or a negative sho_status.  Argument errors are detected
 *             on the host before anything is enqueued; nothing is written then.  CUDA launch errors
 *             return SHO_ERR_CUDA.  Errors raised later on the device are reported by sho_sync().
 *  Precision  sho_prec selects the arithmetic of the contractions.  SHO_P_FP64 and SHO_P_FF64 need
 *             FP64 psi and coefficients.  The other forms take FP32 or BF16 psi and FP32 coefficients
 *             and keep the 1D function tables in FP64 until they are rounded to the contraction type.
 */
#ifndef SHO_H
#define SHO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SHO_VERSION 1
#define SHO_MAX_NUMAX 9      /* largest numax of projection / expansion (forces use numax + 1) */

typedef enum {
  SHO_OK = 0,
  SHO_ERR_ARG = -1,        /* null pointer, negative size, unknown enum value */
  SHO_ERR_NUMAX = -2,      /* numax outside [0, SHO_MAX_NUMAX] */
  SHO_ERR_CUBE = -3,       /* cube not a multiple of 8 in [8, 64], or larger than a grid dimension */
  SHO_ERR_SPACING = -4,    /* h > h_max = pi sigma / sqrt(2 numax + 1) (eq. max_grid_spacing),
                              returned only in strict mode (sho_set_strict) */
  SHO_ERR_DTYPE = -5,      /* dtype / precision combination not supported */
  SHO_ERR_OOM = -6,        /* device or pinned host allocation failed */
  SHO_ERR_CUDA = -7,       /* a CUDA runtime call or launch failed */
  SHO_ERR_TIMEOUT = -8,    /* a bounded wait ran out: a host wait (serving) or a kernel's wait on its
                              own data pipeline (reported by sho_sync) */
  SHO_ERR_DEVICE = -9,     /* a device-side check failed (reported by sho_sync): an SHO_P_FF64 input
                              outside the float-pair range */
  SHO_ERR_CAPACITY = -10,  /* serving admission: request can never fit the memory budget */
  SHO_ERR_STATE = -11,     /* unknown ticket / system, or call not valid in the current state */
  SHO_ERR_CANCELLED = -12  /* serving: the request was cancelled before it started (sho_cancel) */
} sho_status;

typedef enum { SHO_F64 = 0, SHO_F32 = 1, SHO_BF16 = 2 } sho_dtype;

typedef enum {
  SHO_P_FP64 = 0,        /* FP64 throughout (FP64 psi and coefficients) */
  SHO_P_FP32 = 1,        /* FP32 CUDA-core contractions, FP32 accumulation */
  SHO_P_TF32 = 2,        /* x-pass on TF32 tensor cores, FP32 accumulation */
  SHO_P_3XTF32 = 3,      /* x-pass as three TF32 products (hi*hi + hi*lo + lo*hi), FP32 accumulation */
  SHO_P_BF16 = 4,        /* x-pass on BF16 tensor cores, FP32 accumulation */
  SHO_P_SPLIT_FP16 = 5,  /* x-pass as three FP16 products of a hi/lo split, FP32 accumulation */
  SHO_P_FF64 = 6         /* FP64-accurate: FP64 psi and coefficients, x-pass as float-float
                            (double-FP32) dot products on the FP32 pipe, y/z passes and accumulation in
                            FP64.  Range: every nonzero psi value (projection, forces) and every z-pass
                            sum of the coefficients (expansion) must lie in [2^-126, 2^128) in magnitude.
                            The kernels check this on the device; a call that meets a value outside the
                            range completes, but its results are not FP64-accurate and sho_sync returns
                            SHO_ERR_DEVICE.  Such data needs SHO_P_FP64. */
} sho_prec;

typedef struct {
  int n[3];       /* grid points along x, y, z */
  double h;       /* grid spacing (Bohr) */
  int periodic;   /* 1: cube indices wrap around the grid; 0: points outside the grid are dropped */
} sho_grid;

typedef struct sho_handle sho_handle;

/* Library version (SHO_VERSION). */
int sho_version(void);

/* Basis size (numax+1)(numax+2)(numax+3)/6, eq. SHO_basis_size (Sec. 2.5); 0 for numax < 0. */
int sho_nstates(int numax);

/* Largest grid spacing that samples states up to numax without aliasing:
 * h_max = pi sigma / sqrt(2 numax + 1), eq. max_grid_spacing (Sec. 3.6). */
double sho_max_spacing(double sigma, int numax);

/* Static description of a status code (never NULL). */
const char* sho_strerror(int status);

/* Create a handle bound to CUDA device `device` (made current during each call).  The handle owns
 * a device workspace that grows on demand and is freed by sho_destroy. */
int sho_create(sho_handle** out, int device);

/* Wait for the handle's outstanding work, free its workspace and the handle. */
int sho_destroy(sho_handle* handle);

/* Text of the CUDA error behind the handle's most recent SHO_ERR_CUDA ("no error" when none); a
 * diagnostic, valid until the next call on the handle. */
const char* sho_last_cuda_error(const sho_handle* handle);

/* strict != 0: a spacing above h_max (eq. max_grid_spacing) is an error (SHO_ERR_SPACING); default 0
 * (allowed: the method still computes the defined sums, only their sampling is coarse). */
int sho_set_strict(sho_handle* handle, int strict);

/* Spherical projector support (the paper projects over spheres of radius R_prj around each atom, Sec. 6):
 * with rprj > 0 the handle's projections, expansions, forces, non-local actions and stored-projector
 * builds use only the cube points whose offset u from the atom satisfies
 *     (ux*ux + uy*uy) + uz*uz <= rprj*rprj      (each product and sum rounded to FP64 in that order)
 * -- the cube stays the outer bound, so a sphere wider than the cube changes nothing.  Forces hold the
 * set of included points fixed (as they hold the cube origin).  rprj = 0 restores the whole cube
 * (default); negative or non-finite values return SHO_ERR_ARG.  Implemented by SHO_P_FP64 and
 * SHO_P_FF64 (and sho_usu_build, which stores zeros outside the sphere); the other precision forms and
 * the Bloch entry points return SHO_ERR_DTYPE while a radius is set.  The points inside a sphere form
 * one contiguous run of each cube row, and the kernels skip the rest. */
int sho_set_support_radius(sho_handle* handle, double rprj);

/* Engine of the x-pass of the handle's TF32 / BF16 expansions (FP32 or BF16 psi, numax <= 7, bands in
 * whole 16-byte rows, no spherical support): SHO_KERNEL_AUTO (default) and SHO_KERNEL_TCGEN05 take the
 * fifth-generation tensor cores -- tiles of 8 rows x 32 points x 128 bands whose update stays in tensor
 * memory across the atoms, one M=128 N=32 MMA per row and atom; SHO_KERNEL_MMA_SYNC takes the warp-level
 * MMA kernel (tiles of 8 rows x 32 points x 32 bands, accumulators in registers).  Both add the same
 * products in the same atom order; the FP32 sums of the tensor cores may round differently.
 * For SHO_P_FF64 expansions SHO_KERNEL_TCGEN05, and SHO_KERNEL_AUTO (default) when the band count fills
 * its 128-band tiles at least three quarters (real bands; a complex band counts two), take the x-pass to
 * the tensor cores by exact digit slicing (Ozaki scheme: six 8-bit digits of T1 and of the x functions on fixed
 * power-of-two frames, TF32 MMAs whose leading level sums are exact integers; a persistent kernel with
 * list, digit, MMA and read-back warps) where it applies -- numax <= 7, cube <= 32 and even, an even band
 * count, a periodic grid at least cube + 32 points wide along x, at most 204 / (numax + 1) atoms per z
 * plane, no spherical support, device checks off; real or Bloch data); SHO_KERNEL_MMA_SYNC, and every
 * other case, takes the float-float CUDA-core block gather.  The tensor-core form's error is about 2^-44 of each
 * point's frame (a power of two above the largest single-atom contribution there), against 2^-48 of the
 * point's own terms for the float-float kernel; both are far inside the FP64 tolerance of 1e-12.
 * Other calls ignore the setting.  SHO_ERR_ARG for an unknown value. */
typedef enum { SHO_KERNEL_AUTO = 0, SHO_KERNEL_MMA_SYNC = 1, SHO_KERNEL_TCGEN05 = 2 } sho_kernel;
int sho_set_expand_kernel(sho_handle* handle, int kernel);

/* Engine of the x-pass of the handle's SHO_P_FF64 projections (sho_project, and the projection inside
 * sho_apply_nonlocal): SHO_KERNEL_AUTO (default) and SHO_KERNEL_MMA_SYNC take the float-float CUDA-core
 * kernel; SHO_KERNEL_TCGEN05 takes the fifth-generation tensor cores by exact digit slicing -- psi cut into
 * six 8-bit digits on a power-of-two frame per (cube row, band, half row of 16 points), the x functions on
 * a frame per atom, BF16 MMAs (M = 128 bands, N = 64 = 7 levels x 8 states, K = 16 points) whose level
 * sums are exact integers, in a persistent kernel with digit, MMA and read-back warps -- where it applies
 * (numax <= 7, cube <= 32, no spherical support, real data, device checks off).  The tensor-core form is
 * correct to the FP64 tolerance (its error about 2^-48 of each half row's frame times sum |phi|) but
 * measured about 20 % slower than the float-float kernel on GB300.  Forces and served requests always use
 * the float-float kernel.  SHO_ERR_ARG for an unknown value or a null handle. */
int sho_set_project_kernel(sho_handle* handle, int kernel);

/* Debug mode (on != 0; off by default): the handle's SHO_P_FP64 and SHO_P_FF64 projection, expansion and
 * forces kernels (the FP64 per-atom projection and row-gather expansion, the float-float projection and
 * block-gather expansion) check every global index of psi, of the coefficients and of their z-pass /
 * per-plane intermediate against the buffer's extent before the access.  An index outside skips the
 * access and latches SHO_ERR_DEVICE, returned by the next sho_sync (a stand-in for an out-of-bounds
 * access that a memory checker would report).  The checked kernels are separate instantiations: with
 * the mode off nothing is checked and nothing is slower.  With the mode on, SHO_P_FF64 expansions run
 * the (checked) float-float block gather whatever sho_set_expand_kernel says.  The z-pass, table,
 * tensor-core, FP32-class, Bloch and serving kernels are not checked.  SHO_ERR_ARG for a null handle. */
int sho_set_device_checks(sho_handle* handle, int on);

/* Block until the handle's enqueued work is complete; return the first device-side error since the
 * previous sho_sync (SHO_ERR_TIMEOUT when a kernel's bounded wait on its own data pipeline expired --
 * its results are then incomplete; SHO_ERR_DEVICE when an SHO_P_FF64 input lay outside its range) or a
 * CUDA error, else SHO_OK.  The device status word is cleared. */
int sho_sync(sho_handle* handle);

/*
 * Projection -- step (1) of the non-local action (Sec. 3.2) with the SHO basis injected (Sec. 3.5):
 *     coeff[a][k][b] = h^3 * sum_{cube points i of atom a} Psi_k(u_i) * psi[j(i)][b]
 * evaluated as three separable passes (x, then y, then z; eq. TuckerTensor, Sec. 3.4) with the 1D
 * functions generated on the fly from the Hermite recursion (Sec. 3.7).
 *   psi    device [n[2]][n[1]][n[0]][nbands], type psi_dtype (read only)
 *   coeff  device [natoms][sho_nstates(numax)][nbands], type coeff_dtype (written, fully)
 * Supported: (SHO_P_FP64 | FF64, psi F64, coeff F64); (SHO_P_FP32 | TF32 | 3XTF32 | BF16 | SPLIT_FP16,
 * psi F32 or BF16, coeff F32).  The tensor-core forms (TF32, 3XTF32, BF16, SPLIT_FP16) need
 * numax <= 7 (SHO_ERR_NUMAX otherwise; for sho_forces numax + 1 <= 7) and a cube that is a multiple
 * of 16 (SHO_ERR_CUBE).  natoms == 0 or nbands == 0 is a no-op returning SHO_OK.
 * Workspace: SHO_P_FF64 keeps the per-plane y-pass sums of every cube in the handle's workspace,
 * natoms * cube * (numax+1)(numax+2)/2 * nbands * 8 bytes (SHO_ERR_OOM when it cannot grow).
 */
int sho_project(sho_handle* handle, const sho_grid* grid, const void* psi, sho_dtype psi_dtype, int nbands,
                int natoms, const double* pos, const double* sigma, int numax, int cube, sho_prec prec,
                void* coeff, sho_dtype coeff_dtype, void* stream);

/* Kernel family sho_project runs for these arguments (a host-side query; no GPU work):
 *   SHO_PATH_PLANE  plane sweep: one CTA per (grid plane, 32 bands) streams the plane's rows once
 *                   through shared memory (TMA) for all atoms whose cubes meet it, then a z-pass per
 *                   atom; taken for psi F32 (16-byte aligned, nbands % 4 == 0), coeff F32, a FP32-class
 *                   form, numax <= 7, cube % 16 == 0, n[0] <= 256 (and cube <= n[0] when periodic)
 *   SHO_PATH_ATOM   per-atom kernels: each (atom, 32 bands, z-slab) streams its own cube
 * Returns SHO_ERR_ARG for a NULL grid. */
typedef enum { SHO_PATH_ATOM = 1, SHO_PATH_PLANE = 2 } sho_path;

/* Host-side check of the plane-sweep plan for a geometry (no GPU work): builds the plan the plane sweep
 * would use and verifies it -- every (atom, cube plane, grid row) covered exactly once, the row segments
 * of each register slot disjoint and ordered, both halves of a wrapped cube in one sweep.  Returns
 * SHO_OK, SHO_ERR_STATE for a violated rule, or an argument error; *nitems / *nsegs (optional) receive
 * the number of plane sweeps (CTA rows of work) and row segments. */
int sho_plane_plan_check(const sho_grid* grid, int natoms, const double* pos, const double* sigma, int cube,
                         int* nitems, int* nsegs);
int sho_project_path(const sho_grid* grid, const void* psi, sho_dtype psi_dtype, int nbands, int numax, int cube,
                     sho_prec prec, sho_dtype coeff_dtype);

/*
 * Expansion -- step (3) of the non-local action (Sec. 3.2), the adjoint of the projection:
 *     psi[j][b] += sum_a sum_{i: j(i) = j} sum_k coeff[a][k][b] * Psi_k(u_i)      (no h^3 factor)
 * so that <P psi, c> = h^3 <psi, E c>.  Evaluated z-pass, y-pass, x-pass.  Every grid row is
 * read and written once, atoms are added in ascending index order: the result is deterministic.
 *   coeff  device [natoms][sho_nstates(numax)][nbands], type coeff_dtype (read only)
 *   psi    device [n[2]][n[1]][n[0]][nbands], type psi_dtype (read-modify-write)
 * Same dtype / precision combinations as sho_project.
 */
int sho_add(sho_handle* handle, const sho_grid* grid, const void* coeff, sho_dtype coeff_dtype, int nbands,
            int natoms, const double* pos, const double* sigma, int numax, int cube, sho_prec prec, void* psi,
            sho_dtype psi_dtype, void* stream);

/*
 * Scaled expansion -- psi = (overwrite ? 0 : psi) + alpha * E c, the expansion of sho_add with the
 * factor alpha applied inside the kernels (to the z-pass table).  With alpha = h^3 this is the adjoint
 * of the projection in the plain grid inner product, <P psi, c> = <psi, h^3 E c> (Sec. 3.2, steps 1
 * and 3), i.e. the gradient of a function of the coefficients with respect to psi.  overwrite != 0
 * first clears the whole psi array on `stream` (points outside every cube end as zero), so the caller
 * needs no separate fill.  alpha must be finite (SHO_ERR_ARG).  alpha = 1, overwrite = 0 is sho_add
 * bit for bit.  Other arguments, dtypes and precisions as sho_add; natoms == 0 with overwrite != 0
 * only clears psi.
 */
int sho_add_scaled(sho_handle* handle, const sho_grid* grid, double alpha, int overwrite, const void* coeff,
                   sho_dtype coeff_dtype, int nbands, int natoms, const double* pos, const double* sigma, int numax,
                   int cube, sho_prec prec, void* psi, sho_dtype psi_dtype, void* stream);

/*
 * Forces -- gradient of a function E(c) of the projection coefficients with respect to the atom
 * positions, the cube origins held fixed:
 *     dEdX[a][d] = sum_b sum_k dEdc[a][k][b] * d coeff[a][k][b] / d pos[a][d]
 * Built from a projection at numax + 1 and the ladder relation of Hermite functions (derivative of
 * the Hermite recursion, Sec. 3.7):  d phi_n / du = (1/sigma) [ sqrt(n/2) phi_{n-1} - sqrt((n+1)/2) phi_{n+1} ],
 * so  d C_n / dX = (1/sigma) [ sqrt((n+1)/2) C_{n+1} - sqrt(n/2) C_{n-1} ]  per axis.
 *   psi    device [n[2]][n[1]][n[0]][nbands], type psi_dtype
 *   dEdc   device [natoms][sho_nstates(numax)][nbands], type coeff_dtype
 *   dEdX   device [natoms][3] double (written); the physical force is -dEdX.
 * numax may be at most SHO_MAX_NUMAX.  The band/state reduction is done in FP64 in a fixed order.
 */
int sho_forces(sho_handle* handle, const sho_grid* grid, const void* psi, sho_dtype psi_dtype, int nbands,
               int natoms, const double* pos, const double* sigma, int numax, int cube, sho_prec prec,
               const void* dEdc, sho_dtype coeff_dtype, double* dEdX, void* stream);

/*
 * Non-local action -- the three steps of Sec. 3.2 with the SHO basis injected (Sec. 3.5):
 *     hpsi[j][b] += sum_a sum_{k,k'} Psi_k(u) D[a][k][k'] c[a][k'][b],   c = projection of psi
 * i.e. projection, multiplication by the atomic matrix (D = U^T F^T D F U of Sec. 3.5, an N x N matrix
 * per atom in the Cartesian SHO basis) and expansion.  The projection and the multiplied coefficients
 * live in the handle's workspace; psi and hpsi may not overlap.
 *   psi    device [n[2]][n[1]][n[0]][nbands], psi_dtype (read only)
 *   D      device [natoms][N][N], coefficient type of `prec` (F64 for FP64 / FF64, F32 otherwise),
 *          row-major D[a][k][k'] with the library's state order
 *   hpsi   device, same shape and dtype as psi (read-modify-write)
 * Same precision / dtype rules as sho_project.
 */
int sho_apply_nonlocal(sho_handle* handle, const sho_grid* grid, const void* psi, sho_dtype psi_dtype, int nbands,
                       int natoms, const double* pos, const double* sigma, int numax, int cube, sho_prec prec,
                       const void* D, void* hpsi, void* stream);

/* ----------------------------------------------------------------------------------------------
 * Bloch (complex) wave functions on a periodic grid.  The SHO states span functions R^3 -> C
 * (Sec. 2.5); for psi(r + T) = e^{i k.T} psi(r) a cube point i outside the cell maps to grid point
 * j(i) = r_i - T_i with the lattice translation T_i = (o + i - j(i)) h (per axis), and
 *     sho_project_bloch   coeff[a][k][b] = h^3 sum_i Psi_k(u_i) e^{+i k.T_i} psi[j(i)][b]
 *     sho_add_bloch       psi[j][b] += sum_a sum_{i: j(i)=j} sum_k coeff[a][k][b] Psi_k(u_i) e^{-i k.T_i}
 * (adjoint in the h^3-weighted complex inner product; k = 0 is the real transform of the real and
 * imaginary parts).  The three-pass form is kept: the phase is a product over the axes and, along each
 * axis, constant on the (at most two) runs of a cube on either side of the cell boundary.
 *   grid   periodic (SHO_ERR_ARG otherwise); sho_add_bloch with SHO_P_FP64 needs n[0] <= 448
 *   kvec   host double[3], the Bloch vector in inverse length units
 *   psi    device complex [n[2]][n[1]][n[0]][nbands] as (re, im) pairs: double for SHO_P_FP64 and
 *          SHO_P_FF64, float for SHO_P_FP32
 *   prec   SHO_P_FP64: complex 1D tables (phase included), complex FMAs on the FP64 pipe;
 *          SHO_P_FF64: the real FP64-accurate kernels (float-float x- and y-passes, FP64 z-pass) over
 *          the (re, im) pairs as 2 nbands real bands, each x-pass sum turned by its run's phase in
 *          float pairs -- same accuracy class and input range as SHO_P_FF64 of sho_project (an input
 *          outside it latches SHO_ERR_DEVICE), and the same workspace for 2 nbands bands;
 *          SHO_P_FP32: the real FP32 CUDA-core kernels (streaming projection, block gather) over the
 *          (re, im) pairs as 2 nbands real bands, each x-pass sum (projection) or y-pass result
 *          (expansion) turned by its run's phase in FP32; psi 16-byte aligned and nbands even
 *          (SHO_ERR_ARG otherwise); the FP32 accuracy class of sho_project with SHO_P_FP32;
 *          any other value: SHO_ERR_DTYPE
 *   coeff  device complex [natoms][sho_nstates(numax)][nbands] as (re, im) pairs, of psi's type
 * numax <= 7 (SHO_ERR_NUMAX).  Deterministic (fixed summation order, no atomics).
 */
int sho_project_bloch(sho_handle* handle, const sho_grid* grid, const double* kvec, const void* psi, int nbands,
                      int natoms, const double* pos, const double* sigma, int numax, int cube, sho_prec prec,
                      void* coeff, void* stream);
int sho_add_bloch(sho_handle* handle, const sho_grid* grid, const double* kvec, const void* coeff, int nbands,
                  int natoms, const double* pos, const double* sigma, int numax, int cube, sho_prec prec, void* psi,
                  void* stream);

/* ----------------------------------------------------------------------------------------------
 * Cartesian <-> radial SHO coefficients -- eq. SHO-transform-Cartesian-to-radial (Sec. 2.4): within an
 * energy shell nx + ny + nz = 2 nr + l the Cartesian states (Sec. 2.2) and the radial states
 * Psi_{nr l m} = R_{nr l}(r) Y_{l m} (eq. SHO-eigenstate-radial, Sec. 2.3) span the same space, related
 * by the orthogonal, shell-block-diagonal U[k][j] = <Psi_j^rad | Psi_k^cart>.  Conventions: real Y_{l m}
 * from the complex ones with the Condon-Shortley phase (m > 0: sqrt(2)(-1)^m Re Y_l^m, m < 0:
 * sqrt(2)(-1)^m Im Y_l^|m|, so l = 1, m = +1 / -1 / 0 are x / y / z); R_{nr l} ~ r^l L_nr^(l+1/2)(r^2/sigma^2)
 * e^{-r^2/2sigma^2} normalised and positive at the origin; radial order nu ascending, then l ascending
 * (l = nu mod 2 .. nu), then m = -l .. l.  U does not depend on sigma.
 *   sho_radial_labels   host: nr[j], ell[j], m[j] of the N = sho_nstates(numax) radial states
 *   sho_radial_matrix   host: U as N x N doubles, row-major U[k * N + j] (k Cartesian, library order)
 *   sho_radial_transform  device arrays [natoms][N][nbands] of dtype F64 or F32, in != out:
 *       direction 0 (Cartesian -> radial)  out[a][j][b] = sum_k U[k][j] in[a][k][b]
 *       direction 1 (radial -> Cartesian)  out[a][k][b] = sum_j U[k][j] in[a][j][b]  (the inverse)
 * numax <= SHO_MAX_NUMAX (SHO_ERR_NUMAX).  The handle caches the device copy of U per numax.
 */
int sho_radial_labels(int numax, int* nr, int* ell, int* m);
int sho_radial_matrix(int numax, double* U);
int sho_radial_transform(sho_handle* handle, int natoms, int numax, int nbands, const void* in, void* out,
                         sho_dtype dtype, int direction, void* stream);

/* ----------------------------------------------------------------------------------------------
 * Stored-projector baseline: the conventional scheme the paper measures against ("USU", Sec. 6,
 * Tables 1 and 2, in double and float): projector values sampled once onto each atom's cube and kept in
 * device memory, then streamed by the projection and expansion.  With the stored values taken from the
 * SHO basis the results equal sho_project / sho_add (up to rounding order).
 *   numax  basis the stored projectors are sampled from (numax <= SHO_USU_MAX_NUMAX)
 *   nproj  number of stored projectors: the first nproj states of that basis; one of 1, 4, 10, 18, 20,
 *          35, 56 (the SHO sizes of numax 0..5, and 18 = the s, s*, p, p*, d, d* set of Sec. 6)
 *   dtype  SHO_F64 or SHO_F32: type of proj, psi and coeff alike (and of the arithmetic)
 *   proj   device [natoms][cube^3][nproj], cube point index (iz*cube + iy)*cube + ix; written by
 *          sho_usu_build, read by the other two (caller allocates sizeof(dtype) * A * C^3 * nproj bytes)
 *   psi, coeff as for sho_project / sho_add ([A][nproj][B]).  pos / sigma host arrays.
 */
#define SHO_USU_MAX_NUMAX 5
int sho_usu_build(sho_handle* handle, const sho_grid* grid, int natoms, const double* pos, const double* sigma,
                  int numax, int nproj, int cube, sho_dtype dtype, void* proj, void* stream);
int sho_usu_project(sho_handle* handle, const sho_grid* grid, const void* psi, int nbands, int natoms,
                    const double* pos, const double* sigma, int nproj, int cube, sho_dtype dtype, const void* proj,
                    void* coeff, void* stream);
int sho_usu_add(sho_handle* handle, const sho_grid* grid, const void* coeff, int nbands, int natoms,
                const double* pos, const double* sigma, int nproj, int cube, sho_dtype dtype, const void* proj,
                void* psi, void* stream);

/* ----------------------------------------------------------------------------------------------
 * Serving: a continuous-batching request loop over device-resident systems.  (The paper applies the
 * non-local operator inside an iterative eigensolver, Sec. 3.2; serving many independent systems
 * with one GPU is this library's deployment form of the same two operations.)
 *
 * A server owns `slots` execution slots (a CUDA stream and a workspace each) and one scheduler
 * thread.  Systems are registered once: the server copies psi into device memory it owns and
 * allocates the coefficients, so both stay resident between requests.  Requests (project: psi ->
 * coeff; expand: psi += E coeff) are queued by sho_submit and started by the scheduler as soon as a
 * slot is free, the request's workspace fits the memory budget next to the resident systems and
 * in-flight workspaces, and no earlier request of the same system is still running (requests of one
 * system run in submission order; requests of different systems overlap on the device).  When several
 * requests are startable the scheduler takes the one with the smallest expected service time (its
 * algorithmic bytes at 500 GB/s) minus the time it has already waited: small requests do not queue
 * behind large ones, and a large one waits at most about its own service time longer.  Results of
 * a request do not depend on what else runs: every kernel is deterministic and works on its own
 * system's buffers.
 *   budget_bytes  device memory the server may hold: resident systems + slot workspaces.
 *   errors        sho_system_register returns SHO_ERR_CAPACITY when the system does not fit the
 *                 budget; sho_submit returns SHO_ERR_CAPACITY when the request could never be admitted
 *                 and SHO_ERR_STATE for an unknown system; sho_wait returns SHO_ERR_TIMEOUT when the
 *                 ticket is not complete within timeout_ms (the request keeps running), or the
 *                 request's own error status.
 */
typedef struct sho_server sho_server;

typedef enum { SHO_OP_PROJECT = 0, SHO_OP_EXPAND = 1 } sho_op;

typedef struct {
  uint64_t submitted;        /* requests accepted by sho_submit */
  uint64_t completed;        /* requests finished (successfully or not) */
  uint64_t failed;           /* requests that finished with an error */
  double p50_ms, p99_ms;     /* latency percentiles (submit -> completion seen by the scheduler) */
  double mean_ms, max_ms;
  double busy_seconds;       /* wall time from the first admission to the last completion */
  double algorithmic_bytes;  /* psi and coefficient bytes of the completed requests */
  double gbs;                /* algorithmic_bytes / busy_seconds / 1e9 */
  size_t resident_bytes;     /* device memory of the registered systems */
  size_t workspace_bytes;    /* device memory of the slot workspaces */
  size_t peak_bytes;         /* peak of resident + workspace */
  int max_inflight;          /* most requests running at the same time */
} sho_server_stats;

int sho_server_create(sho_server** out, int device, size_t budget_bytes, int slots);
/* Waits (bounded by each request finishing) for running requests, drops queued ones, frees everything. */
int sho_server_destroy(sho_server* server);
/* Register a system.  psi: [n[2]][n[1]][n[0]][nbands] of psi_dtype at any address cudaMemcpy accepts
 * (host or device); it is copied.  Coefficients (FP64 for F64 psi, FP32 otherwise) start at zero. */
int sho_system_register(sho_server* server, const sho_grid* grid, int nbands, int natoms, const double* pos,
                        const double* sigma, int numax, int cube, sho_dtype psi_dtype, const void* psi,
                        int* system_id);
/* Remove a system once its requests are done (SHO_ERR_STATE while any is queued or running). */
int sho_system_unregister(sho_server* server, int system_id);
/* Copy a system's psi and/or coefficients (either pointer may be NULL) to any address cudaMemcpy
 * accepts, or its coefficients from one; waits for the system's requests to finish first. */
int sho_system_read(sho_server* server, int system_id, void* psi_out, void* coeff_out);
int sho_system_write_coeff(sho_server* server, int system_id, const void* coeff_in);
/* Queue a request; *ticket identifies it for sho_wait. */
int sho_submit(sho_server* server, int system_id, sho_op op, sho_prec prec, uint64_t* ticket);
int sho_wait(sho_server* server, uint64_t ticket, int timeout_ms);
/* sho_wait with the two outcomes kept apart: returns SHO_OK once the request is complete and stores its
 * status in *request_status (the ticket is then released; a request whose kernel's bounded wait expired
 * has status SHO_ERR_TIMEOUT, one whose SHO_P_FF64 input was out of range SHO_ERR_DEVICE) and, when
 * latency_ms is not NULL, its latency (submission to completion seen by the scheduler, ms; 0 for a
 * cancelled request); or SHO_ERR_TIMEOUT when it is not complete within timeout_ms (the ticket stays
 * valid). */
int sho_wait_status(sho_server* server, uint64_t ticket, int timeout_ms, int* request_status, double* latency_ms);
/* Cancel a queued request: it is removed from the queue and never starts; a later sho_wait on its
 * ticket returns SHO_ERR_CANCELLED.  Returns SHO_OK, or SHO_ERR_STATE when the ticket is unknown, has
 * already started (GPU work is not interrupted) or has finished. */
int sho_cancel(sho_server* server, uint64_t ticket);
int sho_server_get_stats(sho_server* server, sho_server_stats* stats);
/* Clear latency records and counters (not the systems). */
int sho_server_reset_stats(sho_server* server);

/* Size of the fixed device scratch array of sho_forces_noalloc: 16 MiB. */
#define SHO_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)

/*
 * Allocation-free forces.  The paper has no counterpart to this entry point; it exists for callers
 * that cannot let a library allocate device memory -- for example an application whose own pool
 * allocator owns all device memory, a plug-in inside a host program that forbids foreign
 * allocations, or a process so close to its memory limit that an allocation could fail mid-step.
 *
 * It computes what sho_forces computes, with the same arguments minus the handle, on the device that
 * is current for the calling thread and on `stream`.  It calls no cudaMalloc, cudaFree or other
 * allocating routine: its scratch (the per-atom plan and the numax+1 projection) is one file-scope
 * static device array of SHO_NOALLOC_SCRATCH_BYTES, loaded with the library, which every GPU that
 * loads libsho.so holds until the process exits.
 *   limit     ceil256(48 * natoms) + natoms * sho_nstates(numax + 1) * nbands * s <= SHO_NOALLOC_SCRATCH_BYTES,
 *             s = 8 for SHO_P_FP64 and 4 for SHO_P_FP32; larger problems return SHO_ERR_CAPACITY before
 *             anything is enqueued.
 *   set-up    the first call on a device looks up the array's device address once (the device must be
 *             current, which it is for that call).
 *   sharing   all calls on a device share the array and it keeps the last call's contents; each call
 *             writes every scratch element before reading it, so nothing needs clearing.  Calls whose
 *             GPU work overlaps (different streams with no ordering between them) race on the array:
 *             order them, for instance on one stream.
 * Precisions: SHO_P_FP64 (psi, dEdc F64) and SHO_P_FP32 (psi F32/BF16, dEdc F32).
 */
int sho_forces_noalloc(const sho_grid* grid, const void* psi, sho_dtype psi_dtype, int nbands, int natoms,
                       const double* pos, const double* sigma, int numax, int cube, sho_prec prec,
                       const void* dEdc, sho_dtype coeff_dtype, double* dEdX, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SHO_H */
