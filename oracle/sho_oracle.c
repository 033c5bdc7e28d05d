/*
 * sho_oracle.c -- plain, slow, FP64 CPU oracle for SHO projection, expansion and forces.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this file's library.  The product path (the CUDA library) shares no code,
 * header, table or constant with it, and never calls it.
 *
 * What it computes (Baumeister & Tsukamoto, PASC'19, "Analytical PAW Projector Functions"):
 *
 *   1D functions  (Sec. 2.2, eq. 1HO-eigenstate): psi_n(x) ~ H_n(x/sigma) exp(-x^2 / 2 sigma^2), with
 *                 H_n the Hermite polynomials.  The paper omits the normalising factor (Sec. 2.2, and
 *                 Sec. 3.7 says it can be folded into the atomic matrix); this oracle uses the
 *                 L2-normalised functions
 *                     phi_n(u) = (sigma sqrt(pi) 2^n n!)^(-1/2) H_n(u/sigma) exp(-u^2 / 2 sigma^2)
 *                 with physicists' H_n.  (The monic recursion of Sec. 3.7 gives h_n = H_n / 2^n, so the
 *                 normalised function is the same in either convention.)
 *   3D projector  (Sec. 2.2, eq. SHO-eigenstate-Cartesian): the product of three 1D polynomials times a
 *                 single 3D Gaussian exp(-|u|^2 / 2 sigma^2), sampled directly at every cube point.
 *   Basis         (Sec. 2.5, eq. SHO-basis / SHO_basis_size): all (nx,ny,nz) with nx+ny+nz <= numax,
 *                 (numax+1)(numax+2)(numax+3)/6 states, enumerated nz outer, ny middle, nx inner.
 *   Projection    (Sec. 3.2 step 1, Sec. 3.5): c[a][k][b] = h^3 sum_{cube points i} Psi_k(u_i) psi[j(i)][b].
 *   Expansion     (Sec. 3.2 step 3): psi[j][b] += sum_a sum_{i: j(i)=j} sum_k c[a][k][b] Psi_k(u_i)
 *                 (no h^3 factor), atoms added in ascending index order.
 *   Forces        dE/dX_a = sum_b sum_k dEdc[a][k][b] dc[a][k][b]/dX_a, with the derivative of the 3D
 *                 projector taken analytically (d/dX = -d/du, physicists' H_n' = 2n H_{n-1}); the cube
 *                 origin is held fixed (it is piecewise constant in X).
 *
 * Geometry (the paper states no grid convention; this is the reading used throughout):
 *   grid point j = (jx,jy,jz) sits at r_j = h*j, j_d in [0, N_d); psi is stored psi[jz][jy][jx][b].
 *   atom a at X_a, cube edge C (points).  Per axis the cube origin is o_d = floor(X_d / h) - C/2 + 1
 *   and cube point i_d in [0, C) maps to grid index (o_d + i_d) mod N_d when periodic; when not
 *   periodic, points outside [0, N_d) contribute nothing.  The offset used in the functions is the
 *   unwrapped u_d = (o_d + i_d)*h - X_d.
 *
 * 1D polynomials are evaluated by the explicit power sum in long double -- deliberately not by the
 * three-term recursion -- and the 3D Gaussian by one exponential per point.
 *
 * Spherical support (the *_r entry points; the paper projects over spheres of radius R_prj around the
 * atoms, Sec. 6): with rprj > 0 only cube points whose offset lies in the sphere contribute,
 *     (ux*ux + uy*uy) + uz*uz <= rprj*rprj,
 * each product and sum rounded to FP64 in that order (the library decides boundary points the same
 * way); rprj <= 0 is the plain cube.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#define ORACLE_MAX_NUMAX 16

#ifdef _OPENMP
#include <omp.h>
#endif

/* Number of OpenMP threads the oracle uses (for timing it on one core and on all cores). */
int oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

int oracle_nstates(int numax) {
  if (numax < 0) return 0;
  return (numax + 1) * (numax + 2) * (numax + 3) / 6;
}

/* Basis enumeration: k runs over nz outer, ny middle, nx inner with nx+ny+nz <= numax. */
int oracle_basis(int numax, int* nxyz /* [N][3] out */) {
  int k = 0;
  for (int nz = 0; nz <= numax; nz++)
    for (int ny = 0; ny <= numax - nz; ny++)
      for (int nx = 0; nx <= numax - nz - ny; nx++) {
        nxyz[3 * k + 0] = nx;
        nxyz[3 * k + 1] = ny;
        nxyz[3 * k + 2] = nz;
        k++;
      }
  return k;
}

static long double factorial_ld(int n) {
  long double f = 1.0L;
  for (int i = 2; i <= n; i++) f *= (long double)i;
  return f;
}

/* Physicists' Hermite polynomial from its explicit sum:
 *   H_n(x) = n! * sum_{m=0}^{floor(n/2)} (-1)^m (2x)^(n-2m) / (m! (n-2m)!)            */
static long double hermite_ld(int n, long double x) {
  if (n < 0) return 0.0L;
  long double sum = 0.0L;
  for (int m = 0; 2 * m <= n; m++) {
    long double term = powl(2.0L * x, (long double)(n - 2 * m)) / (factorial_ld(m) * factorial_ld(n - 2 * m));
    sum += (m & 1) ? -term : term;
  }
  return factorial_ld(n) * sum;
}

double oracle_hermite(int n, double x) { return (double)hermite_ld(n, (long double)x); }

/* Normalising constant of the 1D function: (sigma sqrt(pi) 2^n n!)^(-1/2). */
static long double norm_ld(int n, double sigma) {
  const long double pi = 3.141592653589793238462643383279502884L;
  return 1.0L / sqrtl((long double)sigma * sqrtl(pi) * powl(2.0L, (long double)n) * factorial_ld(n));
}

/* The normalised 1D function phi_n(u). */
double oracle_phi(int n, double u, double sigma) {
  long double xi = (long double)u / (long double)sigma;
  return (double)(norm_ld(n, sigma) * hermite_ld(n, xi) * expl(-0.5L * xi * xi));
}

/* Its derivative d phi_n / du (analytic: H_n' = 2n H_{n-1}). */
double oracle_dphi(int n, double u, double sigma) {
  long double xi = (long double)u / (long double)sigma;
  long double d = (2.0L * n * hermite_ld(n - 1, xi) - xi * hermite_ld(n, xi)) / (long double)sigma;
  return (double)(norm_ld(n, sigma) * d * expl(-0.5L * xi * xi));
}

/* Cube origin along one axis: floor(X/h) - C/2 + 1. */
static int cube_origin(double X, double h, int cube) { return (int)floor(X / h) - cube / 2 + 1; }

/* Grid index of cube point i along an axis, or -1 when clipped (non-periodic). */
static int grid_index(int o, int i, int n, int periodic) {
  int j = o + i;
  if (periodic) {
    j %= n;
    if (j < 0) j += n;
    return j;
  }
  return (j >= 0 && j < n) ? j : -1;
}

/* Per-atom sampled data: 1D normalised polynomial values N_n H_n(u/sigma) per axis and cube point,
 * the 3D Gaussian per cube point and the flat grid index per cube point (-1 = clipped). */
typedef struct {
  int cube, numax;
  double* poly[3];   /* [numax+1][cube] */
  double* dpoly[3];  /* [numax+1][cube]: d/du of (N_n H_n(u/sigma) exp(-u^2/2s^2)) / exp(-u^2/2s^2) */
  double* gauss;     /* [cube^3] */
  int64_t* gidx;     /* [cube^3] */
  double shift[3][256]; /* lattice translation (o + i - j) h of cube point i along each axis */
} atom_samples;

/* Is the offset u inside the sphere of radius rprj (always, for rprj <= 0)? */
static int in_sphere(double ux, double uy, double uz, double rprj) {
  if (!(rprj > 0.0)) return 1;
  const double r2 = (ux * ux + uy * uy) + uz * uz;
  return r2 <= rprj * rprj;
}

static void atom_samples_init(atom_samples* s, const int n[3], double h, int periodic, const double X[3],
                              double sigma, int numax, int cube, int with_deriv, double rprj) {
  s->cube = cube;
  s->numax = numax;
  long double sg = (long double)sigma;
  double u[3][256];
  int j[3][256];
  for (int d = 0; d < 3; d++) {
    int o = cube_origin(X[d], h, cube);
    s->poly[d] = (double*)malloc(sizeof(double) * (numax + 1) * cube);
    s->dpoly[d] = with_deriv ? (double*)malloc(sizeof(double) * (numax + 1) * cube) : NULL;
    for (int i = 0; i < cube; i++) {
      u[d][i] = (double)(o + i) * h - X[d];
      j[d][i] = grid_index(o, i, n[d], periodic);
      s->shift[d][i] = j[d][i] < 0 ? 0.0 : (double)(o + i - j[d][i]) * h;
      long double xi = (long double)u[d][i] / sg;
      for (int m = 0; m <= numax; m++) {
        long double nm = norm_ld(m, sigma);
        s->poly[d][m * cube + i] = (double)(nm * hermite_ld(m, xi));
        if (with_deriv)
          s->dpoly[d][m * cube + i] =
              (double)(nm * (2.0L * m * hermite_ld(m - 1, xi) - xi * hermite_ld(m, xi)) / sg);
      }
    }
  }
  int64_t c3 = (int64_t)cube * cube * cube;
  s->gauss = (double*)malloc(sizeof(double) * c3);
  s->gidx = (int64_t*)malloc(sizeof(int64_t) * c3);
  for (int iz = 0; iz < cube; iz++)
    for (int iy = 0; iy < cube; iy++)
      for (int ix = 0; ix < cube; ix++) {
        int64_t i = ((int64_t)iz * cube + iy) * cube + ix;
        long double r2 = (long double)u[0][ix] * u[0][ix] + (long double)u[1][iy] * u[1][iy] +
                         (long double)u[2][iz] * u[2][iz];
        s->gauss[i] = (double)expl(-r2 / (2.0L * sg * sg));
        if (j[0][ix] < 0 || j[1][iy] < 0 || j[2][iz] < 0 || !in_sphere(u[0][ix], u[1][iy], u[2][iz], rprj))
          s->gidx[i] = -1;
        else
          s->gidx[i] = ((int64_t)j[2][iz] * n[1] + j[1][iy]) * n[0] + j[0][ix];
      }
}

static void atom_samples_free(atom_samples* s) {
  for (int d = 0; d < 3; d++) {
    free(s->poly[d]);
    free(s->dpoly[d]);
  }
  free(s->gauss);
  free(s->gidx);
}

/* Fully sampled 3D projector of state (nx,ny,nz) at every cube point. */
static void sample_projector(const atom_samples* s, int nx, int ny, int nz, double* P) {
  int C = s->cube;
  for (int iz = 0; iz < C; iz++)
    for (int iy = 0; iy < C; iy++)
      for (int ix = 0; ix < C; ix++) {
        int64_t i = ((int64_t)iz * C + iy) * C + ix;
        P[i] = s->poly[0][nx * C + ix] * s->poly[1][ny * C + iy] * s->poly[2][nz * C + iz] * s->gauss[i];
      }
}

/* d Psi_k / d X_dir = - d Psi_k / d u_dir at every cube point. */
static void sample_projector_dX(const atom_samples* s, int nx, int ny, int nz, int dir, double* P) {
  int C = s->cube;
  for (int iz = 0; iz < C; iz++)
    for (int iy = 0; iy < C; iy++)
      for (int ix = 0; ix < C; ix++) {
        int64_t i = ((int64_t)iz * C + iy) * C + ix;
        double fx = (dir == 0) ? s->dpoly[0][nx * C + ix] : s->poly[0][nx * C + ix];
        double fy = (dir == 1) ? s->dpoly[1][ny * C + iy] : s->poly[1][ny * C + iy];
        double fz = (dir == 2) ? s->dpoly[2][nz * C + iz] : s->poly[2][nz * C + iz];
        P[i] = -(fx * fy * fz * s->gauss[i]);
      }
}

static int check_args(const int n[3], double h, int natoms, int numax, int cube, int nbands) {
  if (!n || n[0] <= 0 || n[1] <= 0 || n[2] <= 0) return -1;
  if (!(h > 0.0)) return -1;
  if (natoms < 0 || nbands < 0) return -1;
  if (numax < 0 || numax > ORACLE_MAX_NUMAX) return -2;
  if (cube <= 0 || cube > 256 || (cube & 1)) return -3;
  return 0;
}

/* Projection: coeff[a][k][b] = h^3 sum_i Psi_k(u_i) psi[j(i)][b].  Loop order atoms -> k -> cube
 * points -> bands.  Returns 0 or a negative error. */
int oracle_project_r(const int n[3], double h, int periodic, const double* psi, int nbands, int natoms,
                     const double* pos, const double* sigma, int numax, int cube, double rprj, double* coeff) {
  int err = check_args(n, h, natoms, numax, cube, nbands);
  if (err) return err;
  int N = oracle_nstates(numax);
  int* nxyz = (int*)malloc(sizeof(int) * 3 * N);
  oracle_basis(numax, nxyz);
  const double h3 = h * h * h;
  const int64_t c3 = (int64_t)cube * cube * cube;
#pragma omp parallel for schedule(dynamic, 1)
  for (int a = 0; a < natoms; a++) {
    atom_samples s;
    atom_samples_init(&s, n, h, periodic, pos + 3 * a, sigma[a], numax, cube, 0, rprj);
    double* P = (double*)malloc(sizeof(double) * c3);
    double* acc = (double*)malloc(sizeof(double) * (nbands > 0 ? nbands : 1));
    for (int k = 0; k < N; k++) {
      sample_projector(&s, nxyz[3 * k], nxyz[3 * k + 1], nxyz[3 * k + 2], P);
      for (int b = 0; b < nbands; b++) acc[b] = 0.0;
      for (int64_t i = 0; i < c3; i++) {
        if (s.gidx[i] < 0) continue;
        const double* row = psi + s.gidx[i] * nbands;
        double w = P[i];
        for (int b = 0; b < nbands; b++) acc[b] += w * row[b];
      }
      double* out = coeff + ((int64_t)a * N + k) * nbands;
      for (int b = 0; b < nbands; b++) out[b] = h3 * acc[b];
    }
    free(acc);
    free(P);
    atom_samples_free(&s);
  }
  free(nxyz);
  return 0;
}

/* Expansion: psi[j][b] += sum_a sum_{i: j(i)=j} sum_k coeff[a][k][b] Psi_k(u_i).  Atoms are added one
 * after another in ascending order; within an atom the cube points map to distinct grid points, so
 * they are processed in parallel without conflict. */
int oracle_project(const int n[3], double h, int periodic, const double* psi, int nbands, int natoms,
                   const double* pos, const double* sigma, int numax, int cube, double* coeff) {
  return oracle_project_r(n, h, periodic, psi, nbands, natoms, pos, sigma, numax, cube, 0.0, coeff);
}

int oracle_add_r(const int n[3], double h, int periodic, double* psi, int nbands, int natoms, const double* pos,
                 const double* sigma, int numax, int cube, double rprj, const double* coeff) {
  int err = check_args(n, h, natoms, numax, cube, nbands);
  if (err) return err;
  if (cube > n[0] || cube > n[1] || cube > n[2]) {
    if (periodic) return -3; /* a wrapped cube would hit one grid point twice */
  }
  int N = oracle_nstates(numax);
  int* nxyz = (int*)malloc(sizeof(int) * 3 * N);
  oracle_basis(numax, nxyz);
  const int64_t c3 = (int64_t)cube * cube * cube;
  double* P = (double*)malloc(sizeof(double) * c3 * N);
  for (int a = 0; a < natoms; a++) {
    atom_samples s;
    atom_samples_init(&s, n, h, periodic, pos + 3 * a, sigma[a], numax, cube, 0, rprj);
    for (int k = 0; k < N; k++) sample_projector(&s, nxyz[3 * k], nxyz[3 * k + 1], nxyz[3 * k + 2], P + k * c3);
    const double* ca = coeff + (int64_t)a * N * nbands;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c3; i++) {
      if (s.gidx[i] < 0) continue;
      double* row = psi + s.gidx[i] * nbands;
      for (int b = 0; b < nbands; b++) {
        double sum = 0.0;
        for (int k = 0; k < N; k++) sum += ca[(int64_t)k * nbands + b] * P[k * c3 + i];
        row[b] += sum;
      }
    }
    atom_samples_free(&s);
  }
  free(P);
  free(nxyz);
  return 0;
}

/* Expansion evaluated only at selected grid points: out[p][b] = sum_a sum_k coeff[a][k][b] Psi_k(u)
 * for every atom whose cube holds grid point flat index pts[p] (atoms in ascending order).  Used to
 * check full-size expansions point by point. */
int oracle_add(const int n[3], double h, int periodic, double* psi, int nbands, int natoms, const double* pos,
               const double* sigma, int numax, int cube, const double* coeff) {
  return oracle_add_r(n, h, periodic, psi, nbands, natoms, pos, sigma, numax, cube, 0.0, coeff);
}

int oracle_expand_points_r(const int n[3], double h, int periodic, int nbands, int natoms, const double* pos,
                           const double* sigma, int numax, int cube, double rprj, const double* coeff, int npts,
                           const int64_t* pts, double* out) {
  int err = check_args(n, h, natoms, numax, cube, nbands);
  if (err) return err;
  int N = oracle_nstates(numax);
  int* nxyz = (int*)malloc(sizeof(int) * 3 * N);
  oracle_basis(numax, nxyz);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int64_t q = 0; q < (int64_t)npts * nbands; q++) out[q] = 0.0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int p = 0; p < npts; p++) {
    int64_t g = pts[p];
    int jx = (int)(g % n[0]), jy = (int)((g / n[0]) % n[1]), jz = (int)(g / ((int64_t)n[0] * n[1]));
    int jd[3] = {jx, jy, jz};
    for (int a = 0; a < natoms; a++) {
      const double* X = pos + 3 * a;
      double u[3];
      int inside = 1;
      for (int d = 0; d < 3; d++) {
        int o = cube_origin(X[d], h, cube);
        int i;
        if (periodic) {
          i = (jd[d] - o) % n[d];
          if (i < 0) i += n[d];
        } else {
          i = jd[d] - o;
        }
        if (i < 0 || i >= cube) {
          inside = 0;
          break;
        }
        u[d] = (double)(o + i) * h - X[d];
      }
      if (!inside || !in_sphere(u[0], u[1], u[2], rprj)) continue;
      long double sg = sigma[a];
      long double r2 = (long double)u[0] * u[0] + (long double)u[1] * u[1] + (long double)u[2] * u[2];
      long double g3 = expl(-r2 / (2.0L * sg * sg));
      for (int k = 0; k < N; k++) {
        int m[3] = {nxyz[3 * k], nxyz[3 * k + 1], nxyz[3 * k + 2]};
        long double v = g3;
        for (int d = 0; d < 3; d++) {
          long double nm = 1.0L / sqrtl(sg * sqrtl(pi) * powl(2.0L, (long double)m[d]) * factorial_ld(m[d]));
          v *= nm * hermite_ld(m[d], (long double)u[d] / sg);
        }
        double w = (double)v;
        const double* ck = coeff + ((int64_t)a * N + k) * nbands;
        for (int b = 0; b < nbands; b++) out[(int64_t)p * nbands + b] += ck[b] * w;
      }
    }
  }
  free(nxyz);
  return 0;
}

/* Forces: dEdX[a][d] = sum_b sum_k dEdc[a][k][b] * h^3 sum_i dPsi_k/dX_d(u_i) psi[j(i)][b]. */
int oracle_forces_r(const int n[3], double h, int periodic, const double* psi, int nbands, int natoms,
                    const double* pos, const double* sigma, int numax, int cube, double rprj, const double* dEdc,
                    double* dEdX) {
  int err = check_args(n, h, natoms, numax, cube, nbands);
  if (err) return err;
  int N = oracle_nstates(numax);
  int* nxyz = (int*)malloc(sizeof(int) * 3 * N);
  oracle_basis(numax, nxyz);
  const double h3 = h * h * h;
  const int64_t c3 = (int64_t)cube * cube * cube;
#pragma omp parallel for schedule(dynamic, 1)
  for (int a = 0; a < natoms; a++) {
    atom_samples s;
    atom_samples_init(&s, n, h, periodic, pos + 3 * a, sigma[a], numax, cube, 1, rprj);
    double* P = (double*)malloc(sizeof(double) * c3);
    double* acc = (double*)malloc(sizeof(double) * (nbands > 0 ? nbands : 1));
    for (int d = 0; d < 3; d++) {
      double f = 0.0;
      for (int k = 0; k < N; k++) {
        sample_projector_dX(&s, nxyz[3 * k], nxyz[3 * k + 1], nxyz[3 * k + 2], d, P);
        for (int b = 0; b < nbands; b++) acc[b] = 0.0;
        for (int64_t i = 0; i < c3; i++) {
          if (s.gidx[i] < 0) continue;
          const double* row = psi + s.gidx[i] * nbands;
          double w = P[i];
          for (int b = 0; b < nbands; b++) acc[b] += w * row[b];
        }
        const double* g = dEdc + ((int64_t)a * N + k) * nbands;
        for (int b = 0; b < nbands; b++) f += g[b] * h3 * acc[b];
      }
      dEdX[3 * a + d] = f;
    }
    free(acc);
    free(P);
    atom_samples_free(&s);
  }
  free(nxyz);
  return 0;
}

/* Forces for spherical support hold the set of included points fixed, as they hold the cube origin. */
int oracle_forces(const int n[3], double h, int periodic, const double* psi, int nbands, int natoms,
                  const double* pos, const double* sigma, int numax, int cube, const double* dEdc,
                  double* dEdX) {
  return oracle_forces_r(n, h, periodic, psi, nbands, natoms, pos, sigma, numax, cube, 0.0, dEdc, dEdX);
}

int oracle_expand_points(const int n[3], double h, int periodic, int nbands, int natoms, const double* pos,
                         const double* sigma, int numax, int cube, const double* coeff, int npts,
                         const int64_t* pts, double* out) {
  return oracle_expand_points_r(n, h, periodic, nbands, natoms, pos, sigma, numax, cube, 0.0, coeff, npts, pts, out);
}


/* ---------------------------------------------------------------------------------------------
 * Bloch (complex) wave functions on a periodic grid.  psi and coeff hold complex numbers as (re, im)
 * pairs: psi[j][b][2], coeff[a][k][b][2].  A cube point i that lies outside the cell maps to grid point
 * j(i) = r_i - T_i with the lattice translation T_i; the Bloch condition psi(r + T) = e^{i k.T} psi(r)
 * gives the value there, so
 *   projection  c[a][k][b] = h^3 sum_i Psi_k(u_i) e^{+i k.T_i} psi[j(i)][b]
 *   expansion   psi[j][b] += sum_a sum_{i: j(i)=j} sum_k c[a][k][b] Psi_k(u_i) e^{-i k.T_i}
 * (adjoint in the complex inner product weighted by h^3; k = 0 gives the real transform of the real
 * and imaginary parts). */
int oracle_project_bloch(const int n[3], double h, const double kvec[3], const double* psi, int nbands, int natoms,
                         const double* pos, const double* sigma, int numax, int cube, double* coeff) {
  int err = check_args(n, h, natoms, numax, cube, nbands);
  if (err) return err;
  int N = oracle_nstates(numax);
  int* nxyz = (int*)malloc(sizeof(int) * 3 * N);
  oracle_basis(numax, nxyz);
  const double h3 = h * h * h;
  const int64_t c3 = (int64_t)cube * cube * cube;
#pragma omp parallel for schedule(dynamic, 1)
  for (int a = 0; a < natoms; a++) {
    atom_samples s;
    atom_samples_init(&s, n, h, 1, pos + 3 * a, sigma[a], numax, cube, 0, 0.0);
    double* P = (double*)malloc(sizeof(double) * c3);
    double* cph = (double*)malloc(sizeof(double) * c3);
    double* sph = (double*)malloc(sizeof(double) * c3);
    for (int iz = 0; iz < cube; iz++)
      for (int iy = 0; iy < cube; iy++)
        for (int ix = 0; ix < cube; ix++) {
          int64_t i = ((int64_t)iz * cube + iy) * cube + ix;
          double th = kvec[0] * s.shift[0][ix] + kvec[1] * s.shift[1][iy] + kvec[2] * s.shift[2][iz];
          cph[i] = cos(th);
          sph[i] = sin(th);
        }
    double* acc = (double*)malloc(sizeof(double) * 2 * (nbands > 0 ? nbands : 1));
    for (int k = 0; k < N; k++) {
      sample_projector(&s, nxyz[3 * k], nxyz[3 * k + 1], nxyz[3 * k + 2], P);
      for (int b = 0; b < 2 * nbands; b++) acc[b] = 0.0;
      for (int64_t i = 0; i < c3; i++) {
        const double* row = psi + s.gidx[i] * 2 * nbands;
        const double wr = P[i] * cph[i], wi = P[i] * sph[i];
        for (int b = 0; b < nbands; b++) {
          const double pr = row[2 * b], pi = row[2 * b + 1];
          acc[2 * b] += wr * pr - wi * pi;
          acc[2 * b + 1] += wr * pi + wi * pr;
        }
      }
      double* out = coeff + ((int64_t)a * N + k) * 2 * nbands;
      for (int b = 0; b < 2 * nbands; b++) out[b] = h3 * acc[b];
    }
    free(acc);
    free(sph);
    free(cph);
    free(P);
    atom_samples_free(&s);
  }
  free(nxyz);
  return 0;
}

int oracle_add_bloch(const int n[3], double h, const double kvec[3], double* psi, int nbands, int natoms,
                     const double* pos, const double* sigma, int numax, int cube, const double* coeff) {
  int err = check_args(n, h, natoms, numax, cube, nbands);
  if (err) return err;
  if (cube > n[0] || cube > n[1] || cube > n[2]) return -3;
  int N = oracle_nstates(numax);
  int* nxyz = (int*)malloc(sizeof(int) * 3 * N);
  oracle_basis(numax, nxyz);
  const int64_t c3 = (int64_t)cube * cube * cube;
  double* P = (double*)malloc(sizeof(double) * c3 * N);
  for (int a = 0; a < natoms; a++) {
    atom_samples s;
    atom_samples_init(&s, n, h, 1, pos + 3 * a, sigma[a], numax, cube, 0, 0.0);
    for (int k = 0; k < N; k++) sample_projector(&s, nxyz[3 * k], nxyz[3 * k + 1], nxyz[3 * k + 2], P + k * c3);
    const double* ca = coeff + (int64_t)a * N * 2 * nbands;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c3; i++) {
      const int ix = (int)(i % cube), iy = (int)((i / cube) % cube), iz = (int)(i / ((int64_t)cube * cube));
      const double th = kvec[0] * s.shift[0][ix] + kvec[1] * s.shift[1][iy] + kvec[2] * s.shift[2][iz];
      const double cr = cos(th), ci = -sin(th);  /* e^{-i k.T} */
      double* row = psi + s.gidx[i] * 2 * nbands;
      for (int b = 0; b < nbands; b++) {
        double sr = 0.0, si = 0.0;
        for (int k = 0; k < N; k++) {
          const double w = P[k * c3 + i];
          sr += ca[((int64_t)k * nbands + b) * 2] * w;
          si += ca[((int64_t)k * nbands + b) * 2 + 1] * w;
        }
        row[2 * b] += sr * cr - si * ci;
        row[2 * b + 1] += sr * ci + si * cr;
      }
    }
    atom_samples_free(&s);
  }
  free(P);
  free(nxyz);
  return 0;
}
