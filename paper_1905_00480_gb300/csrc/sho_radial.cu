// sho_radial.cu -- Cartesian <-> radial SHO coefficients (eq. SHO-transform-Cartesian-to-radial, Sec. 2.4).
//
// Within an energy shell nu = nx + ny + nz = 2 nr + l the Cartesian states Psi_{nx ny nz} (Sec. 2.2) and
// the radial states Psi_{nr l m} = R_{nr l}(r) Y_{l m} (Sec. 2.3) span one space; U[k][j] =
// <Psi_j^rad | Psi_k^cart> is orthogonal and block-diagonal by shell.  It depends on neither sigma nor
// the atom, so it is built once per numax on the host by exact polynomial algebra:
//   Cartesian state  prod_d (sqrt(pi) 2^n n!)^(-1/2) H_n(x_d)        (Hermite by its recursion)
//   radial state     L_nr^(l+1/2)(r^2) S_lm(x, y, z), normalised     (Laguerre by its explicit sum)
//   S_lm             Re / Im (x + i y)^|m| * sum_i d_i z^i r^(l-|m|-i), d = coefficients of the |m|-th
//                    derivative of the Legendre polynomial P_l: the real solid harmonic of the
//                    Condon-Shortley convention up to a positive factor (m > 0: cos, m < 0: sin)
// and every inner product reduces to the Gaussian moments int t^p e^{-t^2} dt = Gamma((p+1)/2).
// Radial order: nu ascending, l ascending (l = nu mod 2 .. nu), m = -l .. l.  The device transform is a
// sparse product per (atom, band): one lane per band, the shell blocks stored as CSR rows.
#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include "sho_device.cuh"

namespace sho {
namespace {

// Sparse polynomial in (x, y, z), exponents below 64.
struct Poly {
  std::map<int, double> c;  // key = (a * 64 + b) * 64 + e  for x^a y^b z^e
  static int key(int a, int b, int e) { return (a * 64 + b) * 64 + e; }
  void add(int a, int b, int e, double v) {
    if (v != 0.0) c[key(a, b, e)] += v;
  }
};

Poly mul(const Poly& p, const Poly& q) {
  Poly r;
  for (const auto& u : p.c)
    for (const auto& v : q.c) {
      const int a = u.first / 4096 + v.first / 4096, b = (u.first / 64) % 64 + (v.first / 64) % 64,
                e = u.first % 64 + v.first % 64;
      r.add(a, b, e, u.second * v.second);
    }
  return r;
}

// int t^p exp(-t^2) dt over the real line
double moment(int p) {
  if (p & 1) return 0.0;
  return std::tgamma(0.5 * (p + 1));
}

// <p e^{-r^2/2}, q e^{-r^2/2}>
double inner(const Poly& p, const Poly& q) {
  double s = 0.0;
  for (const auto& u : p.c)
    for (const auto& v : q.c) {
      const int a = u.first / 4096 + v.first / 4096, b = (u.first / 64) % 64 + (v.first / 64) % 64,
                e = u.first % 64 + v.first % 64;
      if ((a | b | e) & 1) continue;
      s += u.second * v.second * moment(a) * moment(b) * moment(e);
    }
  return s;
}

// Physicists' Hermite polynomial coefficients (H_0 = 1, H_1 = 2t, H_{n+1} = 2t H_n - 2n H_{n-1}).
std::vector<double> hermite_coeffs(int n) {
  std::vector<double> h0(n + 2, 0.0), h1(n + 2, 0.0);
  h0[0] = 1.0;
  if (n == 0) return std::vector<double>(h0.begin(), h0.begin() + 1);
  h1[1] = 2.0;
  for (int k = 1; k < n; k++) {
    std::vector<double> h2(n + 2, 0.0);
    for (int i = 0; i <= k; i++) h2[i + 1] += 2.0 * h1[i];
    for (int i = 0; i <= k - 1; i++) h2[i] -= 2.0 * k * h0[i];
    h0 = h1;
    h1 = h2;
  }
  return std::vector<double>(h1.begin(), h1.begin() + n + 1);
}

// Legendre polynomial coefficients ((l+1) P_{l+1} = (2l+1) t P_l - l P_{l-1}).
std::vector<double> legendre_coeffs(int l) {
  std::vector<double> p0(l + 2, 0.0), p1(l + 2, 0.0);
  p0[0] = 1.0;
  if (l == 0) return std::vector<double>(1, 1.0);
  p1[1] = 1.0;
  for (int k = 1; k < l; k++) {
    std::vector<double> p2(l + 2, 0.0);
    for (int i = 0; i <= k; i++) p2[i + 1] += (2.0 * k + 1.0) * p1[i] / (k + 1.0);
    for (int i = 0; i <= k - 1; i++) p2[i] -= (double)k * p0[i] / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  return std::vector<double>(p1.begin(), p1.begin() + l + 1);
}

// (x^2 + y^2 + z^2)^k
Poly r2pow(int k) {
  Poly p;
  p.add(0, 0, 0, 1.0);
  Poly r2;
  r2.add(2, 0, 0, 1.0);
  r2.add(0, 2, 0, 1.0);
  r2.add(0, 0, 2, 1.0);
  for (int i = 0; i < k; i++) p = mul(p, r2);
  return p;
}

double binom_real(double top, int k) {  // binomial coefficient C(top, k) for real top
  double r = 1.0;
  for (int t = 1; t <= k; t++) r *= (top - k + t) / t;
  return r;
}

Poly radial_poly(int nr, int l, int m) {
  // angular factor Re / Im (x + i y)^|m|
  const int am = m < 0 ? -m : m;
  Poly ang;
  for (int k = 0; k <= am; k++) {
    // (x + i y)^am = sum_k C(am, k) x^(am-k) (i y)^k ; i^k = 1, i, -1, -i
    const double c = binom_real((double)am, k);
    const int ph = k % 4;
    if (m >= 0 && (ph == 0 || ph == 2)) ang.add(am - k, k, 0, ph == 0 ? c : -c);
    if (m < 0 && (ph == 1 || ph == 3)) ang.add(am - k, k, 0, ph == 1 ? c : -c);
  }
  // sum_i d_i z^i r^(l-|m|-i), d = |m|-th derivative of P_l
  std::vector<double> d = legendre_coeffs(l);
  for (int t = 0; t < am; t++) {
    std::vector<double> dd(d.size() > 1 ? d.size() - 1 : 1, 0.0);
    for (size_t i = 1; i < d.size(); i++) dd[i - 1] = d[i] * (double)i;
    d = dd;
  }
  Poly zr;
  for (size_t i = 0; i < d.size(); i++) {
    if (d[i] == 0.0) continue;
    const int rest = l - am - (int)i;  // even: the derivative has the parity of l - |m|
    Poly zi;
    zi.add(0, 0, (int)i, d[i]);
    for (const auto& u : mul(zi, r2pow(rest / 2)).c) zr.c[u.first] += u.second;
  }
  Poly solid = mul(ang, zr);
  // L_nr^(l+1/2)(r^2) = sum_i (-1)^i C(nr + l + 1/2, nr - i) r^(2i) / i!
  Poly lag;
  const double alpha = l + 0.5;
  double fact = 1.0;
  for (int i = 0; i <= nr; i++) {
    if (i > 0) fact *= i;
    const double a = ((i & 1) ? -1.0 : 1.0) * binom_real(nr + alpha, nr - i) / fact;
    for (const auto& u : r2pow(i).c) lag.c[u.first] += a * u.second;
  }
  Poly q = mul(lag, solid);
  const double nrm = std::sqrt(inner(q, q));
  for (auto& u : q.c) u.second /= nrm;
  return q;
}

Poly cart_poly(int nx, int ny, int nz) {
  const int n[3] = {nx, ny, nz};
  Poly p;
  p.add(0, 0, 0, 1.0);
  for (int d = 0; d < 3; d++) {
    const std::vector<double> h = hermite_coeffs(n[d]);
    double f = 1.0;
    for (int i = 1; i <= n[d]; i++) f *= i;
    const double c = 1.0 / std::sqrt(std::sqrt(M_PI) * std::ldexp(1.0, n[d]) * f);
    Poly q;
    for (size_t i = 0; i < h.size(); i++) q.add(d == 0 ? (int)i : 0, d == 1 ? (int)i : 0, d == 2 ? (int)i : 0, c * h[i]);
    p = mul(p, q);
  }
  return p;
}

struct RadialTables {
  std::vector<int> nr, l, m;  // labels, radial order
  std::vector<double> U;      // [N][N], U[k][j]
};

std::mutex g_radial_mu;
std::map<int, RadialTables> g_radial;

const RadialTables& radial_tables(int numax) {
  std::lock_guard<std::mutex> lk(g_radial_mu);
  auto it = g_radial.find(numax);
  if (it != g_radial.end()) return it->second;
  RadialTables t;
  const int N = nstates(numax);
  for (int nu = 0; nu <= numax; nu++)
    for (int l = nu % 2; l <= nu; l += 2)
      for (int m = -l; m <= l; m++) {
        t.nr.push_back((nu - l) / 2);
        t.l.push_back(l);
        t.m.push_back(m);
      }
  t.U.assign((size_t)N * N, 0.0);
  std::vector<Poly> rad(N);
  for (int j = 0; j < N; j++) rad[(size_t)j] = radial_poly(t.nr[(size_t)j], t.l[(size_t)j], t.m[(size_t)j]);
  for (int nz = 0; nz <= numax; nz++)
    for (int ny = 0; ny + nz <= numax; ny++)
      for (int nx = 0; nx + ny + nz <= numax; nx++) {
        const int k = state_index(numax, nx, ny, nz);
        const Poly c = cart_poly(nx, ny, nz);
        for (int j = 0; j < N; j++)
          if (2 * t.nr[(size_t)j] + t.l[(size_t)j] == nx + ny + nz) t.U[(size_t)k * N + j] = inner(rad[(size_t)j], c);
      }
  return g_radial.emplace(numax, std::move(t)).first->second;
}

// out[a][r][b] = sum over CSR row r of val * in[a][col][b]; one lane per band.
template <typename T>
__global__ void __launch_bounds__(kWarp) k_radial(int N, int B, const int* __restrict__ rowp,
                                                  const int* __restrict__ col, const T* __restrict__ val,
                                                  const T* __restrict__ in, T* __restrict__ out) {
  const int a = blockIdx.x, b = blockIdx.y * kWarp + threadIdx.x;
  if (b >= B) return;
  const T* src = in + (size_t)a * N * B + b;
  T* dst = out + (size_t)a * N * B + b;
  for (int r = 0; r < N; r++) {
    T s = (T)0;
    for (int q = rowp[r]; q < rowp[r + 1]; q++) s = fma(val[q], src[(size_t)col[q] * B], s);
    dst[(size_t)r * B] = s;
  }
}

}  // namespace

int radial_labels(int numax, int* nr, int* l, int* m) {
  const RadialTables& t = radial_tables(numax);
  for (size_t j = 0; j < t.nr.size(); j++) {
    if (nr) nr[j] = t.nr[j];
    if (l) l[j] = t.l[j];
    if (m) m[j] = t.m[j];
  }
  return (int)t.nr.size();
}

const double* radial_matrix(int numax) { return radial_tables(numax).U.data(); }

// CSR (rows = outputs) of U^T (direction 0) or U (direction 1), entries with |U| > 1e-15 only.
void radial_csr(int numax, int direction, std::vector<int>& rowp, std::vector<int>& col, std::vector<double>& val) {
  const RadialTables& t = radial_tables(numax);
  const int N = nstates(numax);
  rowp.assign((size_t)N + 1, 0);
  col.clear();
  val.clear();
  for (int r = 0; r < N; r++) {
    for (int c = 0; c < N; c++) {
      const double u = direction == 0 ? t.U[(size_t)c * N + r] : t.U[(size_t)r * N + c];
      if (std::fabs(u) > 1e-15) {
        col.push_back(c);
        val.push_back(u);
      }
    }
    rowp[(size_t)r + 1] = (int)col.size();
  }
}

cudaError_t launch_radial(int natoms, int N, int nbands, sho_dtype dt, const int* rowp, const int* col,
                          const void* val, const void* in, void* out, cudaStream_t s) {
  const dim3 grid(natoms, (nbands + kWarp - 1) / kWarp);
  if (dt == SHO_F64)
    k_radial<double><<<grid, kWarp, 0, s>>>(N, nbands, rowp, col, static_cast<const double*>(val),
                                            static_cast<const double*>(in), static_cast<double*>(out));
  else
    k_radial<float><<<grid, kWarp, 0, s>>>(N, nbands, rowp, col, static_cast<const float*>(val),
                                           static_cast<const float*>(in), static_cast<float*>(out));
  return cudaGetLastError();
}

}  // namespace sho
