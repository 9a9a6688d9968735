// Host-side helpers shared by the handle API (capi.cu) and the
// allocation-free entry point (noalloc.cu): radix schedules, twiddle tables,
// stiffness checks and the quadratic-form coefficients of the preconditioner.
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace wfft {

// Longest axis a radix schedule is made for.  Whether an axis is supported is decided
// by the tiles of the passes (every stage's register batch and the shared memory):
// up to 1365 points in FP32 and 597-1365 in FP64, depending on the radices.
constexpr int kMaxAxis = 2048;

// The prime factor of n above 7 that a general prime-length stage takes: 0 if n is
// 7-smooth, -1 if what is left after dividing out 2, 3, 5 and 7 is not one prime of
// 11..kMaxPrime (two such primes, a square of one, or a larger prime).
static inline int axis_prime(int n) {
  if (n < 1) return -1;
  int m = n;
  const int small[4] = {2, 3, 5, 7};
  for (int q = 0; q < 4; ++q)
    while (m % small[q] == 0) m /= small[q];
  if (m == 1) return 0;
  if (m > kMaxPrime) return -1;
  for (int d = 2; d * d <= m; ++d)
    if (m % d == 0) return -1;
  return m;
}

// radix schedule: as many 8s as possible, the rest of the power of two as 4s / a 2
// (4*4 rather than 8*2), then the odd radices 3, 5, 7, and the prime factor above 7
// (if any) as one general stage
static inline bool factorize(int n, AxisPlan& pl) {
  pl.n = n;
  for (int i = 0; i < 7; ++i) pl.cnt[i] = 0;
  pl.prime = 0;
  if (n < 1 || n > kMaxAxis) return false;
  const int prime = axis_prime(n);
  if (prime < 0) return false;
  pl.prime = prime;
  int m = prime ? n / prime : n, e2 = 0;
  while (m % 2 == 0) {
    m /= 2;
    ++e2;
  }
  while (e2 >= 3 && e2 != 4) {
    pl.cnt[0]++;
    e2 -= 3;
  }
  if (e2 == 4) pl.cnt[1] += 2;
  else if (e2 == 2) pl.cnt[1] += 1;
  else if (e2 == 1) pl.cnt[2] += 1;
  const int odd[3] = {3, 5, 7};
  for (int q = 0; q < 3; ++q)
    while (m % odd[q] == 0) {
      pl.cnt[3 + q]++;
      m /= odd[q];
    }
  return m == 1;
}

// Every decomposition of n the FFT stages support: the power-of-two part as radix-16
// (when allow16), radix-8, radix-4 and at most one radix-2 stage in any
// mix, the odd part as 3s, 5s and 7s (and the general prime stage, if any).  Empty if
// n is not supported.
static inline std::vector<AxisPlan> factor_candidates(int n, bool allow16) {
  std::vector<AxisPlan> out;
  AxisPlan base;
  if (!factorize(n, base)) return out;
  const int e2 = 3 * base.cnt[0] + 2 * base.cnt[1] + base.cnt[2];
  for (int n16 = 0; allow16 ? 4 * n16 <= e2 : n16 == 0; ++n16)
    for (int n8 = 0; 4 * n16 + 3 * n8 <= e2; ++n8)
      for (int n2 = 0; n2 <= 1; ++n2) {
        const int rest = e2 - 4 * n16 - 3 * n8 - n2;
        if (rest < 0 || (rest & 1)) continue;
        AxisPlan c = base;
        c.cnt[6] = n16;
        c.cnt[0] = n8;
        c.cnt[1] = rest / 2;
        c.cnt[2] = n2;
        out.push_back(c);
      }
  return out;
}

// Radix schedule of an axis at plan creation: the built-in one (factorize), unless a
// tile of three line pairs or three slots (3 n elements) would exceed what its stages
// hold per block (cap(schedule), the register batch of each radix x 256 threads); a
// long axis then takes the decomposition whose stages hold the most.
template <typename Cap>
static inline bool initial_schedule(int n, AxisPlan& pl, Cap cap) {
  if (!factorize(n, pl)) return false;
  if (cap(pl) < 3 * n)
    for (const AxisPlan& c : factor_candidates(n, true))
      if (cap(c) > cap(pl)) pl = c;
  return true;
}

// W_n^m = exp(-2 pi i m / n), m = 0..n-1, evaluated in long double on the host
template <typename T>
static inline void fill_twiddles(cplx<T>* w, int n) {
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int m = 0; m < n; ++m) {
    const long double a = -2.0L * pi * (long double)m / (long double)n;
    w[m].x = (T)cosl(a);
    w[m].y = (T)sinl(a);
  }
}
template <typename T>
static inline std::vector<cplx<T>> twiddles(int n) {
  std::vector<cplx<T>> w(n);
  fill_twiddles<T>(w.data(), n);
  return w;
}

// Per-stage twiddle table of a radix schedule (the stages in the order the FFT runs
// them: the general prime stage P, then 16s, 8s, 4s, 2s, 3s, 5s, 7s).  The stage of
// radix R after Ns points have been combined uses W_{Ns R}^{r k} (r = 1..R-1,
// k = 0..Ns-1), kept at (Ns - 1) + (r - 1) Ns + k: consecutive butterflies of a stage
// read consecutive entries (no shared-memory bank conflicts), and since the blocks of
// successive stages have Ns (R - 1) = Ns' - Ns entries the table has exactly n - 1
// entries (n entries are written, the last one unused).  The prime stage runs at
// Ns = 1, where those twiddles are all 1; its block of P - 1 entries holds the roots
// of its own DFT instead: W_P^m at m - 1 (m = 1..P-1).
template <typename T>
static inline void fill_stage_twiddles(cplx<T>* w, const AxisPlan& pl) {
  const long double pi = 3.141592653589793238462643383279502884L;
  const int rad[7] = {16, 8, 4, 2, 3, 5, 7};
  const int cnt[7] = {pl.cnt[6], pl.cnt[0], pl.cnt[1], pl.cnt[2], pl.cnt[3], pl.cnt[4], pl.cnt[5]};
  for (int i = 0; i < pl.n; ++i) {
    w[i].x = (T)1;
    w[i].y = (T)0;
  }
  int Ns = 1;
  if (pl.prime) {
    const int P = pl.prime;
    for (int m = 1; m < P; ++m) {
      const long double a = -2.0L * pi * (long double)m / (long double)P;
      w[m - 1].x = (T)cosl(a);
      w[m - 1].y = (T)sinl(a);
    }
    Ns = P;
  }
  for (int q = 0; q < 7; ++q)
    for (int s = 0; s < cnt[q]; ++s) {
      const int R = rad[q];
      for (int r = 1; r < R; ++r)
        for (int k = 0; k < Ns; ++k) {
          const long double a = -2.0L * pi * (long double)(r * k) / (long double)(Ns * R);
          w[(Ns - 1) + (r - 1) * Ns + k].x = (T)cosl(a);
          w[(Ns - 1) + (r - 1) * Ns + k].y = (T)sinl(a);
        }
      Ns *= R;
    }
}

// Cholesky test of a symmetric matrix (row-major, size k)
static inline bool spd(const double* m, int k) {
  double L[36] = {0};
  for (int i = 0; i < k; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = m[i * k + j];
      for (int q = 0; q < j; ++q) s -= L[i * 6 + q] * L[j * 6 + q];
      if (i == j) {
        if (!(s > 0)) return false;
        L[i * 6 + i] = std::sqrt(s);
      } else {
        L[i * 6 + j] = s / L[j * 6 + j];
      }
    }
  }
  return true;
}

static inline void voigt_full(const double* c21, double* m6) {
  int k = 0;
  for (int i = 0; i < 6; ++i)
    for (int j = i; j < 6; ++j) {
      m6[i * 6 + j] = m6[j * 6 + i] = c21[k];
      ++k;
    }
}

// Largest eigenvalue of Q_ik = C_ijkl xi_j xi_l (the acoustic tensor times |xi|^2,
// Eq. Eigenvalues_1D_homogeneo without the 1/rho) for one 21-value Voigt row; 2-D
// uses the in-plane block (i, k in {1, 2}).  Cyclic Jacobi rotations on the 3x3
// symmetric matrix.
static inline double acoustic_max_eig(const double* c21, int ndim, const double xi[3]) {
  double m6[36];
  voigt_full(c21, m6);
  static const int vi[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};  // Voigt index of (i, j)
  const int d = ndim == 3 ? 3 : 2;
  double Q[3][3] = {};
  for (int i = 0; i < d; ++i)
    for (int k = 0; k < d; ++k)
      for (int j = 0; j < d; ++j)
        for (int l = 0; l < d; ++l) Q[i][k] += m6[vi[i][j] * 6 + vi[k][l]] * xi[j] * xi[l];
  if (d == 2) Q[2][2] = 0.0;
  for (int sweep = 0; sweep < 50; ++sweep) {
    const double off = Q[0][1] * Q[0][1] + Q[0][2] * Q[0][2] + Q[1][2] * Q[1][2];
    const double diag = Q[0][0] * Q[0][0] + Q[1][1] * Q[1][1] + Q[2][2] * Q[2][2];
    if (off <= 1e-30 * diag) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (Q[p][q] == 0.0) continue;
        const double th = (Q[q][q] - Q[p][p]) / (2.0 * Q[p][q]);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int r = 0; r < 3; ++r) {  // columns p, q
          const double a = Q[r][p], b = Q[r][q];
          Q[r][p] = c * a - sn * b;
          Q[r][q] = sn * a + c * b;
        }
        for (int r = 0; r < 3; ++r) {  // rows p, q
          const double a = Q[p][r], b = Q[q][r];
          Q[p][r] = c * a - sn * b;
          Q[q][r] = sn * a + c * b;
        }
      }
  }
  return std::max(Q[0][0], std::max(Q[1][1], Q[2][2]));
}

// Largest eigenvalue of a symmetric n x n matrix (n <= 6, row-major, overwritten):
// cyclic Jacobi rotations.
static inline double sym_max_eig(double* a, int n) {
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int p = 0; p < n; ++p) {
      diag += a[p * n + p] * a[p * n + p];
      for (int q = p + 1; q < n; ++q) off += a[p * n + q] * a[p * n + q];
    }
    if (off <= 1e-30 * diag) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (a[p * n + q] == 0.0) continue;
        const double th = (a[q * n + q] - a[p * n + p]) / (2.0 * a[p * n + q]);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int r = 0; r < n; ++r) {
          const double x = a[r * n + p], y = a[r * n + q];
          a[r * n + p] = c * x - sn * y;
          a[r * n + q] = sn * x + c * y;
        }
        for (int r = 0; r < n; ++r) {
          const double x = a[p * n + r], y = a[q * n + r];
          a[p * n + r] = c * x - sn * y;
          a[q * n + r] = sn * x + c * y;
        }
      }
  }
  double m = a[0];
  for (int p = 1; p < n; ++p) m = std::max(m, a[p * n + p]);
  return m;
}

// Upper bound of the largest eigenvalue of C(x) as a map on symmetric tensors
// (Mandel form: the Voigt matrix with the shear rows and columns scaled by sqrt2,
// so that eps : C : eps = e^T M e with |e| = |eps|_F); 2-D takes the in-plane block.
// exact: Jacobi; otherwise the Gershgorin row-sum bound (cheap, for per-voxel tables).
static inline double mandel_max_eig(const double* c21, int ndim, bool exact) {
  double m6[36];
  voigt_full(c21, m6);
  const double w[6] = {1.0, 1.0, 1.0, 1.4142135623730951, 1.4142135623730951, 1.4142135623730951};
  static const int in2[3] = {0, 1, 5};
  const int n = ndim == 3 ? 6 : 3;
  double a[36];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const int I = ndim == 3 ? i : in2[i], J = ndim == 3 ? j : in2[j];
      a[i * n + j] = m6[I * 6 + J] * w[I] * w[J];
    }
  if (exact) return sym_max_eig(a, n);
  double g = 0.0;
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += std::fabs(a[i * n + j]);
    g = std::max(g, s);
  }
  return g;
}

// Upper bound of the largest eigenvalue of the operator A u = rho u + theta B^T C B u
// (Eq. A_oper) on a periodic grid: for any u, u^T B^T C B u = sum_x eps : C : eps <=
// max_x lambda_max(C(x)) |B u|^2 and |B u| <= |xi|_max |u| (|sym(xi (x) u)|_F <= |xi| |u|),
// with |xi|_max^2 = sum_i (2 pi / L_i * floor((N_i - 1) / 2))^2 (the Nyquist index carries
// no frequency).  rows: nrows Voigt rows of 21 values with their densities.
static inline double operator_max_eig_bound(int ndim, const int n[3], const double h[3], const double* c21,
                                            const double* rho, long long nrows, double theta) {
  const double two_pi = 6.283185307179586476925286766559;
  double xi2 = 0.0;
  for (int i = 0; i < ndim; ++i) {
    const double k = (double)((n[i] - 1) / 2);
    const double x = two_pi / (n[i] * h[i]) * k;
    xi2 += x * x;
  }
  const bool exact = nrows <= 4096;
  double cmax = 0.0, rmax = 0.0;
  for (long long r = 0; r < nrows; ++r) {
    cmax = std::max(cmax, mandel_max_eig(c21 + 21 * r, ndim, exact));
    rmax = std::max(rmax, rho[r]);
  }
  return rmax + theta * cmax * xi2;
}

// Quadratic-form coefficients of theta*K(xi), K = B^T Cbar B (Eq. acous), B the
// engineering strain-displacement map of xi.
static inline void precond_coeffs(const double* cbar21, double theta, double kq[6][6]) {
  double C[36];
  voigt_full(cbar21, C);
  double b[6][3][3] = {};
  b[0][0][0] = 1;
  b[1][1][1] = 1;
  b[2][2][2] = 1;
  b[3][1][2] = 1;
  b[3][2][1] = 1;
  b[4][0][2] = 1;
  b[4][2][0] = 1;
  b[5][0][1] = 1;
  b[5][1][0] = 1;
  const int pi_[6] = {0, 1, 2, 1, 0, 0}, pj_[6] = {0, 1, 2, 2, 2, 1};
  const int mk[6] = {0, 1, 2, 1, 0, 0}, mm[6] = {0, 1, 2, 2, 2, 1};
  for (int pr = 0; pr < 6; ++pr) {
    const int i = pi_[pr], j = pj_[pr];
    double G[3][3] = {};
    for (int k = 0; k < 3; ++k)
      for (int m = 0; m < 3; ++m)
        for (int I = 0; I < 6; ++I)
          for (int J = 0; J < 6; ++J) G[k][m] += b[I][i][k] * C[I * 6 + J] * b[J][j][m];
    for (int mo = 0; mo < 6; ++mo) {
      const int k = mk[mo], m = mm[mo];
      kq[pr][mo] = theta * (k == m ? G[k][k] : G[k][m] + G[m][k]);
    }
  }
}

}  // namespace wfft
