// Host linear algebra for small symmetric matrices (the p x p Gram Y'Y of the
// rank update, the Lanczos tridiagonal): Householder tridiagonalisation, Sturm
// counts, bisection, inverse iteration.  Header-only and free of CUDA so that the
// host tests can compile it on its own.
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

namespace mds {
namespace hostla {

// Householder reduction of a symmetric n x n matrix to tridiagonal form
// T = Q' A Q (Golub and Van Loan, Matrix Computations, Sec. 8.3.1): diagonal d,
// off-diagonal e, and the reflectors H_k = I - beta_k v_k v_k' (v_k acting on
// entries k+1 .. n-1, v_k[0] = 1) with Q = H_0 H_1 ... H_{n-3}.  Row-major
// storage keeps every inner loop contiguous: about 4/3 n^3 flops.
struct SymTridiag {
  int n = 0;
  std::vector<double> d, e;      // T
  std::vector<double> v, beta;   // reflector k: v[k * n + 0 .. n - k - 2], beta[k]
};

inline SymTridiag sym_tridiag(std::vector<double> A, int n) {
  SymTridiag t;
  t.n = n;
  t.d.assign(n, 0.0);
  t.e.assign(n > 1 ? n - 1 : 0, 0.0);
  t.v.assign(size_t(n) * n, 0.0);
  t.beta.assign(n, 0.0);
  std::vector<double> pv(n), wv(n);
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;               // x = A[k+1 .., k]
    const double* x = &A[size_t(k) * n + k + 1];  // row k (A symmetric)
    double sig = 0.0;
    for (int j = 1; j < m; ++j) sig += x[j] * x[j];
    const double x0 = x[0];
    double* v = &t.v[size_t(k) * n];
    if (sig == 0.0) {  // already tridiagonal in this column
      t.e[k] = x0;
      continue;
    }
    // v = x - mu e_1 scaled to v[0] = 1, H x = mu e_1 with mu = ||x||
    const double mu = std::sqrt(x0 * x0 + sig);
    const double v0 = x0 <= 0.0 ? x0 - mu : -sig / (x0 + mu);
    const double beta = 2.0 * v0 * v0 / (sig + v0 * v0);
    v[0] = 1.0;
    for (int j = 1; j < m; ++j) v[j] = x[j] / v0;
    t.beta[k] = beta;
    t.e[k] = mu;
    // p = beta A22 v;  w = p - (beta p'v / 2) v;  A22 -= v w' + w v'
    // rows are independent in both passes: threads split them (same arithmetic
    // per entry whatever the thread count, so the result does not depend on it)
#pragma omp parallel for schedule(static) if (m >= 128)
    for (int i = 0; i < m; ++i) {
      const double* row = &A[size_t(k + 1 + i) * n + k + 1];
      double s = 0.0;
      for (int j = 0; j < m; ++j) s += row[j] * v[j];
      pv[i] = beta * s;
    }
    double pvv = 0.0;
    for (int i = 0; i < m; ++i) pvv += pv[i] * v[i];
    const double K = 0.5 * beta * pvv;
    for (int i = 0; i < m; ++i) wv[i] = pv[i] - K * v[i];
#pragma omp parallel for schedule(static) if (m >= 128)
    for (int i = 0; i < m; ++i) {
      double* row = &A[size_t(k + 1 + i) * n + k + 1];
      const double vi = v[i], wi = wv[i];
      for (int j = 0; j < m; ++j) row[j] -= vi * wv[j] + wi * v[j];
    }
  }
  if (n >= 2) t.e[n - 2] = A[size_t(n - 2) * n + n - 1];
  for (int i = 0; i < n; ++i) t.d[i] = A[size_t(i) * n + i];
  return t;
}

// y <- Q y: an eigenvector of T mapped to one of A (reflectors applied last to first).
inline void tridiag_backtransform(const SymTridiag& t, std::vector<double>& y) {
  const int n = t.n;
  for (int k = n - 3; k >= 0; --k) {
    if (t.beta[k] == 0.0) continue;
    const double* v = &t.v[size_t(k) * n];
    const int m = n - k - 1;
    double s = 0.0;
    for (int j = 0; j < m; ++j) s += v[j] * y[k + 1 + j];
    s *= t.beta[k];
    for (int j = 0; j < m; ++j) y[k + 1 + j] -= s * v[j];
  }
}

// ---- symmetric tridiagonal T (diagonal a[0..k-1], off-diagonal b[0..k-2]) ----
inline int sturm_below(const std::vector<double>& a, const std::vector<double>& b, int k, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < k; ++i) {
    const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
    d = (a[i] - x) - (i > 0 ? bb / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0) ++cnt;
  }
  return cnt;
}

// i-th smallest eigenvalue (0-based) by bisection on Sturm counts.
inline double tridiag_eig(const std::vector<double>& a, const std::vector<double>& b, int k, int i) {
  double lo = a[0], hi = a[0];
  for (int j = 0; j < k; ++j) {
    const double r = (j > 0 ? std::fabs(b[j - 1]) : 0.0) + (j < k - 1 ? std::fabs(b[j]) : 0.0);
    lo = std::min(lo, a[j] - r);
    hi = std::max(hi, a[j] + r);
  }
  const double scale = std::max(std::fabs(lo), std::fabs(hi)) + 1e-300;
  for (int it = 0; it < 200 && hi - lo > 1e-17 * scale; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_below(a, b, k, mid) > i)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Eigenvector of T for eigenvalue theta by inverse iteration (LU without pivoting,
// tiny pivots replaced), orthogonalised against `prev`.
inline std::vector<double> tridiag_vec(const std::vector<double>& a, const std::vector<double>& b, int k,
                                double theta, const std::vector<std::vector<double>>& prev) {
  double tn = 0.0;
  for (int j = 0; j < k; ++j) tn = std::max(tn, std::fabs(a[j]) + (j < k - 1 ? std::fabs(b[j]) : 0.0));
  const double tiny = 1e-14 * (tn + 1e-300);
  std::vector<double> x(k), u(k), l(k), d(k);
  for (int j = 0; j < k; ++j) x[j] = 1.0 + 0.01 * ((j * 7919) % 101);
  for (int it = 0; it < 4; ++it) {
    // factor T - theta I = L U with U bidiagonal (d on diagonal, b above)
    d[0] = a[0] - theta;
    if (std::fabs(d[0]) < tiny) d[0] = tiny;
    for (int j = 1; j < k; ++j) {
      l[j] = b[j - 1] / d[j - 1];
      d[j] = (a[j] - theta) - l[j] * b[j - 1];
      if (std::fabs(d[j]) < tiny) d[j] = tiny;
    }
    for (int j = 1; j < k; ++j) x[j] -= l[j] * x[j - 1];
    x[k - 1] /= d[k - 1];
    for (int j = k - 2; j >= 0; --j) x[j] = (x[j] - b[j] * x[j + 1]) / d[j];
    for (const auto& pv : prev) {
      double dp = 0.0;
      for (int j = 0; j < k; ++j) dp += pv[j] * x[j];
      for (int j = 0; j < k; ++j) x[j] -= dp * pv[j];
    }
    double nrm = 0.0;
    for (int j = 0; j < k; ++j) nrm += x[j] * x[j];
    nrm = std::sqrt(nrm);
    for (int j = 0; j < k; ++j) x[j] /= nrm;
  }
  return x;
}

}  // namespace hostla
}  // namespace mds
