// Test driver for the host linear algebra of the rank update: reads n and a
// row-major symmetric n x n matrix, prints every eigenvalue (bisection on the
// Householder tridiagonal form) and the eigenvectors of the r largest
// (inverse iteration, back-transformed), as the rank update forms them.
#include <cstdio>
#include <vector>

#include "host_linalg.h"

using namespace mds::hostla;

int main() {
  int n = 0, r = 0;
  if (std::scanf("%d %d", &n, &r) != 2 || n < 1 || r < 0 || r > n) return 2;
  std::vector<double> A(size_t(n) * n);
  for (auto& a : A)
    if (std::scanf("%lf", &a) != 1) return 2;
  const SymTridiag T = sym_tridiag(A, n);
  for (int i = 0; i < n; ++i) std::printf("%.17g\n", tridiag_eig(T.d, T.e, n, i));
  std::vector<std::vector<double>> vecs;
  for (int i = n - 1; i >= n - r; --i)
    vecs.push_back(tridiag_vec(T.d, T.e, n, tridiag_eig(T.d, T.e, n, i), vecs));
  for (auto x : vecs) {
    tridiag_backtransform(T, x);
    for (int i = 0; i < n; ++i) std::printf("%.17g%c", x[i], i + 1 < n ? ' ' : '\n');
  }
  return 0;
}
