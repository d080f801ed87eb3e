// Host helpers: the moment-relaxation data of a binary quadratic program
// (Section 3.1) and the per-class inverse map used by the projector kernels.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/manidsdp.h"

namespace {

int64_t binom(int64_t n, int64_t k) {
  if (k < 0 || n < 0 || k > n) return 0;
  if (k > n - k) k = n - k;
  int64_t r = 1;
  for (int64_t i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// Basis monomial t (0-based) of v(x) as a sorted variable set of size <= 2.
struct Mono {
  int d;
  int v[4];
};

Mono basis_element(int q, int t) {
  Mono m{0, {0, 0, 0, 0}};
  if (t == 0) return m;
  if (t <= q) {
    m.d = 1;
    m.v[0] = t - 1;
    return m;
  }
  // pairs (i, j), i < j, in lexicographic order
  int r = t - 1 - q;
  int i = 0;
  while (r >= q - 1 - i) {
    r -= q - 1 - i;
    ++i;
  }
  m.d = 2;
  m.v[0] = i;
  m.v[1] = i + 1 + r;
  return m;
}

// Symmetric difference of two sorted sets.
Mono xor_sets(const Mono& a, const Mono& b) {
  Mono o{0, {0, 0, 0, 0}};
  int i = 0, j = 0;
  while (i < a.d || j < b.d) {
    if (j >= b.d || (i < a.d && a.v[i] < b.v[j])) {
      o.v[o.d++] = a.v[i++];
    } else if (i >= a.d || b.v[j] < a.v[i]) {
      o.v[o.d++] = b.v[j++];
    } else {
      ++i;
      ++j;
    }
  }
  return o;
}

}  // namespace

extern "C" int manidsdp_bqp_index_map(int32_t q, int32_t order, int32_t* N_out, int64_t* m_out,
                                      int32_t* idx) {
  if (q < 1 || (order != 1 && order != 2) || N_out == nullptr || m_out == nullptr)
    return MANIDSDP_E_ARG;
  const int64_t N = 1 + q + (order == 2 ? binom(q, 2) : 0);
  if (N > 65535) return MANIDSDP_E_ARG;
  const int dmax = 2 * order;
  std::vector<int64_t> offset(dmax + 2, 0);
  for (int d = 0; d <= dmax; ++d) offset[d + 1] = offset[d] + binom(q, d);
  *N_out = int32_t(N);
  *m_out = offset[dmax + 1];
  if (idx == nullptr) return MANIDSDP_OK;
  // The rank of a sorted d-subset c_1 < ... < c_d counts the d-subsets before it
  // in lexicographic order; summing C(q-1-j, d-i) over the skipped values j at
  // position i telescopes (hockey stick) to C(q-c_{i-1}-1, d-i+1) - C(q-c_i, d-i+1).
  std::vector<std::vector<int64_t>> Cq(q + 2, std::vector<int64_t>(dmax + 2, 0));
  for (int a = 0; a <= q + 1; ++a)
    for (int k = 0; k <= dmax + 1; ++k) Cq[a][k] = binom(a, k);
  std::vector<Mono> B(N);
  for (int t = 0; t < N; ++t) B[t] = basis_element(q, t);
  for (int64_t r = 0; r < N; ++r) {
    for (int64_t c = 0; c < N; ++c) {
      const Mono s = xor_sets(B[r], B[c]);
      int64_t rank = offset[s.d];
      int prev = -1;
      for (int i = 1; i <= s.d; ++i) {
        const int ci = s.v[i - 1];
        rank += Cq[q - prev - 1][s.d - i + 1] - Cq[q - ci][s.d - i + 1];
        prev = ci;
      }
      idx[r * N + c] = int32_t(rank);
    }
  }
  return MANIDSDP_OK;
}

extern "C" int manidsdp_bqp_rhs(int32_t q, int32_t order, const double* Q, const double* c,
                                double* b) {
  if (q < 1 || (order != 1 && order != 2) || Q == nullptr || b == nullptr) return MANIDSDP_E_ARG;
  int32_t N;
  int64_t m;
  int st = manidsdp_bqp_index_map(q, order, &N, &m, nullptr);
  if (st != MANIDSDP_OK) return st;
  for (int64_t a = 0; a < m; ++a) b[a] = 0.0;
  double tr = 0.0;
  for (int i = 0; i < q; ++i) tr += Q[size_t(i) * q + i];
  b[0] = tr;  // x_i^2 = 1 turns the diagonal of Q into a constant
  for (int i = 0; i < q; ++i) b[1 + i] = c ? c[i] : 0.0;
  int64_t k = 1 + q;  // degree-2 monomials x_i x_j (i < j) in lexicographic order
  for (int i = 0; i < q; ++i)
    for (int j = i + 1; j < q; ++j) b[k++] = Q[size_t(i) * q + j] + Q[size_t(j) * q + i];
  return MANIDSDP_OK;
}
