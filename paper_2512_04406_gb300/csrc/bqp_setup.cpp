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

// ---- real second-order UCQP relaxation (Section 3.1, UCQP paragraph) -----------------
// A Laurent exponent with ||delta||_1 <= 4 has at most four nonzero entries.  Its key
// packs (||delta||_1, then each nonzero (index, value) in increasing index, each as
// ((index + 1) << 4) | (value + 4) in 12 bits, unused slots 0) into an integer whose
// order is: degree first, then the lexicographic order of the (index, value) list.
namespace {

struct Laurent {
  int n = 0;
  int i[4] = {0, 0, 0, 0};
  int v[4] = {0, 0, 0, 0};
};

uint64_t laurent_key(const Laurent& d) {
  int l1 = 0;
  for (int t = 0; t < d.n; ++t) l1 += d.v[t] < 0 ? -d.v[t] : d.v[t];
  uint64_t k = uint64_t(l1);
  for (int t = 0; t < 4; ++t) {
    k <<= 12;
    if (t < d.n) k |= (uint64_t(d.i[t] + 1) << 4) | uint64_t(d.v[t] + 4);
  }
  return k;
}

// beta - gamma, zeros dropped, sign fixed so that the first nonzero entry is positive
Laurent laurent_class(const Laurent& b, const Laurent& g) {
  Laurent o;
  int ib = 0, ig = 0;
  while (ib < b.n || ig < g.n) {
    int idx, val;
    if (ig >= g.n || (ib < b.n && b.i[ib] < g.i[ig])) {
      idx = b.i[ib];
      val = b.v[ib++];
    } else if (ib >= b.n || g.i[ig] < b.i[ib]) {
      idx = g.i[ig];
      val = -g.v[ig++];
    } else {
      idx = b.i[ib];
      val = b.v[ib++] - g.v[ig++];
    }
    if (val != 0) {
      o.i[o.n] = idx;
      o.v[o.n] = val;
      ++o.n;
    }
  }
  if (o.n > 0 && o.v[0] < 0)
    for (int t = 0; t < o.n; ++t) o.v[t] = -o.v[t];
  return o;
}

std::vector<Laurent> ucqp_basis(int q) {
  std::vector<Laurent> B;
  B.push_back(Laurent{});
  for (int a = 0; a < q; ++a)
    for (int v : {1, -1, 2, -2}) {
      Laurent d;
      d.n = 1;
      d.i[0] = a;
      d.v[0] = v;
      B.push_back(d);
    }
  for (int a = 0; a < q; ++a)
    for (int c = a + 1; c < q; ++c)
      for (int s : {1, -1})
        for (int t : {1, -1}) {
          Laurent d;
          d.n = 2;
          d.i[0] = a;
          d.v[0] = s;
          d.i[1] = c;
          d.v[1] = t;
          B.push_back(d);
        }
  std::sort(B.begin(), B.end(),
            [](const Laurent& x, const Laurent& y) { return laurent_key(x) < laurent_key(y); });
  return B;
}

}  // namespace

extern "C" int manidsdp_ucqp_index_map(int32_t q, int32_t* N_out, int64_t* m_out, int32_t* idx) {
  if (q < 1 || q > 254 || N_out == nullptr || m_out == nullptr) return MANIDSDP_E_ARG;
  const int64_t N = 2 * int64_t(q) * q + 2 * q + 1;
  if (N > 65535) return MANIDSDP_E_ARG;
  const int64_t q4 = int64_t(q) * q * q * q;
  *N_out = int32_t(N);
  *m_out = (q4 + 2 * int64_t(q) * q * q + 5 * int64_t(q) * q + 4 * q + 3) / 3;
  if (idx == nullptr) return MANIDSDP_OK;
  const std::vector<Laurent> B = ucqp_basis(q);
  std::vector<uint64_t> keys(size_t(N) * N);
  for (int64_t r = 0; r < N; ++r)
    for (int64_t c = 0; c < N; ++c) keys[size_t(r) * N + c] = laurent_key(laurent_class(B[r], B[c]));
  std::vector<uint64_t> uniq(keys);
  std::sort(uniq.begin(), uniq.end());
  uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
  if (int64_t(uniq.size()) != *m_out) return MANIDSDP_E_ARG;
  for (size_t e = 0; e < keys.size(); ++e)
    idx[e] = int32_t(std::lower_bound(uniq.begin(), uniq.end(), keys[e]) - uniq.begin());
  return MANIDSDP_OK;
}

extern "C" int manidsdp_ucqp_rhs(int32_t q, const double* Q, const double* c, double* b) {
  if (q < 1 || Q == nullptr || b == nullptr) return MANIDSDP_E_ARG;
  int32_t N;
  int64_t m;
  int st = manidsdp_ucqp_index_map(q, &N, &m, nullptr);
  if (st != MANIDSDP_OK) return st;
  // class ranks of the few classes that carry coefficients: rebuild the sorted key list
  const std::vector<Laurent> B = ucqp_basis(q);
  std::vector<uint64_t> uniq;
  uniq.reserve(size_t(m));
  for (int32_t r = 0; r < N; ++r)
    for (int32_t s = 0; s < N; ++s) uniq.push_back(laurent_key(laurent_class(B[r], B[s])));
  std::sort(uniq.begin(), uniq.end());
  uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
  auto rank_of = [&](const Laurent& d) {
    return size_t(std::lower_bound(uniq.begin(), uniq.end(), laurent_key(d)) - uniq.begin());
  };
  for (int64_t a = 0; a < m; ++a) b[a] = 0.0;
  double tr = 0.0;
  for (int i = 0; i < q; ++i) tr += Q[size_t(i) * q + i];
  b[rank_of(Laurent{})] = tr;  // x_i conj(x_i) = 1
  for (int i = 0; i < q; ++i) {
    Laurent d;
    d.n = 1;
    d.i[0] = i;
    d.v[0] = 1;
    b[rank_of(d)] += c ? c[i] : 0.0;  // Re(c_i x_i) = c_i (x_i + conj(x_i)) / 2
  }
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) {
      if (i == j) continue;
      Laurent xj, xi;  // conj(x_i) Q_ij x_j = Q_ij x^(e_j - e_i)
      xj.n = 1;
      xj.i[0] = j;
      xj.v[0] = 1;
      xi.n = 1;
      xi.i[0] = i;
      xi.v[0] = 1;
      b[rank_of(laurent_class(xj, xi))] += Q[size_t(i) * q + j];
    }
  return MANIDSDP_OK;
}

// ---- sparse BQP with overlapping variable blocks (Section 6, sparse BQPs) -------------
// Block k holds the q consecutive variables (q-2)k .. (q-2)k+q-1 (0-based).  A monomial
// class is a set of at most four variables inside one block; its key packs the degree
// and the sorted variables (12 bits each), so sorting keys sorts by degree and then
// lexicographically.  Entries outside the diagonal blocks of the stacked moment matrix
// are classes of their own (one per unordered pair), numbered after the monomials in
// row-major order of (r < c).
namespace {

uint64_t mono_key(int d, const int* v) {
  uint64_t k = uint64_t(d);
  for (int s = 0; s < 4; ++s) k = (k << 12) | uint64_t(s < d ? v[s] : 0);
  return k;
}

struct SparseBqp {
  int q = 0, t = 0, nb = 0, nvars = 0;
  std::vector<uint64_t> keys;  // sorted monomial keys
};

bool sparse_bqp_layout(int q, int t, SparseBqp* L) {
  if (q < 2 || t < 1) return false;
  const int64_t nb = 1 + q + binom(q, 2);
  const int64_t nvars = int64_t(q - 2) * t + 2;
  if (nb * t > 65535 || nvars > 4095) return false;
  L->q = q;
  L->t = t;
  L->nb = int(nb);
  L->nvars = int(nvars);
  L->keys.clear();
  for (int k = 0; k < t; ++k) {
    const int s0 = (q - 2) * k;
    int v[4];
    L->keys.push_back(mono_key(0, v));
    for (int a = 0; a < q; ++a) {
      v[0] = s0 + a;
      L->keys.push_back(mono_key(1, v));
      for (int b = a + 1; b < q; ++b) {
        v[1] = s0 + b;
        L->keys.push_back(mono_key(2, v));
        for (int c = b + 1; c < q; ++c) {
          v[2] = s0 + c;
          L->keys.push_back(mono_key(3, v));
          for (int e = c + 1; e < q; ++e) {
            v[3] = s0 + e;
            L->keys.push_back(mono_key(4, v));
          }
        }
      }
    }
  }
  std::sort(L->keys.begin(), L->keys.end());
  L->keys.erase(std::unique(L->keys.begin(), L->keys.end()), L->keys.end());
  return true;
}

int64_t mono_rank(const SparseBqp& L, const Mono& m) {
  const uint64_t k = mono_key(m.d, m.v);
  return std::lower_bound(L.keys.begin(), L.keys.end(), k) - L.keys.begin();
}

// Basis element a of block k: [1, x_i, x_i x_j (i < j)] over the block's variables.
Mono block_basis_element(const SparseBqp& L, int k, int a) {
  Mono m = basis_element(L.q, a);
  for (int s = 0; s < m.d; ++s) m.v[s] += (L.q - 2) * k;
  return m;
}

}  // namespace

extern "C" int manidsdp_sparse_bqp_index_map(int32_t q, int32_t t, int32_t* N_out, int64_t* m_out,
                                             int64_t* m_mono_out, int32_t* idx) {
  if (N_out == nullptr || m_out == nullptr) return MANIDSDP_E_ARG;
  SparseBqp L;
  if (!sparse_bqp_layout(q, t, &L)) return MANIDSDP_E_ARG;
  const int64_t N = int64_t(L.nb) * t;
  const int64_t m_mono = int64_t(L.keys.size());
  const int64_t m = m_mono + (N * N - int64_t(L.nb) * L.nb * t) / 2;
  if (m > INT32_MAX) return MANIDSDP_E_ARG;
  *N_out = int32_t(N);
  *m_out = m;
  if (m_mono_out) *m_mono_out = m_mono;
  if (idx == nullptr) return MANIDSDP_OK;
  for (int k = 0; k < t; ++k) {
    const int64_t o = int64_t(k) * L.nb;
    for (int a = 0; a < L.nb; ++a) {
      const Mono ba = block_basis_element(L, k, a);
      for (int g = 0; g < L.nb; ++g) {
        const Mono s = xor_sets(ba, block_basis_element(L, k, g));
        idx[(o + a) * N + o + g] = int32_t(mono_rank(L, s));
      }
    }
  }
  int64_t next = m_mono;
  for (int64_t r = 0; r < N; ++r)
    for (int64_t c = r + 1; c < N; ++c)
      if (r / L.nb != c / L.nb) {
        idx[r * N + c] = int32_t(next);
        idx[c * N + r] = int32_t(next);
        ++next;
      }
  return MANIDSDP_OK;
}

extern "C" int manidsdp_sparse_bqp_rhs(int32_t q, int32_t t, const double* Qs, const double* cs,
                                       double* b) {
  if (Qs == nullptr || b == nullptr) return MANIDSDP_E_ARG;
  SparseBqp L;
  if (!sparse_bqp_layout(q, t, &L)) return MANIDSDP_E_ARG;
  int32_t N;
  int64_t m, m_mono;
  const int st = manidsdp_sparse_bqp_index_map(q, t, &N, &m, &m_mono, nullptr);
  if (st != MANIDSDP_OK) return st;
  for (int64_t a = 0; a < m; ++a) b[a] = 0.0;
  double tr = 0.0;
  for (int k = 0; k < t; ++k) {
    const double* Q = Qs + size_t(k) * q * q;
    for (int i = 0; i < q; ++i) tr += Q[size_t(i) * q + i];
    const int s0 = (q - 2) * k;
    Mono m1{1, {0, 0, 0, 0}};
    for (int i = 0; i < q; ++i) {
      m1.v[0] = s0 + i;
      b[mono_rank(L, m1)] += cs ? cs[size_t(k) * q + i] : 0.0;
    }
    Mono m2{2, {0, 0, 0, 0}};
    for (int i = 0; i < q; ++i)
      for (int j = i + 1; j < q; ++j) {
        m2.v[0] = s0 + i;
        m2.v[1] = s0 + j;
        b[mono_rank(L, m2)] += Q[size_t(i) * q + j] + Q[size_t(j) * q + i];
      }
  }
  b[0] = tr;  // x_i^2 = 1 turns the diagonals of the Q_k into one constant
  return MANIDSDP_OK;
}
