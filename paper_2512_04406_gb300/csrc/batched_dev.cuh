// Device code of the batched solver (batched.cu), compiled once per CTA size:
// batched.cu includes this file inside a namespace that defines kBT, the
// number of threads per CTA.  Every block-wide helper is called by all kBT
// threads of the CTA, and every branch around a barrier depends only on values
// that all threads hold alike (block reductions hand the same sum to every
// thread).

constexpr int kWarps = kBT / 32;

// ---------------------------------------------------------------------------
// block-wide helpers

__device__ double bsum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < kWarps; ++i) s += red[i];  // fixed order: deterministic
  __syncthreads();
  return s;
}

__device__ double bdot(int n, const double* x, const double* y, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += kBT) s = fma(x[i], y[i], s);
  return bsum(s, red);
}

__device__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// out rows = rows of (Y + t E) normalised (N x p); E may be null (t ignored).
__device__ void bretract(int N, int p, const double* Y, const double* E, double t, double* out) {
  for (int r = threadIdx.x; r < N; r += kBT) {
    double s = 0.0;
    for (int c = 0; c < p; ++c) {
      const double v = Y[r * p + c] + (E ? t * E[r * p + c] : 0.0);
      s = fma(v, v, s);
    }
    const double inv = 1.0 / sqrt(s);
    for (int c = 0; c < p; ++c) out[r * p + c] = (Y[r * p + c] + (E ? t * E[r * p + c] : 0.0)) * inv;
  }
  __syncthreads();
}

// out (N x p) = A B for a symmetric N x N A (read by columns: lanes take
// consecutive rows, so the loads of A[k][r] = A[r][k] are contiguous).
__device__ void bsymm(int N, int p, const double* A, const double* B, double* out) {
  for (int e = threadIdx.x; e < N * p; e += kBT) {
    const int r = e % N, c = e / N;
    double s = 0.0;
    for (int k = 0; k < N; ++k) s = fma(A[k * N + r], B[k * p + c], s);
    out[r * p + c] = s;
  }
  __syncthreads();
}

// z_r = <A_r, B_r>
__device__ void browdot(int N, int p, const double* A, const double* B, double* z) {
  for (int r = threadIdx.x; r < N; r += kBT) {
    double s = 0.0;
    for (int c = 0; c < p; ++c) s = fma(A[r * p + c], B[r * p + c], s);
    z[r] = s;
  }
  __syncthreads();
}

// Symmetric eigendecomposition of the small n x n matrix A (row-major,
// destroyed; the p x p Gram Y'Y) by the parallel two-sided Jacobi method:
// n/2 disjoint rotations per step in round-robin order until the off-diagonal
// mass is below 1e-30 of the total.  Eigenvalues ascending in ev; vectors in the
// columns of V (V[k*n + j] = component k of vector j), column perm[i] holding
// the i-th smallest.  n <= 32.
__device__ void bjacobi(int n, double* A, double* V, double* ev, double* red, int* perm) {
  __shared__ double cs_c[kBMaxP / 2 + 1], cs_s[kBMaxP / 2 + 1];
  __shared__ int pr_p[kBMaxP / 2 + 1], pr_q[kBMaxP / 2 + 1];
  const int ne = n + (n & 1);  // even number of slots (slot n is a dummy when n is odd)
  const int half = ne / 2;
  for (int e = threadIdx.x; e < n * n; e += kBT) V[e] = (e / n == e % n) ? 1.0 : 0.0;
  __syncthreads();
  for (int sweep = 0; sweep < 40 && n > 1; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = threadIdx.x; e < n * n; e += kBT) {
      const double a = A[e];
      tot += a * a;
      if (e / n != e % n) off += a * a;
    }
    off = bsum(off, red);
    tot = bsum(tot, red);
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int step = 0; step < ne - 1; ++step) {
      if (threadIdx.x < half) {
        const int i = threadIdx.x;
        auto slot = [&](int k) { return k == 0 ? 0 : 1 + (k - 1 + step) % (ne - 1); };
        int a = slot(i), b = slot(ne - 1 - i);
        if (a > b) { const int t = a; a = b; b = t; }
        double c = 1.0, s = 0.0;
        if (b < n) {
          const double apq = A[a * n + b];
          if (apq != 0.0) {
            const double th = (A[b * n + b] - A[a * n + a]) / (2.0 * apq);
            const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        pr_p[i] = a; pr_q[i] = b; cs_c[i] = c; cs_s[i] = s;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < half * n; e += kBT) {  // rows: A <- J' A
        const int i = e / n, k = e % n, a = pr_p[i], b = pr_q[i];
        if (b < n && cs_s[i] != 0.0) {
          const double x = A[a * n + k], y = A[b * n + k];
          A[a * n + k] = cs_c[i] * x - cs_s[i] * y;
          A[b * n + k] = cs_s[i] * x + cs_c[i] * y;
        }
      }
      __syncthreads();
      for (int e = threadIdx.x; e < half * n; e += kBT) {  // columns: A <- A J, V <- V J
        const int i = e / n, k = e % n, a = pr_p[i], b = pr_q[i];
        if (b < n && cs_s[i] != 0.0) {
          const double x = A[k * n + a], y = A[k * n + b];
          A[k * n + a] = cs_c[i] * x - cs_s[i] * y;
          A[k * n + b] = cs_s[i] * x + cs_c[i] * y;
          const double vx = V[k * n + a], vy = V[k * n + b];
          V[k * n + a] = cs_c[i] * vx - cs_s[i] * vy;
          V[k * n + b] = cs_s[i] * vx + cs_c[i] * vy;
        }
      }
      __syncthreads();
    }
  }
  for (int j = threadIdx.x; j < n; j += kBT) {  // ascending order (ties by index)
    const double dj = A[j * n + j];
    int rk = 0;
    for (int i = 0; i < n; ++i) {
      const double di = A[i * n + i];
      rk += (di < dj) || (di == dj && i < j);
    }
    perm[rk] = j;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += kBT) ev[j] = A[perm[j] * n + perm[j]];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Symmetric tridiagonal eigenproblem for the certificate (all FP64).

// Householder reduction T = Q' A Q of the symmetric N x N matrix A (row-major,
// in place), Q = H_0 H_1 ... H_{N-3}, H_k = I - beta_k v_k v_k' acting on entries
// k+1 .. N-1 (Golub and Van Loan, Sec. 8.3.1).  v_k[0] = 1 is implicit and
// v_k[1 ..] overwrites row k right of A[k][k+1] (no longer read after step k);
// diagonal d, off-diagonal e.  The rank-2 update touches the lower triangle of
// the trailing block and mirrors it (N^3 * 2/3 FP64 multiply-adds in all).
// Warp per row in both passes; A and the vectors in shared memory in the mixed
// form.
__device__ void btridiag(int N, double* A, double* beta, double* d, double* e, double* pv,
                         double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k + 2 < N; ++k) {
    const int m = N - k - 1;
    double* x = A + size_t(k) * N + k + 1;  // row k right of the diagonal
    double sig = 0.0;
    for (int j = 1 + threadIdx.x; j < m; j += kBT) sig = fma(x[j], x[j], sig);
    sig = bsum(sig, red);
    const double x0 = x[0];
    if (sig == 0.0) {  // this column is already reduced
      if (threadIdx.x == 0) {
        e[k] = x0;
        beta[k] = 0.0;
      }
      continue;
    }
    const double mu = sqrt(x0 * x0 + sig);
    const double v0 = x0 <= 0.0 ? x0 - mu : -sig / (x0 + mu);
    const double bk = 2.0 * v0 * v0 / (sig + v0 * v0);
    const double inv0 = 1.0 / v0;
    for (int j = 1 + threadIdx.x; j < m; j += kBT) x[j] *= inv0;  // v_k[j], each by its reader
    if (threadIdx.x == 0) {
      e[k] = mu;
      beta[k] = bk;
    }
    __syncthreads();
    const double* v = x;  // v[0] is 1, not x[0]
    // p = beta A22 v
    for (int i = wid; i < m; i += kWarps) {
      const double* row = A + size_t(k + 1 + i) * N + k + 1;
      double s = 0.0;
      for (int j = lane; j < m; j += 32) s = fma(row[j], j == 0 ? 1.0 : v[j], s);
      s = wsum(s);
      if (lane == 0) pv[i] = bk * s;
    }
    __syncthreads();
    double pvv = 0.0;
    for (int i = threadIdx.x; i < m; i += kBT) pvv = fma(pv[i], i == 0 ? 1.0 : v[i], pvv);
    const double K = 0.5 * bk * bsum(pvv, red);
    for (int i = threadIdx.x; i < m; i += kBT) pv[i] -= K * (i == 0 ? 1.0 : v[i]);  // w
    __syncthreads();
    // A22 -= v w' + w v' on j <= i, mirrored
    for (int i = wid; i < m; i += kWarps) {
      double* row = A + size_t(k + 1 + i) * N + k + 1;
      const double vi = i == 0 ? 1.0 : v[i], wi = pv[i];
      for (int j = lane; j <= i; j += 32) {
        const double val = row[j] - fma(vi, pv[j], wi * (j == 0 ? 1.0 : v[j]));
        row[j] = val;
        A[size_t(k + 1 + j) * N + k + 1 + i] = val;
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < N; i += kBT) {
    d[i] = A[size_t(i) * N + i];
    if (i == N - 2) e[i] = A[size_t(i) * N + i + 1];
  }
  __syncthreads();
}

// Number of eigenvalues of T (diagonal d, squared off-diagonal e2) below x: the
// sign changes of the leading principal minors P_0 = 1, P_1, ..., P_N of T - x I
// (P_{i+1} = (d_i - x) P_i - e2_{i-1} P_{i-1}), kept in range by rescaling both
// carried minors by 2^-600 or 2^600 when the exponent of P leaves
// [2^-600, 2^600]; a zero minor is replaced by -2^-300 times its predecessor.
// Division-free: three FP64 operations a step.
__device__ int bsturm(int N, const double* d, const double* e2, double x) {
  double pm = 1.0, pc = d[0] - x;
  if (pc == 0.0) pc = -0x1p-300;
  int cnt = pc < 0.0;
  for (int i = 1; i < N; ++i) {
    double pn = fma(d[i] - x, pc, -e2[i - 1] * pm);
    if (pn == 0.0) pn = -0x1p-300 * pc;
    cnt += (__double2hiint(pn) ^ __double2hiint(pc)) < 0;  // sign change
    pm = pc;
    pc = pn;
    const int ex = (__double2hiint(pc) >> 20) & 0x7ff;
    if (ex > 1023 + 600) {
      pc *= 0x1p-600;
      pm *= 0x1p-600;
    } else if (ex < 1023 - 600) {
      pc *= 0x1p600;
      pm *= 0x1p600;
    }
  }
  return cnt;
}

// The j-th smallest eigenvalue (0-based) of T in [lo, hi] by multisection, run
// by one whole warp: each round evaluates the Sturm count at 32 interior points
// of the bracket (one per lane) and keeps the 1/33 sub-interval where the count
// passes j, until the bracket is below rel * max(|lo|, |hi|) + tiny.
__device__ double bmultisect(int N, const double* d, const double* e2, int j, double lo, double hi,
                             double rel, double tiny) {
  const int lane = threadIdx.x & 31;
  for (int it = 0; it < 64; ++it) {
    if (hi - lo <= rel * fmax(fabs(lo), fabs(hi)) + tiny) break;
    const double h = (hi - lo) * (1.0 / 33.0);
    const unsigned above = __ballot_sync(0xffffffffu, bsturm(N, d, e2, lo + (lane + 1) * h) > j);
    const int l1 = above ? __ffs(above) - 1 : 32;  // first point with more than j below
    const double nlo = l1 == 0 ? lo : lo + l1 * h;
    const double nhi = l1 == 32 ? hi : lo + (l1 + 1) * h;
    if (!(nlo > lo || nhi < hi)) break;  // no progress left at this precision
    lo = nlo;
    hi = nhi;
  }
  return 0.5 * (lo + hi);
}

// Eigenvector of T for the eigenvalue th by inverse iteration (four steps of
// (T - th I) x = x_prev with LU without pivoting, tiny pivots replaced), run by
// one thread; x normalised.  lw, rw: N-long scratch (multipliers, reciprocal
// pivots).
__device__ void binverse(int N, const double* d, const double* e, double th, double tn, double* x,
                         double* lw, double* rw) {
  const double tiny = 1e-14 * (tn + 1e-300);
  for (int j = 0; j < N; ++j) x[j] = 1.0 + 0.01 * ((j * 7919) % 101);
  double dj = d[0] - th;
  if (fabs(dj) < tiny) dj = tiny;
  rw[0] = 1.0 / dj;
  for (int j = 1; j < N; ++j) {
    lw[j] = e[j - 1] * rw[j - 1];
    dj = (d[j] - th) - lw[j] * e[j - 1];
    if (fabs(dj) < tiny) dj = tiny;
    rw[j] = 1.0 / dj;
  }
  for (int it = 0; it < 4; ++it) {
    for (int j = 1; j < N; ++j) x[j] -= lw[j] * x[j - 1];
    x[N - 1] *= rw[N - 1];
    for (int j = N - 2; j >= 0; --j) x[j] = (x[j] - e[j] * x[j + 1]) * rw[j];
    double s = 0.0;
    for (int j = 0; j < N; ++j) s = fma(x[j], x[j], s);
    const double inv = 1.0 / sqrt(s);
    for (int j = 0; j < N; ++j) x[j] *= inv;
  }
}

// ---------------------------------------------------------------------------
// The instance being solved by this CTA.
struct BCtx {
  int N, m, p, P4;
  const int32_t* idx;     // N x N class map (global)
  const int32_t* cptr;    // class a: upper entries cent[cptr[a] .. cptr[a+1])
  const uint32_t* cent;   // (r << 16) | c with r <= c
  int np;                 // pieces: runs of at most kBPiece entries of one class
  const int32_t* pstart;  // piece k: entries pstart[k] .. pstart[k+1]
  const int32_t* pcls;    // class of piece k
  const int32_t* cpc;     // pieces of class a: cpc[a] .. cpc[a+1]
  const double* mult;
  const double* b;
  const double* invm;     // 1 / mult
  const float* invmf;
  double sigma;
  bool fp64;              // FP64 Hessian-vector products (else FP32 in shared memory)
  double* w;              // workspace base
  BLayout L;
  double* red;
  int* gperm;
  long long* prof;        // shared per-phase cycle counters, or null
  // shared memory of the FP32 Hessian-vector product
  float* G32;             // N x N
  const uint16_t* idx16;  // N x N class map in 16 bits (global, read-only)
  float* wf;              // m
  float* Yf;              // N x P4 (columns p .. P4-1 zero)
  float* Upf;             // N x P4
  float* M1;              // P4 x P4: Up' Y
  float* M2;              // P4 x P4: Y' Y
  float* part;            // max(4 kBT, np): partial sums of the T loop, piece sums of w
  double* cs;             // the certificate's scratch (aliases all of the above)
};

// Phase timer (params.profile): thread 0 adds the clock64 cycles of the scope to
// slot k of the CTA's per-instance counters.
struct BTimer {
  long long* slot;
  long long t0;
  __device__ BTimer(long long* prof, int k) : slot(prof ? prof + k : nullptr), t0(0) {
    if (slot && threadIdx.x == 0) t0 = clock64();
  }
  __device__ ~BTimer() {
    if (slot && threadIdx.x == 0) *slot += clock64() - t0;
  }
};

__device__ inline double* WS(const BCtx& c, long long off) { return c.w + off; }

__device__ inline void entry(const BCtx& c, int e, int* r, int* cc) {
  const uint32_t rc = c.cent[e];
  *r = int(rc >> 16);
  *cc = int(rc & 0xffffu);
}

// Psi and y (per-class means of S = Y Y') at Y: S on the upper entries into S
// (class-list order), Psi = <XD, S> + sigma/2 ||R||^2 with R = A*(y) - S.
__device__ void beval(const BCtx& c, const double* Y, double* y, double* S, double* f, double* r2) {
  BTimer tm(c.prof, 3);
  const int N = c.N, p = c.p;
  const double* XD = WS(c, c.L.XD);
  double* ps = WS(c, c.L.ps);
  for (int k = threadIdx.x; k < c.np; k += kBT) {  // S on the entries, piece sums
    double s = 0.0;
    for (int e = c.pstart[k]; e < c.pstart[k + 1]; ++e) {
      int r, cc;
      entry(c, e, &r, &cc);
      double d = 0.0;
      for (int q = 0; q < p; ++q) d = fma(Y[r * p + q], Y[cc * p + q], d);
      S[e] = d;
      s += (r == cc ? 1.0 : 2.0) * d;
    }
    ps[k] = s;
  }
  __syncthreads();
  for (int a = threadIdx.x; a < c.m; a += kBT) {
    double s = 0.0;
    for (int k = c.cpc[a]; k < c.cpc[a + 1]; ++k) s += ps[k];
    y[a] = s * c.invm[a];
  }
  __syncthreads();
  double pf = 0.0, pr = 0.0;
  for (int k = threadIdx.x; k < c.np; k += kBT) {
    const double ya = y[c.pcls[k]];
    for (int e = c.pstart[k]; e < c.pstart[k + 1]; ++e) {
      int r, cc;
      entry(c, e, &r, &cc);
      const double wt = r == cc ? 1.0 : 2.0, R = ya - S[e];
      pr = fma(wt * R, R, pr);
      pf = fma(wt * XD[r * N + cc], S[e], pf);
    }
  }
  pf = bsum(pf, c.red);
  pr = bsum(pr, c.red);
  *r2 = pr;
  *f = pf + 0.5 * c.sigma * pr;
}

// G = XD - sigma R at the point (y, S) in FP64 (workspace) and, for the FP32
// Hessian-vector product, in FP32 (shared memory).
__device__ void bbuild_g(const BCtx& c, const double* y, const double* S) {
  const int N = c.N;
  const double* XD = WS(c, c.L.XD);
  double* G = WS(c, c.L.G);
  for (int k = threadIdx.x; k < c.np; k += kBT) {
    const double ya = y[c.pcls[k]];
    for (int e = c.pstart[k]; e < c.pstart[k + 1]; ++e) {
      int r, cc;
      entry(c, e, &r, &cc);
      const double g = XD[r * N + cc] - c.sigma * (ya - S[e]);
      G[r * N + cc] = g;
      G[cc * N + r] = g;
      if (!c.fp64) {
        c.G32[r * N + cc] = float(g);
        c.G32[cc * N + r] = float(g);
      }
    }
  }
  __syncthreads();
}

// GY = G Y, z = rowdot(GY, Y), grad = 2 (GY - z Y).  Returns ||grad||.
__device__ double bgrad(const BCtx& c, const double* Y, double* grad) {
  const int N = c.N, p = c.p;
  double* GY = WS(c, c.L.GY);
  double* z = WS(c, c.L.z);
  bsymm(N, p, WS(c, c.L.G), Y, GY);
  browdot(N, p, GY, Y, z);
  double gg = 0.0;
  for (int e = threadIdx.x; e < N * p; e += kBT) {
    const double g = 2.0 * (GY[e] - z[e / p] * Y[e]);
    grad[e] = g;
    gg = fma(g, g, gg);
  }
  return sqrt(bsum(gg, c.red));
}

// HU = Hess Psi(Y)[P_Y(U)] (Proposition 4.2): with Up = P_Y(U) and W = Y Up' + Up Y',
//   T = 2 (G Up + sigma (W - A*(w)) Y),  w = class means of W,
//   HU = T - (T_r . Y_r) Y_r - 2 z_r Up_r.
// W is never formed: W Y = Y (Up' Y) + Up (Y' Y) takes two p x p Grams, and w
// comes from the class lists (w_a = sum over the class's upper entries of
// (2 - [r = c]) (Y_r . Up_c + Up_r . Y_c) / mult_a).  Mixed form: the products in
// FP32 from shared memory (G32, the class map, Y and Up in FP32); FP64 form: the
// same steps in FP64 from the workspace.
__device__ void bhess(const BCtx& c, const double* Y, const double* U, double* HU) {
  BTimer tm(c.prof, 1);
  const int N = c.N, p = c.p;
  double* Up = WS(c, c.L.Up);
  double* T = WS(c, c.L.T);
  const double* z = WS(c, c.L.z);
  const double sg = c.sigma;
  if (c.fp64) {
    double* M1 = WS(c, c.L.M1d);
    double* M2 = WS(c, c.L.M2d);
    double* wd = WS(c, c.L.wd);
    const double* G = WS(c, c.L.G);
    for (int r = threadIdx.x; r < N; r += kBT) {
      double d = 0.0;
      for (int k = 0; k < p; ++k) d = fma(U[r * p + k], Y[r * p + k], d);
      for (int k = 0; k < p; ++k) Up[r * p + k] = U[r * p + k] - d * Y[r * p + k];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < p * p; e += kBT) {
      const int i = e / p, j = e % p;
      double s1 = 0.0, s2 = 0.0;
      for (int k = 0; k < N; ++k) {
        s1 = fma(Up[k * p + i], Y[k * p + j], s1);
        s2 = fma(Y[k * p + i], Y[k * p + j], s2);
      }
      M1[e] = s1;
      M2[e] = s2;
    }
    double* ps = WS(c, c.L.ps);
    for (int k = threadIdx.x; k < c.np; k += kBT) {
      double s = 0.0;
      for (int e = c.pstart[k]; e < c.pstart[k + 1]; ++e) {
        int r, cc;
        entry(c, e, &r, &cc);
        double d = 0.0;
        for (int q = 0; q < p; ++q)
          d = fma(Y[r * p + q], Up[cc * p + q], fma(Up[r * p + q], Y[cc * p + q], d));
        s += (r == cc ? 1.0 : 2.0) * d;
      }
      ps[k] = s;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < c.m; a += kBT) {
      double s = 0.0;
      for (int k = c.cpc[a]; k < c.cpc[a + 1]; ++k) s += ps[k];
      wd[a] = -sg * s * c.invm[a];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < N * p; e += kBT) {
      const int r = e % N, j = e / N;
      double s = 0.0;
      for (int k = 0; k < N; ++k)
        s = fma(G[k * N + r], Up[k * p + j], fma(wd[c.idx[k * N + r]], Y[k * p + j], s));
      for (int i = 0; i < p; ++i) s = fma(sg * Y[r * p + i], M1[i * p + j], fma(sg * Up[r * p + i], M2[i * p + j], s));
      T[r * p + j] = 2.0 * s;
    }
    __syncthreads();
  } else {
    const int P4 = c.P4, ng = (p + 3) >> 2;
    for (int r = threadIdx.x; r < N; r += kBT) {
      double d = 0.0;
      for (int k = 0; k < p; ++k) d = fma(U[r * p + k], Y[r * p + k], d);
      for (int k = 0; k < 4 * ng; ++k) {
        if (k < p) {
          const double u = U[r * p + k] - d * Y[r * p + k];
          Up[r * p + k] = u;
          c.Upf[r * P4 + k] = float(u);
          c.Yf[r * P4 + k] = float(Y[r * p + k]);
        } else {
          c.Upf[r * P4 + k] = 0.f;
          c.Yf[r * P4 + k] = 0.f;
        }
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < p * p; e += kBT) {
      const int i = e / p, j = e % p;
      float s1 = 0.f, s2 = 0.f;
      for (int k = 0; k < N; ++k) {
        const float yj = c.Yf[k * P4 + j];
        s1 = fmaf(c.Upf[k * P4 + i], yj, s1);
        s2 = fmaf(c.Yf[k * P4 + i], yj, s2);
      }
      c.M1[i * P4 + j] = s1;
      c.M2[i * P4 + j] = s2;
    }
    const float sgf = float(sg);
    for (int k = threadIdx.x; k < c.np; k += kBT) {  // piece sums of W over the upper entries
      float s = 0.f;
      for (int e = c.pstart[k]; e < c.pstart[k + 1]; ++e) {
        int r, cc;
        entry(c, e, &r, &cc);
        const float4* yr = reinterpret_cast<const float4*>(c.Yf + r * P4);
        const float4* ur = reinterpret_cast<const float4*>(c.Upf + r * P4);
        const float4* yc = reinterpret_cast<const float4*>(c.Yf + cc * P4);
        const float4* uc = reinterpret_cast<const float4*>(c.Upf + cc * P4);
        float d1 = 0.f, d2 = 0.f;
        for (int g = 0; g < ng; ++g) {
          const float4 a1 = yr[g], b1 = uc[g], a2 = ur[g], b2 = yc[g];
          d1 = fmaf(a1.x, b1.x, fmaf(a1.y, b1.y, fmaf(a1.z, b1.z, fmaf(a1.w, b1.w, d1))));
          d2 = fmaf(a2.x, b2.x, fmaf(a2.y, b2.y, fmaf(a2.z, b2.z, fmaf(a2.w, b2.w, d2))));
        }
        s = fmaf(r == cc ? 1.f : 2.f, d1 + d2, s);
      }
      c.part[k] = s;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < c.m; a += kBT) {
      float s = 0.f;
      for (int k = c.cpc[a]; k < c.cpc[a + 1]; ++k) s += c.part[k];
      c.wf[a] = -sgf * s * c.invmf[a];
    }
    __syncthreads();
    // G Up + A*(wf) Y over items (row r, column group g of 4, k-part ks); lanes
    // take consecutive rows, so G32[k][r] and the class map are read contiguously
    // (both symmetric) and the Y, Up rows are broadcasts.  With few items the
    // k range is split (KS parts, at most kBT items) and the parts are summed
    // in a fixed order.
    const int items0 = N * ng;
    const int KS = max(1, min(8, kBT / items0));
    for (int t = threadIdx.x; t < items0 * KS; t += kBT) {
      const int ks = t / items0, rem = t - ks * items0, g = rem / N, r = rem - g * N;
      const int k0 = ks * N / KS, k1 = (ks + 1) * N / KS;
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
      for (int k = k0; k < k1; ++k) {
        const float gv = c.G32[k * N + r];
        const float wv = c.wf[c.idx16[k * N + r]];
        const float4 u = reinterpret_cast<const float4*>(c.Upf + k * P4)[g];
        const float4 yv = reinterpret_cast<const float4*>(c.Yf + k * P4)[g];
        acc.x = fmaf(gv, u.x, fmaf(wv, yv.x, acc.x));
        acc.y = fmaf(gv, u.y, fmaf(wv, yv.y, acc.y));
        acc.z = fmaf(gv, u.z, fmaf(wv, yv.z, acc.z));
        acc.w = fmaf(gv, u.w, fmaf(wv, yv.w, acc.w));
      }
      if (KS > 1) {
        reinterpret_cast<float4*>(c.part)[t] = acc;
      } else {
        const float a4[4] = {acc.x, acc.y, acc.z, acc.w};
        for (int jj = 0; jj < 4; ++jj) {
          const int j = 4 * g + jj;
          if (j >= p) break;
          float lr = 0.f;
          for (int i = 0; i < p; ++i)
            lr = fmaf(c.Yf[r * P4 + i], c.M1[i * P4 + j], fmaf(c.Upf[r * P4 + i], c.M2[i * P4 + j], lr));
          T[r * p + j] = 2.0 * double(fmaf(sgf, lr, a4[jj]));
        }
      }
    }
    __syncthreads();
    if (KS > 1) {
      for (int e = threadIdx.x; e < N * p; e += kBT) {
        const int r = e % N, j = e / N, g = j >> 2, jj = j & 3;
        float s = 0.f;
        for (int ks = 0; ks < KS; ++ks) s += c.part[4 * (ks * items0 + g * N + r) + jj];
        float lr = 0.f;
        for (int i = 0; i < p; ++i)
          lr = fmaf(c.Yf[r * P4 + i], c.M1[i * P4 + j], fmaf(c.Upf[r * P4 + i], c.M2[i * P4 + j], lr));
        T[r * p + j] = 2.0 * double(fmaf(sgf, lr, s));
      }
      __syncthreads();
    }
  }
  for (int r = threadIdx.x; r < N; r += kBT) {
    double d = 0.0;
    for (int k = 0; k < p; ++k) d = fma(T[r * p + k], Y[r * p + k], d);
    for (int k = 0; k < p; ++k) HU[r * p + k] = T[r * p + k] - d * Y[r * p + k] - 2.0 * z[r] * Up[r * p + k];
  }
  __syncthreads();
}

// Truncated CG on the trust-region model at Y (gradient grad); eta, Heta out.
// Returns the iterations; *bnd set on a boundary or negative-curvature stop.
__device__ int btcg(const BCtx& c, const BParams& P, const double* Y, const double* grad,
                    double Delta, double tol_grad, bool* bnd) {
  const int n = c.N * c.p;
  double* eta = WS(c, c.L.eta);
  double* Heta = WS(c, c.L.Heta);
  double* r = WS(c, c.L.r);
  double* dl = WS(c, c.L.dlt);
  double* Hd = WS(c, c.L.Hd);
  for (int i = threadIdx.x; i < n; i += kBT) {
    eta[i] = 0.0; Heta[i] = 0.0; r[i] = grad[i]; dl[i] = -grad[i];
  }
  __syncthreads();
  double rr = bdot(n, r, r, c.red);
  const double r0 = sqrt(rr);
  double ee = 0.0, ed = 0.0, dd = rr;
  const double target = fmax(r0 * fmax(fmin(r0, 0.1), P.tcg_floor), P.tcg_abs * tol_grad);
  *bnd = false;
  for (int j = 1; j <= P.max_tcg; ++j) {
    bhess(c, Y, dl, Hd);
    const double kap = bdot(n, dl, Hd, c.red);
    const double alpha = kap != 0.0 ? rr / kap : INFINITY;
    const double ee_new = ee + 2.0 * alpha * ed + alpha * alpha * dd;
    if (kap <= 0.0 || ee_new >= Delta * Delta) {
      const double tau = (-ed + sqrt(ed * ed + dd * (Delta * Delta - ee))) / dd;
      for (int i = threadIdx.x; i < n; i += kBT) {
        eta[i] += tau * dl[i];
        Heta[i] += tau * Hd[i];
      }
      __syncthreads();
      *bnd = true;
      return j;
    }
    double rn = 0.0;
    for (int i = threadIdx.x; i < n; i += kBT) {
      eta[i] += alpha * dl[i];
      Heta[i] += alpha * Hd[i];
      const double ri = r[i] + alpha * Hd[i];
      r[i] = ri;
      rn = fma(ri, ri, rn);
    }
    ee = ee_new;
    const double rr_new = bsum(rn, c.red);
    if (sqrt(rr_new) <= target) return j;
    const double beta = rr_new / rr;
    rr = rr_new;
    for (int i = threadIdx.x; i < n; i += kBT) dl[i] = -r[i] + beta * dl[i];
    __syncthreads();
    ed = beta * (ed + alpha * dd);
    dd = rr + beta * beta * dd;
  }
  return P.max_tcg;
}

// Riemannian trust region on Psi from the factor *Yp (the trial buffer *Ytp
// swapped in on accepted steps).  Leaves y (L.y), S (L.S), G, z, grad at the
// final point; returns ||grad||.
__device__ double brtr(const BCtx& c, const BParams& P, double** Yp, double** Ytp, double tol_grad,
                       int* hv, double* fx_out) {
  const int N = c.N, p = c.p, n = N * p;
  double* y = WS(c, c.L.y);
  double* yt = WS(c, c.L.yt);
  double* S = WS(c, c.L.S);
  double* St = WS(c, c.L.St);
  double* grad = WS(c, c.L.grad);
  const double Delta_bar = M_PI * sqrt(double(N));
  double Delta = Delta_bar / 8.0;
  double fx, r2;
  beval(c, *Yp, y, S, &fx, &r2);
  bbuild_g(c, y, S);
  double gn = bgrad(c, *Yp, grad);
  for (int it = 0; it < P.max_rtr; ++it) {
    if (gn <= tol_grad) break;
    bool bnd = false;
    *hv += btcg(c, P, *Yp, grad, Delta, tol_grad, &bnd);
    const double* eta = WS(c, c.L.eta);
    const double* Heta = WS(c, c.L.Heta);
    double ge = 0.0, eh = 0.0;
    for (int i = threadIdx.x; i < n; i += kBT) {
      ge = fma(grad[i], eta[i], ge);
      eh = fma(eta[i], Heta[i], eh);
    }
    ge = bsum(ge, c.red);
    eh = bsum(eh, c.red);
    const double model_dec = -(ge + 0.5 * eh);
    bretract(N, p, *Yp, eta, 1.0, *Ytp);
    double f_new, r2n;
    beval(c, *Ytp, yt, St, &f_new, &r2n);
    const double reg = fmax(1.0, fabs(fx)) * 1e3 * 2.220446049250313e-16;
    const double rho = (model_dec + reg > 0.0) ? (fx - f_new + reg) / (model_dec + reg) : -INFINITY;
    if (rho < 0.25)
      Delta /= 4.0;
    else if (rho > 0.75 && bnd)
      Delta = fmin(2.0 * Delta, Delta_bar);
    if (rho > 0.1) {
      double* t = *Yp; *Yp = *Ytp; *Ytp = t;
      double* u = y; y = yt; yt = u;
      u = S; S = St; St = u;
      fx = f_new;
      bbuild_g(c, y, S);
      gn = bgrad(c, *Yp, grad);
    }
  }
  if (y != WS(c, c.L.y)) {  // the final point's y and S into L.y, L.S
    for (int a = threadIdx.x; a < c.m; a += kBT) yt[a] = y[a];
    for (int e = threadIdx.x; e < c.cptr[c.m]; e += kBT) St[e] = S[e];
    __syncthreads();
  }
  *fx_out = fx;
  return gn;
}

// Eigen-information of the certificate X = XD - Diag(z): lambda_min, lambda_max,
// nneg = #eigenvalues below -neg_tol (1 + |lambda_max|) (at most delta_max) and,
// with want_vecs, their eigenvectors (ascending) in Vk[j*N ..].  Householder
// tridiagonalisation, Sturm bisection, inverse iteration with Gram-Schmidt among
// the vectors, back-transformation by the reflectors.
struct BEig {
  double lmin, lmax;
  int nneg;
};

__device__ BEig bcert(const BCtx& c, const BParams& P, const double* z, bool want_vecs) {
  BTimer tm(c.prof, 2);
  const int N = c.N;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // scratch: shared memory in the mixed form (free while no Hessian-vector
  // product runs), the workspace in the FP64 form
  double* A = c.fp64 ? WS(c, c.L.E) : c.cs;
  double* pv = A + size_t(N) * N;
  double* d = pv + N;
  double* e = d + N;
  double* e2 = e + N;
  double* beta = e2 + N;
  double* ev = beta + N;  // 32 + N
  const double* XD = WS(c, c.L.XD);
  double* Vk = WS(c, c.L.Vk);
  double* sc = WS(c, c.L.cert);
  for (int i = threadIdx.x; i < N * N; i += kBT) A[i] = XD[i] - (i / N == i % N ? z[i / N] : 0.0);
  __syncthreads();
  BEig r;
  if (N == 1) {
    r.lmin = r.lmax = A[0];
    r.nneg = 0;
    __syncthreads();
    return r;
  }
  btridiag(N, A, beta, d, e, pv, c.red);
  if (threadIdx.x == 0) {
    double lo = d[0], hi = d[0], tn = 0.0;
    for (int j = 0; j < N; ++j) {
      const double rj = (j > 0 ? fabs(e[j - 1]) : 0.0) + (j < N - 1 ? fabs(e[j]) : 0.0);
      lo = fmin(lo, d[j] - rj);
      hi = fmax(hi, d[j] + rj);
      tn = fmax(tn, fabs(d[j]) + rj);
      if (j < N - 1) e2[j] = e[j] * e[j];
    }
    sc[3] = lo;
    sc[4] = hi;
    sc[6] = tn;
  }
  __syncthreads();
  const double lo = sc[3], hi = sc[4], tn = sc[6];
  const double tiny = 1e-300 + 1e-18 * tn;
  // lambda_min (warp 0) to full precision; lambda_max (warp 1) to 1e-10 relative
  // (it only scales eta_d and the negativity threshold)
  if (wid < 2) {
    const double v = bmultisect(N, d, e2, wid == 0 ? 0 : N - 1, lo, hi, wid == 0 ? 2.2e-16 : 1e-10, tiny);
    if (lane == 0) ev[wid == 0 ? 0 : 31] = v;
  }
  __syncthreads();
  r.lmin = ev[0];
  r.lmax = ev[31];
  if (want_vecs && threadIdx.x == 0) {
    const double thr = -P.neg_tol * (1.0 + fabs(r.lmax));
    sc[2] = double(min(min(bsturm(N, d, e2, thr), P.delta_max), 31));
  }
  __syncthreads();
  r.nneg = want_vecs ? int(sc[2]) : 0;
  const int nneg = r.nneg;
  if (nneg > 0) {
    // the other shifts of the inverse iteration, warp per eigenvalue
    for (int j = 1 + wid; j < nneg; j += kWarps) {
      const double v = bmultisect(N, d, e2, j, lo, hi, 1e-13, tiny);
      if (lane == 0) ev[j] = v;
    }
    __syncthreads();
    double* ivs = WS(c, c.L.ivs);
    for (int j = threadIdx.x; j < nneg; j += kBT)
      binverse(N, d, e, ev[j], tn, Vk + size_t(j) * N, ivs + size_t(j) * 2 * N, ivs + size_t(j) * 2 * N + N);
    __syncthreads();
    if (wid == 0) {  // modified Gram-Schmidt in eigenvalue order
      for (int j = 0; j < nneg; ++j) {
        double* xj = Vk + size_t(j) * N;
        for (int i = 0; i < j; ++i) {
          const double* xi = Vk + size_t(i) * N;
          double s = 0.0;
          for (int t = lane; t < N; t += 32) s = fma(xi[t], xj[t], s);
          s = wsum(s);
          for (int t = lane; t < N; t += 32) xj[t] -= s * xi[t];
          __syncwarp();
        }
        double s = 0.0;
        for (int t = lane; t < N; t += 32) s = fma(xj[t], xj[t], s);
        const double inv = 1.0 / sqrt(wsum(s));
        for (int t = lane; t < N; t += 32) xj[t] *= inv;
        __syncwarp();
      }
    }
    __syncthreads();
    for (int j = wid; j < nneg; j += kWarps) {  // x <- H_0 ... H_{N-3} x, warp per vector
      double* x = Vk + size_t(j) * N;
      for (int k = N - 3; k >= 0; --k) {
        const double bk = beta[k];
        if (bk == 0.0) continue;
        const double* v = A + size_t(k) * N + k + 1;  // v[0] = 1 implicit
        const int m = N - k - 1;
        double s = 0.0;
        for (int t = lane; t < m; t += 32) s = fma(t == 0 ? 1.0 : v[t], x[k + 1 + t], s);
        s = bk * wsum(s);
        for (int t = lane; t < m; t += 32) x[k + 1 + t] -= s * (t == 0 ? 1.0 : v[t]);
        __syncwarp();
      }
    }
  }
  __syncthreads();
  return r;
}

// Algorithm 1 on one instance; the factor starts at Y0 (N x p0).
__device__ void bsolve(BCtx& c, const BParams& P, const double* Y0, BOut* out, double* y_out) {
  const int N = c.N;
  double* Y = WS(c, c.L.Y);
  double* Yt = WS(c, c.L.Yt);
  double* XD = WS(c, c.L.XD);
  double* U = WS(c, c.L.U);
  double* y = WS(c, c.L.y);
  double* S = WS(c, c.L.S);
  double* z = WS(c, c.L.z);
  double* Vk = WS(c, c.L.Vk);
  // XD = D (Xt = 0): b/mult at every entry
  for (int e = threadIdx.x; e < N * N; e += kBT) XD[e] = c.b[c.idx[e]] * c.invm[c.idx[e]];
  c.p = P.p0;
  c.sigma = P.sigma0;
  bretract(N, c.p, Y0, nullptr, 0.0, Y);
  double sigma = P.sigma0, rscale = -1.0;
  double normb = 0.0;
  for (int a = threadIdx.x; a < c.m; a += kBT) normb = fma(c.b[a], c.b[a], normb);
  normb = sqrt(bsum(normb, c.red));
  bool have_U = false, rounded = false;
  int U_cols = 0, hv = 0, status = MANIDSDP_E_NOCONV, outer = 0;
  double eta_p = 0, eta_d = 0, eta_g = 0, value = 0, lmin = 0;
  for (int k = 0; k < P.max_outer; ++k) {
    c.sigma = sigma;
    outer = k + 1;
    // step 3a: the carried direction U = [0, V]
    if (have_U) {
      double f0, r2;
      beval(c, Y, y, S, &f0, &r2);
      bbuild_g(c, y, S);
      bgrad(c, Y, WS(c, c.L.grad));
      double* HU = WS(c, c.L.Hd);
      bhess(c, Y, U, HU);
      ++hv;
      const double curv = bdot(N * c.p, U, HU, c.red);
      bool moved = false;
      if (curv < 0.0) {
        double t = P.carry_t0 > 0.0 ? P.carry_t0 : sqrt(double(N));
        for (int i = 0; i < P.carry_halvings; ++i) {
          bretract(N, c.p, Y, U, t, Yt);
          double ft, r2t;
          beval(c, Yt, WS(c, c.L.yt), WS(c, c.L.St), &ft, &r2t);
          if (ft <= f0 - 1e-4 * 0.5 * t * t * fabs(curv)) {
            double* tt = Y; Y = Yt; Yt = tt;
            moved = true;
            break;
          }
          t *= 0.5;
        }
      }
      if (!moved) {  // keep the first p - U_cols columns
        const int pn = c.p - U_cols;
        for (int e = threadIdx.x; e < N * pn; e += kBT) Yt[e] = Y[(e / pn) * c.p + e % pn];
        __syncthreads();
        double* tt = Y; Y = Yt; Yt = tt;
        c.p = pn;
      }
      have_U = false;
    }
    // step 3b: RTR
    const double tol_k = rscale < 0.0 ? P.tol_grad_max
                                      : fmax(P.tol_grad_min, fmin(P.tol_grad_max, P.tol_grad_factor * rscale));
    double fx;
    const double gnorm = brtr(c, P, &Y, &Yt, tol_k, &hv, &fx);
    // steps 4-8: y(S) at the final Y is in y; Xt <- Xt - sigma R; z = diag((Xt + D) S)
    const int p = c.p;
    double r2 = 0.0;
    for (int kp = threadIdx.x; kp < c.np; kp += kBT) {
      const double ya = y[c.pcls[kp]];
      for (int e = c.pstart[kp]; e < c.pstart[kp + 1]; ++e) {
        int r, cc;
        entry(c, e, &r, &cc);
        const double R = ya - S[e];
        XD[r * N + cc] -= sigma * R;
        if (r != cc) XD[cc * N + r] -= sigma * R;
        r2 = fma((r == cc ? 1.0 : 2.0) * R, R, r2);
      }
    }
    r2 = bsum(r2, c.red);  // also orders the XD updates before their use
    double* GY = WS(c, c.L.GY);
    bsymm(N, p, XD, Y, GY);
    browdot(N, p, GY, Y, z);
    const BEig ce = bcert(c, P, z, true);
    double sumz = 0.0;
    for (int i = threadIdx.x; i < N; i += kBT) sumz += z[i];
    sumz = bsum(sumz, c.red);
    const double by = bdot(c.m, c.b, y, c.red);
    lmin = ce.lmin;
    const double lmax = ce.lmax;
    eta_p = sqrt(r2);
    eta_d = fmax(0.0, -lmin) / (1.0 + fabs(lmax));
    eta_g = fabs(sumz - by) / (1.0 + fabs(sumz) + fabs(by));
    value = by;
    const double eta = fmax(eta_p, fmax(eta_d, eta_g));
    if (!(eta == eta)) { status = MANIDSDP_E_NONFINITE; break; }
    if (eta <= P.tol) { status = MANIDSDP_OK; break; }
    // step 10: eigenpairs of the Gram Y'Y (p x p) for the rounding and the rank drop
    double* gram = WS(c, c.L.gram);
    for (int e = threadIdx.x; e < p * p; e += kBT) {
      const int i = e / p, j = e % p;
      double s = 0.0;
      for (int r = 0; r < N; ++r) s = fma(Y[r * p + i], Y[r * p + j], s);
      gram[e] = s;
    }
    __syncthreads();
    double* gev = WS(c, c.L.gev);
    double* gvec = WS(c, c.L.gvec);
    {
      BTimer tm(c.prof, 4);
      bjacobi(p, gram, gvec, gev, c.red, c.gperm);
    }
    if (eta <= P.round_eta) {
      // rank-one rounding: Yr = sign(Y w), w the top eigenvector of Y'Y
      const int jt = c.gperm[p - 1];
      double* Yr = WS(c, c.L.tmpN);
      for (int r = threadIdx.x; r < N; r += kBT) {
        double s = 0.0;
        for (int q = 0; q < p; ++q) s = fma(Y[r * p + q], gvec[q * p + jt], s);
        Yr[r] = s < 0.0 ? -1.0 : 1.0;
      }
      __syncthreads();
      // classes consistent with Yr Yr' (R_r = 0 exactly)?
      double* yr = WS(c, c.L.yt);
      int bad = 0;
      for (int kp = threadIdx.x; kp < c.np; kp += kBT) {
        int r0, c0;
        entry(c, c.cptr[c.pcls[kp]], &r0, &c0);
        const double s0 = Yr[r0] * Yr[c0];
        for (int e = c.pstart[kp]; e < c.pstart[kp + 1]; ++e) {
          int r, cc;
          entry(c, e, &r, &cc);
          if (Yr[r] * Yr[cc] != s0) bad = 1;
        }
      }
      for (int a = threadIdx.x; a < c.m; a += kBT) {
        int r0, c0;
        entry(c, c.cptr[a], &r0, &c0);
        yr[a] = Yr[r0] * Yr[c0];
      }
      bad = int(bsum(double(bad), c.red));
      if (bad == 0) {
        double* zr = WS(c, c.L.zt);
        for (int r = threadIdx.x; r < N; r += kBT) {
          double s = 0.0;
          for (int q = 0; q < N; ++q) s = fma(XD[q * N + r], Yr[q], s);
          zr[r] = s * Yr[r];
        }
        __syncthreads();
        const BEig re = bcert(c, P, zr, false);
        double szr = 0.0;
        for (int i = threadIdx.x; i < N; i += kBT) szr += zr[i];
        szr = bsum(szr, c.red);
        const double byr = bdot(c.m, c.b, yr, c.red);
        const double ed = fmax(0.0, -re.lmin) / (1.0 + fabs(re.lmax));
        const double eg = fabs(szr - byr) / (1.0 + fabs(szr) + fabs(byr));
        if (fmax(ed, eg) <= P.tol) {
          for (int r = threadIdx.x; r < N; r += kBT) Y[r] = Yr[r];
          __syncthreads();
          c.p = 1;
          eta_p = 0.0;
          eta_d = ed;
          eta_g = eg;
          value = byr;
          lmin = re.lmin;
          status = MANIDSDP_OK;
          rounded = true;
          break;
        }
      }
    }
    // drop directions of Y below rank_tol lambda_max(Y'Y) (at least p_min kept)
    {
      const double wmax = gev[p - 1];
      int r = 0;
      for (int j = 0; j < p; ++j)
        if (gev[j] > P.rank_tol * wmax || j >= p - P.p_min) ++r;
      if (r < p) {
        for (int e = threadIdx.x; e < N * r; e += kBT) {
          const int row = e / r, jj = e % r;
          const int col = c.gperm[p - r + jj];
          double s = 0.0;
          for (int q = 0; q < p; ++q) s = fma(Y[row * p + q], gvec[q * p + col], s);
          Yt[e] = s;
        }
        __syncthreads();
        bretract(N, r, Yt, nullptr, 0.0, Y);
        c.p = r;
      }
    }
    // step 11: sigma rule (5.1)
    const double lhs = sqrt(r2) / (1.0 + normb);
    const double lhs_prev = rscale;
    rscale = lhs;
    if (lhs < P.kappa1 * gnorm)
      sigma = fmax(sigma / P.gamma, P.sigma_min);
    else if (lhs > P.kappa2 * gnorm)
      sigma = fmin(P.gamma * sigma, P.sigma_max);
    else if (P.sigma_stall > 0.0 && lhs_prev > 0.0 && gnorm <= tol_k && lhs > P.sigma_stall * lhs_prev)
      sigma = fmin(P.gamma * sigma, P.sigma_max);  // stalled primal residual
    // steps 9-10: negative curvature -> Y = [Y, 0], U = [0, V]
    const int pc = c.p;
    const int delta = min(min(ce.nneg, P.delta_max), min(P.p_max, kBMaxP) - pc);
    if (delta > 0) {
      const int pn = pc + delta;
      for (int e = threadIdx.x; e < N * pn; e += kBT) {
        const int row = e / pn, col = e % pn;
        Yt[e] = col < pc ? Y[row * pc + col] : 0.0;
        U[e] = col < pc ? 0.0 : Vk[size_t(col - pc) * N + row];
      }
      __syncthreads();
      double* tt = Y; Y = Yt; Yt = tt;
      c.p = pn;
      have_U = true;
      U_cols = delta;
    }
  }
  {  // y at the final point (the rounded point's when the rounding was accepted)
    const double* ys = rounded ? WS(c, c.L.yt) : y;
    for (int a = threadIdx.x; a < c.m; a += kBT) y_out[a] = ys[a];
  }
  if (threadIdx.x == 0) {
    out->value = value;
    out->eta_p = eta_p;
    out->eta_d = eta_d;
    out->eta_g = eta_g;
    out->lambda_min = lmin;
    out->status = status;
    out->p = c.p;
    out->outer = outer;
    out->hessvecs = hv;
  }
  __syncthreads();
}

// Shared-memory carve-up of the FP32 Hessian-vector product for an instance
// (N, m) at row stride P4: byte offsets, 16-byte aligned.
struct BSmem {
  unsigned G32, wf, Yf, Upf, M1, M2, part, cs, total;
};

__host__ __device__ inline BSmem smem_layout(int N, int m, int np, int P4) {
  auto al = [](unsigned x) { return (x + 15u) & ~15u; };
  BSmem s;
  unsigned o = 0;
  s.cs = o;  // the certificate's eigensolver reuses the whole region
  s.part = o; o = al(o + 4u * (unsigned(np) > 4u * kBT ? unsigned(np) : 4u * kBT));
  s.M1 = o; o = al(o + 4u * P4 * P4);
  s.M2 = o; o = al(o + 4u * P4 * P4);
  s.Yf = o; o = al(o + 4u * N * P4);
  s.Upf = o; o = al(o + 4u * N * P4);
  s.G32 = o; o = al(o + 4u * N * N);
  s.wf = o; o = al(o + 4u * m);
  const unsigned cert = s.cs + 8u * (unsigned(N) * N + 6u * N + 32u);  // N x N + 6 N + 32 doubles
  s.total = o > cert ? o : cert;
  return s;
}

__global__ void __launch_bounds__(kBT, kBT <= 256 ? 2 : 1) batched_solve_kernel(
    int ninst, const BInst* __restrict__ inst, const int* __restrict__ order,
    const char* __restrict__ data, const double* __restrict__ Y0, BParams P,
    double* __restrict__ ws, long long ws_stride, int nmax, int mmax, int* __restrict__ next,
    BOut* __restrict__ out, double* __restrict__ y_out, const long long* __restrict__ y_off) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[kWarps];
  __shared__ int gperm[kBMaxP];
  __shared__ int cur;
  __shared__ long long prof[5];
  BCtx c;
  c.w = ws + size_t(blockIdx.x) * ws_stride;
  c.L = make_layout(nmax, mmax);
  c.red = red;
  c.gperm = gperm;
  c.fp64 = P.fp64 != 0;
  c.prof = P.profile ? prof : nullptr;
  c.P4 = (P.p_max + 3) & ~3;
  for (;;) {
    if (threadIdx.x == 0) cur = atomicAdd(next, 1);
    __syncthreads();
    const int slot = cur;
    __syncthreads();
    if (slot >= ninst) break;
    const int i = order[slot];
    const BInst I = inst[i];
    c.N = I.N;
    c.m = I.m;
    c.idx = reinterpret_cast<const int32_t*>(data + I.off_idx);
    c.cptr = reinterpret_cast<const int32_t*>(data + I.off_cptr);
    c.cent = reinterpret_cast<const uint32_t*>(data + I.off_cent);
    c.idx16 = reinterpret_cast<const uint16_t*>(data + I.off_idx16);
    c.np = I.np;
    c.pstart = reinterpret_cast<const int32_t*>(data + I.off_pstart);
    c.pcls = reinterpret_cast<const int32_t*>(data + I.off_pcls);
    c.cpc = reinterpret_cast<const int32_t*>(data + I.off_cpc);
    c.mult = reinterpret_cast<const double*>(data + I.off_cls);
    c.b = c.mult + I.m;
    c.invm = c.b + I.m;
    c.invmf = reinterpret_cast<const float*>(data + I.off_invmf);
    if (!c.fp64) {
      const BSmem sl = smem_layout(I.N, I.m, I.np, c.P4);
      c.G32 = reinterpret_cast<float*>(smem + sl.G32);
      c.wf = reinterpret_cast<float*>(smem + sl.wf);
      c.Yf = reinterpret_cast<float*>(smem + sl.Yf);
      c.Upf = reinterpret_cast<float*>(smem + sl.Upf);
      c.M1 = reinterpret_cast<float*>(smem + sl.M1);
      c.M2 = reinterpret_cast<float*>(smem + sl.M2);
      c.part = reinterpret_cast<float*>(smem + sl.part);
      c.cs = reinterpret_cast<double*>(smem + sl.cs);
    }
    if (threadIdx.x < 5) prof[threadIdx.x] = 0;
    __syncthreads();
    {
      BTimer tm(c.prof, 0);
      bsolve(c, P, Y0 + I.off_y0, &out[i], y_out + y_off[i]);
    }
    if (threadIdx.x < 5) out[i].cycles[threadIdx.x] = prof[threadIdx.x];  // 0 unless profiling
  }
}
