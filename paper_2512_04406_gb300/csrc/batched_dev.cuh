// Device code of the batched solver (batched.cu), compiled once per CTA size:
// batched.cu includes this file inside a namespace that defines kBT, the
// number of threads per CTA.  Every block-wide helper is called by all kBT
// threads of the CTA.
// ---------------------------------------------------------------------------
// block-wide helpers (every thread of the CTA calls them)

__device__ double bsum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < kBT / 32; ++i) s += red[i];  // fixed order: deterministic
  __syncthreads();
  return s;
}

__device__ double bdot(int n, const double* x, const double* y, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += kBT) s = fma(x[i], y[i], s);
  return bsum(s, red);
}

__device__ void baxpby(int n, double a, const double* x, double b, const double* y, double* out) {
  for (int i = threadIdx.x; i < n; i += kBT) out[i] = a * x[i] + (y ? b * y[i] : 0.0);
  __syncthreads();
}

__device__ void bcopy(int n, const double* x, double* out) {
  for (int i = threadIdx.x; i < n; i += kBT) out[i] = x[i];
  __syncthreads();
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

// out (N x p) = A (N x N, row-major) B (N x p)
__device__ void bgemm(int N, int p, const double* A, const double* B, double* out) {
  for (int e = threadIdx.x; e < N * p; e += kBT) {
    const int r = e / p, c = e % p;
    double s = 0.0;
    for (int k = 0; k < N; ++k) s = fma(A[r * N + k], B[k * p + c], s);
    out[e] = s;
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

// Up = U - Diag(<U_r, Y_r>) Y (tangent projection)
__device__ void bproj(int N, int p, const double* Y, const double* U, double* Up) {
  for (int r = threadIdx.x; r < N; r += kBT) {
    double d = 0.0;
    for (int c = 0; c < p; ++c) d = fma(U[r * p + c], Y[r * p + c], d);
    for (int c = 0; c < p; ++c) Up[r * p + c] = U[r * p + c] - d * Y[r * p + c];
  }
  __syncthreads();
}

// Symmetric eigendecomposition of the n x n matrix A (row-major, destroyed) by
// the parallel two-sided Jacobi method; eigenvalues ascending in ev, vectors in
// the columns of V (row-major, V[k*n + j] = component k of vector j).  n <= 128.
__device__ void bjacobi(int n, double* A, double* V, double* ev, double* red, int* perm) {
  __shared__ double cs_c[kBMaxN / 2 + 1], cs_s[kBMaxN / 2 + 1];
  __shared__ int pr_p[kBMaxN / 2 + 1], pr_q[kBMaxN / 2 + 1];
  const int ne = n + (n & 1);  // even number of slots (slot n is a dummy when n is odd)
  const int half = ne / 2;
  for (int e = threadIdx.x; e < n * n; e += kBT) V[e] = (e / n == e % n) ? 1.0 : 0.0;
  __syncthreads();
  for (int sweep = 0; sweep < 40; ++sweep) {
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
      // round-robin pairs: slot 0 fixed, the others rotate
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
      // rows p, q of every pair (A <- J' A), then columns (A <- A J), V <- V J
      for (int e = threadIdx.x; e < half * n; e += kBT) {
        const int i = e / n, k = e % n, a = pr_p[i], b = pr_q[i];
        if (b < n && cs_s[i] != 0.0) {
          const double x = A[a * n + k], y = A[b * n + k];
          A[a * n + k] = cs_c[i] * x - cs_s[i] * y;
          A[b * n + k] = cs_s[i] * x + cs_c[i] * y;
        }
      }
      __syncthreads();
      for (int e = threadIdx.x; e < half * n; e += kBT) {
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
  // ascending order: rank of each diagonal entry (ties by index)
  for (int j = threadIdx.x; j < n; j += kBT) {
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
// The instance being solved by this CTA.
struct BCtx {
  int N, m, p;
  const int32_t* idx;
  const int32_t* cptr;
  const int32_t* cent;
  const double* mult;
  const double* b;
  double sigma;
  bool fp64;  // FP64 Hessian-vector products (else FP32)
  double* w;  // workspace base
  BLayout L;
  double* red;
  int* perm;
  int* gperm;
};

__device__ inline double* WS(const BCtx& c, long long off) { return c.w + off; }
__device__ inline float* WSf(const BCtx& c, long long off) { return reinterpret_cast<float*>(c.w + off); }

// Psi, y (per-class means of S = Y Y'), G = XD - sigma R at Y; returns Psi, r2 = ||R||^2.
__device__ void beval(const BCtx& c, const double* Y, double* y, double* G, double* f, double* r2) {
  const int N = c.N, p = c.p;
  for (int a = threadIdx.x; a < c.m; a += kBT) {
    double s = 0.0;
    for (int e = c.cptr[a]; e < c.cptr[a + 1]; ++e) {
      const int rc = c.cent[e], r = rc / N, cc = rc % N;
      double d = 0.0;
      for (int k = 0; k < p; ++k) d = fma(Y[r * p + k], Y[cc * p + k], d);
      s += (r == cc ? 1.0 : 2.0) * d;
    }
    y[a] = s / c.mult[a];
  }
  __syncthreads();
  const double* XD = WS(c, c.L.XD);
  double pf = 0.0, pr = 0.0;
  for (int e = threadIdx.x; e < N * N; e += kBT) {
    const int r = e / N, cc = e % N;
    double d = 0.0;
    for (int k = 0; k < p; ++k) d = fma(Y[r * p + k], Y[cc * p + k], d);
    const double R = y[c.idx[e]] - d;
    if (G) G[e] = XD[e] - c.sigma * R;
    pf = fma(XD[e], d, pf);
    pr = fma(R, R, pr);
  }
  pf = bsum(pf, c.red);
  pr = bsum(pr, c.red);
  *r2 = pr;
  *f = pf + 0.5 * c.sigma * pr;
}

// GY = G Y, z = rowdot(GY, Y), grad = 2 (GY - z Y); G32 = float(G).  Returns ||grad||.
__device__ double bgrad(const BCtx& c, const double* Y, const double* G, double* grad) {
  const int N = c.N, p = c.p;
  double* GY = WS(c, c.L.GY);
  double* z = WS(c, c.L.z);
  bgemm(N, p, G, Y, GY);
  browdot(N, p, GY, Y, z);
  float* G32 = WSf(c, c.L.G32);
  double gg = 0.0;
  if (!c.fp64)
    for (int e = threadIdx.x; e < N * N; e += kBT) G32[e] = float(G[e]);
  for (int e = threadIdx.x; e < N * p; e += kBT) {
    const double g = 2.0 * (GY[e] - z[e / p] * Y[e]);
    grad[e] = g;
    gg = fma(g, g, gg);
  }
  gg = bsum(gg, c.red);  // also orders the G32 writes before their first use
  return sqrt(gg);
}

// HU = Hess Psi(Y)[P_Y(U)] (Proposition 4.2): W = Y Up' + Up Y', w = class means
// of W, T = G Up + sigma (W - A*(w)) Y; HU = 2T - (2T . Y_r) Y_r - 2 z Up.  In the
// mixed form the products are FP32 (G32, W in FP32); in the FP64 form W lives in
// the E slot (free while a subproblem is being solved) and G is read in FP64.
__device__ void bhess(const BCtx& c, const double* Y, const double* U, double* HU) {
  const int N = c.N, p = c.p;
  double* Up = WS(c, c.L.Up);
  double* T = WS(c, c.L.T);
  const double* z = WS(c, c.L.z);
  bproj(N, p, Y, U, Up);
  if (c.fp64) {
    double* W = WS(c, c.L.E);
    const double* G = WS(c, c.L.G);
    double* w = WS(c, c.L.w);
    for (int e = threadIdx.x; e < N * N; e += kBT) {
      const int r = e / N, cc = e % N;
      double d = 0.0;
      for (int k = 0; k < p; ++k)
        d = fma(Y[r * p + k], Up[cc * p + k], fma(Up[r * p + k], Y[cc * p + k], d));
      W[e] = d;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < c.m; a += kBT) {
      double s = 0.0;
      for (int e = c.cptr[a]; e < c.cptr[a + 1]; ++e) {
        const int rc = c.cent[e];
        s += (rc / N == rc % N ? 1.0 : 2.0) * W[rc];
      }
      w[a] = s / c.mult[a];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < N * N; e += kBT) W[e] = c.sigma * (W[e] - w[c.idx[e]]);
    __syncthreads();
    for (int e = threadIdx.x; e < N * p; e += kBT) {
      const int r = e / p, cc = e % p;
      double s = 0.0;
      for (int k = 0; k < N; ++k) s = fma(G[r * N + k], Up[k * p + cc], fma(W[r * N + k], Y[k * p + cc], s));
      T[e] = 2.0 * s;
    }
  } else {
    float* W = WSf(c, c.L.W32);
    const float* G32 = WSf(c, c.L.G32);
    float* w = WSf(c, c.L.w);
    for (int e = threadIdx.x; e < N * N; e += kBT) {
      const int r = e / N, cc = e % N;
      float d = 0.f;
      for (int k = 0; k < p; ++k)
        d = fmaf(float(Y[r * p + k]), float(Up[cc * p + k]), fmaf(float(Up[r * p + k]), float(Y[cc * p + k]), d));
      W[e] = d;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < c.m; a += kBT) {
      float s = 0.f;
      for (int e = c.cptr[a]; e < c.cptr[a + 1]; ++e) {
        const int rc = c.cent[e];
        s += (rc / N == rc % N ? 1.f : 2.f) * W[rc];
      }
      w[a] = float(double(s) / c.mult[a]);
    }
    __syncthreads();
    const float sg = float(c.sigma);
    for (int e = threadIdx.x; e < N * N; e += kBT) W[e] = sg * (W[e] - w[c.idx[e]]);
    __syncthreads();
    for (int e = threadIdx.x; e < N * p; e += kBT) {
      const int r = e / p, cc = e % p;
      float s = 0.f;
      for (int k = 0; k < N; ++k)
        s = fmaf(G32[r * N + k], float(Up[k * p + cc]), fmaf(W[r * N + k], float(Y[k * p + cc]), s));
      T[e] = 2.0 * double(s);
    }
  }
  __syncthreads();
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
    for (int i = threadIdx.x; i < n; i += kBT) {
      eta[i] += alpha * dl[i];
      Heta[i] += alpha * Hd[i];
      r[i] += alpha * Hd[i];
    }
    __syncthreads();
    ee = ee_new;
    const double rr_new = bdot(n, r, r, c.red);
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

// Riemannian trust region on Psi from the factor at L.Y (Y swapped with L.Yt on
// accepted steps: *yslot tells which buffer holds Y).  Leaves y, G, z, grad at
// the final point; returns ||grad||.
__device__ double brtr(const BCtx& c, const BParams& P, double** Yp, double** Ytp, double tol_grad,
                       int* hv, double* fx_out) {
  const int N = c.N, p = c.p, n = N * p;
  double* G = WS(c, c.L.G);
  double* Gt = WS(c, c.L.E);  // trial G (the certificate matrix slot is free here)
  double* y = WS(c, c.L.y);
  double* yt = WS(c, c.L.yt);
  double* grad = WS(c, c.L.grad);
  const double Delta_bar = M_PI * sqrt(double(N));
  double Delta = Delta_bar / 8.0;
  double fx, r2;
  beval(c, *Yp, y, G, &fx, &r2);
  double gn = bgrad(c, *Yp, G, grad);
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
    beval(c, *Ytp, yt, Gt, &f_new, &r2n);
    const double reg = fmax(1.0, fabs(fx)) * 1e3 * 2.220446049250313e-16;
    const double rho = (model_dec + reg > 0.0) ? (fx - f_new + reg) / (model_dec + reg) : -INFINITY;
    if (rho < 0.25)
      Delta /= 4.0;
    else if (rho > 0.75 && bnd)
      Delta = fmin(2.0 * Delta, Delta_bar);
    if (rho > 0.1) {
      double* t = *Yp; *Yp = *Ytp; *Ytp = t;
      for (int e = threadIdx.x; e < N * N; e += kBT) G[e] = Gt[e];
      for (int a = threadIdx.x; a < c.m; a += kBT) y[a] = yt[a];
      __syncthreads();
      fx = f_new;
      gn = bgrad(c, *Yp, G, grad);
    }
  }
  *fx_out = fx;
  return gn;
}

// The certificate X = XD - Diag(z) (z at Y) into E and its Jacobi eigenpairs
// (eigenvalues ascending in ev, vectors in EV's columns perm[j]).
__device__ void bcert(const BCtx& c, const double* z) {
  const int N = c.N;
  double* E = WS(c, c.L.E);
  const double* XD = WS(c, c.L.XD);
  for (int e = threadIdx.x; e < N * N; e += kBT) E[e] = XD[e] - (e / N == e % N ? z[e / N] : 0.0);
  __syncthreads();
  bjacobi(N, E, WS(c, c.L.EV), WS(c, c.L.ev), c.red, c.perm);
}

// Algorithm 1 on one instance; the factor starts at Y0 (N x p0).
__device__ void bsolve(BCtx& c, const BParams& P, const double* Y0, BOut* out, double* y_out) {
  const int N = c.N;
  double* Ya = WS(c, c.L.Y);
  double* Yb = WS(c, c.L.Yt);
  double* Y = Ya;
  double* Yt = Yb;
  double* XD = WS(c, c.L.XD);
  double* U = WS(c, c.L.U);
  double* y = WS(c, c.L.y);
  double* z = WS(c, c.L.z);
  double* ev = WS(c, c.L.ev);
  double* EV = WS(c, c.L.EV);
  // XD = D (Xt = 0): b/mult at every entry
  for (int e = threadIdx.x; e < N * N; e += kBT) XD[e] = c.b[c.idx[e]] / c.mult[c.idx[e]];
  c.p = P.p0;
  bretract(N, c.p, Y0, nullptr, 0.0, Y);
  double sigma = P.sigma0, rscale = -1.0;
  double normb = 0.0;
  for (int a = threadIdx.x; a < c.m; a += kBT) normb = fma(c.b[a], c.b[a], normb);
  normb = sqrt(bsum(normb, c.red));
  bool have_U = false;
  int U_cols = 0, hv = 0, status = MANIDSDP_E_NOCONV, outer = 0;
  double eta_p = 0, eta_d = 0, eta_g = 0, value = 0, lmin = 0;
  bool rounded = false;
  for (int k = 0; k < P.max_outer; ++k) {
    c.sigma = sigma;
    outer = k + 1;
    // step 3a: the carried direction U = [0, V]
    if (have_U) {
      double f0, r2;
      double* G = WS(c, c.L.G);
      beval(c, Y, y, G, &f0, &r2);
      bgrad(c, Y, G, WS(c, c.L.grad));
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
          beval(c, Yt, WS(c, c.L.yt), nullptr, &ft, &r2t);
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
    double r2 = 0.0;
    const int p = c.p;
    for (int e = threadIdx.x; e < N * N; e += kBT) {
      const int r = e / N, cc = e % N;
      double d = 0.0;
      for (int q = 0; q < p; ++q) d = fma(Y[r * p + q], Y[cc * p + q], d);
      const double R = y[c.idx[e]] - d;
      XD[e] -= sigma * R;
      r2 = fma(R, R, r2);
    }
    r2 = bsum(r2, c.red);
    double* GY = WS(c, c.L.GY);
    bgemm(N, p, XD, Y, GY);
    browdot(N, p, GY, Y, z);
    bcert(c, z);
    double sumz = 0.0, by = 0.0;
    for (int i = threadIdx.x; i < N; i += kBT) sumz += z[i];
    sumz = bsum(sumz, c.red);
    by = bdot(c.m, c.b, y, c.red);
    lmin = ev[0];
    const double lmax = ev[N - 1];
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
    bjacobi(p, gram, gvec, gev, c.red, c.gperm);
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
      for (int a = threadIdx.x; a < c.m; a += kBT) {
        const int e0 = c.cent[c.cptr[a]];
        const double s0 = Yr[e0 / N] * Yr[e0 % N];
        for (int e = c.cptr[a] + 1; e < c.cptr[a + 1]; ++e) {
          const int rc = c.cent[e];
          if (Yr[rc / N] * Yr[rc % N] != s0) bad = 1;
        }
        yr[a] = s0;
      }
      bad = int(bsum(double(bad), c.red));
      if (bad == 0) {
        double* zr = WS(c, c.L.zt);
        for (int r = threadIdx.x; r < N; r += kBT) {
          double s = 0.0;
          for (int q = 0; q < N; ++q) s = fma(XD[r * N + q], Yr[q], s);
          zr[r] = s * Yr[r];
        }
        __syncthreads();
        bcert(c, zr);
        const double lr = ev[0], lmr = ev[N - 1];
        double szr = 0.0;
        for (int i = threadIdx.x; i < N; i += kBT) szr += zr[i];
        szr = bsum(szr, c.red);
        const double byr = bdot(c.m, c.b, yr, c.red);
        const double ed = fmax(0.0, -lr) / (1.0 + fabs(lmr));
        const double eg = fabs(szr - byr) / (1.0 + fabs(szr) + fabs(byr));
        if (fmax(ed, eg) <= P.tol) {
          for (int r = threadIdx.x; r < N; r += kBT) Y[r] = Yr[r];
          __syncthreads();
          c.p = 1;
          eta_p = 0.0;
          eta_d = ed;
          eta_g = eg;
          value = byr;
          lmin = lr;
          status = MANIDSDP_OK;
          rounded = true;
          break;
        }
        bcert(c, z);  // restore the eigenpairs of X for the rank update below
      }
    }
    // drop directions of Y below rank_tol lambda_max(Y'Y) (at least p_min kept)
    {
      const double wmax = gev[p - 1];
      int r = 0;
      for (int j = 0; j < p; ++j)
        if (gev[j] > P.rank_tol * wmax || j >= p - P.p_min) ++r;
      if (r < p) {
        // Y <- rownorm(Y Wk), Wk the kept eigenvectors (ascending)
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
    rscale = lhs;
    if (lhs < P.kappa1 * gnorm)
      sigma = fmax(sigma / P.gamma, P.sigma_min);
    else if (lhs > P.kappa2 * gnorm)
      sigma = fmin(P.gamma * sigma, P.sigma_max);
    // steps 9-10: negative curvature -> Y = [Y, 0], U = [0, V]
    const double thr = -P.neg_tol * (1.0 + fabs(lmax));
    int nneg = 0;
    while (nneg < min(P.delta_max, N) && ev[nneg] < thr) ++nneg;
    const int pc = c.p;
    const int delta = min(min(nneg, P.delta_max), min(P.p_max, kBMaxP) - pc);
    if (delta > 0) {
      const int pn = pc + delta;
      for (int e = threadIdx.x; e < N * pn; e += kBT) {
        const int row = e / pn, col = e % pn;
        Yt[e] = col < pc ? Y[row * pc + col] : 0.0;
        U[e] = col < pc ? 0.0 : EV[row * N + c.perm[col - pc]];
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

__global__ void __launch_bounds__(kBT) batched_solve_kernel(
    int ninst, const BInst* __restrict__ inst, const char* __restrict__ data,
    const double* __restrict__ Y0, BParams P,
    double* __restrict__ ws, long long ws_stride, int nmax, int mmax, int* __restrict__ next,
    BOut* __restrict__ out, double* __restrict__ y_out, const long long* __restrict__ y_off) {
  __shared__ double red[kBT / 32];
  __shared__ int perm[kBMaxN];
  __shared__ int gperm[kBMaxP];
  __shared__ int cur;
  BCtx c;
  c.w = ws + size_t(blockIdx.x) * ws_stride;
  c.L = make_layout(nmax, mmax);
  c.red = red;
  c.perm = perm;
  c.gperm = gperm;
  c.fp64 = P.fp64 != 0;
  for (;;) {
    if (threadIdx.x == 0) cur = atomicAdd(next, 1);
    __syncthreads();
    const int i = cur;
    __syncthreads();
    if (i >= ninst) break;
    const BInst I = inst[i];
    c.N = I.N;
    c.m = I.m;
    c.idx = reinterpret_cast<const int32_t*>(data + I.off_idx);
    c.cptr = reinterpret_cast<const int32_t*>(data + I.off_cptr);
    c.cent = reinterpret_cast<const int32_t*>(data + I.off_cent);
    c.mult = reinterpret_cast<const double*>(data + I.off_cls);
    c.b = c.mult + I.m;
    bsolve(c, P, Y0 + I.off_y0, &out[i], y_out + y_off[i]);
  }
}

