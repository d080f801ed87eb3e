/*
 * manidsdp.h - C ABI of the GB300 ManiDSDP hot path.
 *
 * ManiDSDP (arXiv 2512.04406) solves the dual unit-diagonal SDP
 *     inf_y b'y   s.t.  S = A*(y) - C >= 0,  diag(S) = 1          (DSDP)
 * by the variable projection y(S) = (AA*)^{-1} A(S + C) (Section 3), an
 * augmented Lagrangian on S (Algorithm 0), and a Burer-Monteiro factor
 * S = Y Y' on the oblique manifold N_p = {Y in R^{N x p}: unit rows}
 * (Section 4) whose subproblems are solved by Riemannian trust region
 * (Algorithm 1).
 *
 * Scope of this library: constraint operators A whose coefficient matrices are
 * 0/1 indicators of disjoint entry sets ("index maps"), as in moment
 * relaxations of binary and unit-modulus problems.  Then A A* is the diagonal
 * of multiplicities (remark on A A* after Algorithm 1), y(S) is a per-class
 * mean of S + C, and A*(y) scatters the means back.
 *
 * Conventions
 *   - All matrices are row-major.  Y, U, HU are N x p with leading dimension p.
 *   - "host or device" pointers are copied with cudaMemcpyDefault (unified
 *     addressing); "device" pointers must be device memory of the context's
 *     device.  The library never frees caller memory; callers never free
 *     library memory except through manidsdp_destroy.
 *   - Every entry point enqueues its work on the stream given to
 *     manidsdp_setup and returns only after the results it reports to the
 *     host are complete (entry points that write device outputs synchronise
 *     the stream before returning as well).
 *   - Return value: MANIDSDP_OK (0) or a negative status.  On
 *     MANIDSDP_E_ARG nothing is written.  No C++ exception crosses the ABI.
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef MANIDSDP_H
#define MANIDSDP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define MANIDSDP_OK 0
#define MANIDSDP_E_ARG (-1)       /* bad shape/pointer, idx out of [0,m), idx not
                                     symmetric, or a class with no entry (then
                                     A A* is singular: Assumption 2 fails) */
#define MANIDSDP_E_NONFINITE (-2) /* NaN/Inf met in inputs or iterates */
#define MANIDSDP_E_NOCONV (-3)    /* iteration limit reached; outputs hold the
                                     last iterate */
#define MANIDSDP_E_TIMEOUT (-4)   /* a device-side wait hit its iteration cap */
#define MANIDSDP_E_CUDA (-5)      /* a CUDA runtime call failed */
#define MANIDSDP_E_NOMEM (-6)     /* device allocation failed */
#define MANIDSDP_E_TOOLARGE (-7)  /* input larger than a fixed-size scratch allows */

/* ---- enums ---------------------------------------------------------------- */
#define MANIDSDP_C_ZERO 0  /* C = 0 (BQP moment relaxations, Section 6.1) */
#define MANIDSDP_C_DENSE 1 /* C given as a dense symmetric N x N FP64 matrix */

#define MANIDSDP_PREC_FP64 0  /* every step in FP64 */
#define MANIDSDP_PREC_MIXED 1 /* Hessian-vector products (tCG) in FP32 with FP32
                                 accumulation; cost, gradient, multiplier update,
                                 KKT residuals and Lanczos in FP64 */

#define MANIDSDP_EIG_MIN 0
#define MANIDSDP_EIG_MAX 1

typedef struct manidsdp_ctx manidsdp_ctx; /* opaque, owned by the library */

/* Algorithm 1 inputs (sigma_0, sigma_min, sigma_max, gamma, kappa_1, kappa_2,
 * p_0) and the knobs of the readings the paper leaves open: inner tolerance
 * eps_k = clamp(tol_grad_factor * ||R^k|| / (1 + ||b||), tol_grad_min,
 * tol_grad_max); rank drop below rank_tol * lambda_max(Y'Y) with p >= p_min;
 * rank growth by at most delta_max eigenvectors whose eigenvalue is below
 * -neg_tol * (1 + |lambda_max(X)|); tCG relative-residual floor tcg_floor and
 * absolute stop tcg_abs * eps_k;
 * carried-direction line search with carry_halvings halvings from carry_t0. */
typedef struct {
  double sigma0, sigma_min, sigma_max, gamma, kappa1, kappa2;
  double tol;             /* stop when eta_max <= tol (Section 6) */
  double tol_grad_min, tol_grad_max, tol_grad_factor;
  double rank_tol, neg_tol, tcg_floor;
  double tcg_abs;         /* tCG also stops once ||r_j|| <= tcg_abs * eps_k */
  double carry_t0;        /* first step of the carried-direction line search; <= 0: sqrt(N) */
  double round_eta;       /* try the rank-one rounding after outer iterations with
                             eta_max <= round_eta (0 disables it) */
  double tc_lowprec_eta;  /* precision schedule of the tensor-core Hess-vec: while the
                             previous outer iteration's eta_max exceeds this value the
                             products use single TF32 operands (about 2^-11 relative
                             per operand) instead of TF32 pairs; 0 (default): pairs
                             throughout */
  int32_t p0, p_min, p_max, delta_max; /* 1 <= p0 <= p_max <= 512 */
  int32_t max_outer, max_rtr, max_tcg, carry_halvings;
  int32_t lanczos_k;      /* Krylov dimension cap for lambda_min / lambda_max (default
                             2000, at most N); a solve stops, and accepts a rank-one
                             rounding, only on a Lanczos run whose smallest Ritz pair
                             converged (residual <= 1e-10 of the spectrum's scale) */
  int32_t precision_mode; /* MANIDSDP_PREC_* */
  int32_t verbose;        /* 1: one line per outer iteration on stderr */
  int32_t profile;        /* 1: time each phase with CUDA events on the context's
                             stream (fills the ms_* fields of the report) */
  int32_t tcg_device;     /* 1 (default): each tCG run is one CUDA-graph launch whose
                             WHILE node loops on the device; 0: host-driven loop */
  int32_t warm_start;     /* 1: manidsdp_solve resumes from the context's factor,
                             multiplier, sigma, inner-tolerance scale and carried
                             negative-curvature direction left by the previous solve
                             (Y0/p0 ignored; a fresh start when no solve ran yet);
                             0 (default): start from Y0 with Xt = 0, sigma0 */
  int32_t tensor_cores;   /* mixed form only: 1 runs the two dense contractions of the
                             FP32 Hessian-vector product (the SDDMM W = Y U' + U Y' and
                             the gather GEMM [G | sigma Q(W)] [U ; Y]) on the tensor
                             cores: TMA-staged operands, tcgen05 kind::tf32 with each
                             operand split into a TF32 pair and three products per K
                             step, FP32 accumulation in chains of at most 640 terms.
                             Hess-vec error within 5e-5 relative (measured 1-3e-5 at
                             N = 3241-7261); about 2x the FP32 FMA kernels at p ~ 300
                             (0.47 vs 0.99 ms at N = 3241, p = 330).  0 (default): FP32
                             FMA kernels */
  int32_t direct;         /* 1: the direct two-block ADMM on (DSDP) itself (Section 3, the
                             comparison with the direct subproblem, Eq.
                             (direct-ALM-subproblem)): each subproblem keeps y frozen at the
                             previous outer iteration's y(S) instead of the best response
                             y(S), so G = Xt + D - sigma (A*(y_k) - S - C) and the Hessian
                             loses the class-mean term (Eq. (hessian-comparison): sigma I in
                             place of sigma Q); the multiplier update is unchanged.  0
                             (default): the variable-projected (DSDP') of Algorithm 1.
                             manidsdp_solve only (not the batched or complex paths) */
  double sigma_stall;     /* safeguard beside rule (5.1) (default 0.5; 0 = off, the rule as
                             printed): after a subproblem solved to its tolerance in which
                             neither branch of (5.1) fired, sigma <- min(gamma sigma,
                             sigma_max) when ||R^{k+1}|| > sigma_stall ||R^k||
                             (0 <= sigma_stall < 1).  The printed rule cannot raise sigma once
                             eps_k tracks ||R||, so a sigma lowered during the capped early
                             subproblems stays low and the ALM crawls */
} manidsdp_params;

/* Per-solve report (host struct filled by manidsdp_solve). */
typedef struct {
  double eta_p, eta_d, eta_g; /* KKT residuals of Section 6 */
  double value;               /* b'y: the relaxation value (dual objective) */
  double pobj;                /* <C, X + Diag z> + sum(z) */
  double lambda_min, lambda_max, sigma;
  /* device time per phase, summed over the solve (params.profile = 1, else 0):
   * Hessian-vector products, subproblem evaluations (y, G, Psi), gradients
   * (G Y, z, grad), Lanczos runs (wall clock); ms_rank: host wall clock of the
   * rank update (eigenvalues of Y'Y, always filled) */
  double ms_hessvec, ms_eval, ms_grad, ms_lanczos, ms_rank;
  double hessvec_p_sum;       /* sum of p over the Hessian-vector products */
  int32_t outer, rtr_iters, hessvecs, p;
  int32_t lanczos_matvecs, status, evals, grads;
} manidsdp_report;

/* Fill *params with the library defaults (the readings listed above). */
void manidsdp_default_params(manidsdp_params* params);

/* Number of CUDA kernels this library has launched since it was loaded (all
 * contexts).  Lets a caller count the device work inside a timed region. */
long long manidsdp_launch_count(void);

/* Device time (ms) spent in the five stages of the Hessian-vector product since the
 * last reset, accumulated when params.profile == 2 on the host-driven path
 * (manidsdp_hessvec, or solves with tcg_device = 0): [0] tangent projection and
 * FP32 copies, [1] class means w, [2] gather GEMM G U - sigma A*(w) Y,
 * [3] Gram pair [U'Y; Y'Y], [4] row epilogue.  reset != 0 zeroes the counters. */
int manidsdp_hessvec_stage_ms(manidsdp_ctx* ctx, double* ms5, int reset);

/* Human-readable text for a status code (static storage). */
const char* manidsdp_strerror(int status);

/*
 * manidsdp_setup - build a context for one SDP instance.
 *   N       order of S (moment-matrix order), N >= 1.
 *   m       number of constraint classes (monomials), m >= 1.
 *   idx     host N x N int32: idx[b*N + g] = class of entry (b, g); must be
 *           symmetric and cover every class in [0, m) at least once.  Copied.
 *   b       host or device, m FP64: right-hand side.  Copied.
 *   c_kind  MANIDSDP_C_ZERO or MANIDSDP_C_DENSE.
 *   c_dense host or device N x N FP64 (symmetric) when c_kind is DENSE, else NULL.
 *   params  NULL for defaults.  Copied.
 *   stream  cudaStream_t cast to void* (NULL = legacy default stream).
 * The context owns device copies of idx, its per-class inverse map (entries
 * (b <= g) grouped by class in row-major order, split into pieces of at most
 * 32 entries), 1/mult, b/mult (the values of D = A*(AA*)^{-1} b), the
 * multiplier Xt (N x N FP64, zero) and all workspace.
 * Definitions: Section 2 (A, A*), Section 3 (y(S), D), remark on AA*.
 */
int manidsdp_setup(manidsdp_ctx** ctx, int32_t N, int64_t m, const int32_t* idx,
                   const double* b, int32_t c_kind, const double* c_dense,
                   const manidsdp_params* params, void* stream);

/* ---- extended set-up: index layouts, sparse C, the complex relaxation ---- */
#define MANIDSDP_C_CSR 2        /* C given as a symmetric CSR matrix (both triangles) */
#define MANIDSDP_IDX_FULL 0     /* idx holds all N x N entries, row-major */
#define MANIDSDP_IDX_PACKED_UPPER 1 /* idx holds the N(N+1)/2 entries (b <= g), row by row */

typedef struct {
  int32_t N;              /* order of S (complex: n, the number of unit-modulus variables) */
  int64_t m;              /* classes (ignored when is_complex) */
  const int32_t* idx;     /* host, layout idx_layout (ignored when is_complex) */
  int32_t idx_layout;     /* MANIDSDP_IDX_FULL or MANIDSDP_IDX_PACKED_UPPER */
  const double* b;        /* host or device, m FP64 (ignored when is_complex) */
  int32_t c_kind;         /* MANIDSDP_C_ZERO, _DENSE or _CSR */
  const double* c_dense;  /* DENSE: host or device N x N FP64 */
  const int64_t* c_rowptr; /* CSR: host N + 1 */
  const int32_t* c_col;   /* CSR: host nnz column indices (sorted or not, no duplicates) */
  const double* c_val;    /* CSR: host nnz values; the matrix must be symmetric */
  int32_t is_complex;     /* 1: the first-order complex relaxation below */
  const double* q_re;     /* complex: host or device n x n FP64, Re Q (symmetric) */
  const double* q_im;     /* complex: host or device n x n FP64, Im Q (antisymmetric), or NULL */
} manidsdp_problem;

/*
 * manidsdp_setup_ex - manidsdp_setup from a problem descriptor.
 *   idx_layout = MANIDSDP_IDX_PACKED_UPPER: idx lists the upper triangle (b <= g)
 *     row by row; the library mirrors it (the classes are symmetric by definition,
 *     Section 2).
 *   c_kind = MANIDSDP_C_CSR: C given in CSR form (Section 2, Eq. (DSDP) with a
 *     sparse cost); it is expanded to the dense N x N operand on the device - the
 *     multiplier Xt and G = Xt + D - sigma R are dense in any case, so the SpMM
 *     form would not remove a dense pass.
 *   is_complex = 1: the first-order relaxation of min z^H Q z over |z_i| = 1,
 *     min <Q, S> over Hermitian S >= 0 with diag(S) = 1 (the complex counterpart of
 *     the relaxations of Section 3.1, solved in the factored form of Section 4 on
 *     the complex oblique manifold).  Every off-diagonal entry is its own class, so
 *     R = 0 on the manifold and a solve is a rank-adaptive Riemannian trust region
 *     certified by X = Q - Diag(mu), mu_i = Re (Q Y Y^H)_ii (Proposition 4.2 with
 *     G = Q; Theorem 4.5).  For such a context, factors Y (n x 2p FP64) hold
 *     Y = A + iB as [A | B] row-major with p complex columns, and the entry points
 *     take p as that number of complex columns: manidsdp_subproblem_eval (psi = f,
 *     rgrad, z = mu; y and rnorm unused), manidsdp_hessvec, manidsdp_lanczos (on the
 *     real embedding [[Xre, -Xim], [Xim, Xre]], v of length 2n = [Re; Im]) and
 *     manidsdp_solve (y_out and Xt_out must be NULL; eta_p = 0).  Defaults of the
 *     complex solve: RTR to ||grad|| <= tol_grad_min (at most 500 iterations), one
 *     column appended per outer round while lambda_min < -neg_tol (1 + |lambda_max|),
 *     p <= min(p_max, 256).  The optimal value's sensitivity is dV/dQ = S* = Y Y^H.
 * Errors as manidsdp_setup (E_ARG for an inconsistent descriptor).
 */
int manidsdp_setup_ex(manidsdp_ctx** ctx, const manidsdp_problem* prob,
                      const manidsdp_params* params, void* stream);

/* Release every resource of the context (NULL is a no-op). */
void manidsdp_destroy(manidsdp_ctx* ctx);

/* Replace the parameters of a context.  p_max and precision_mode size the
 * context's buffers and must equal the values given to manidsdp_setup; the Krylov
 * cap cannot grow beyond the setup value.  E_ARG otherwise (nothing changed). */
int manidsdp_set_params(manidsdp_ctx* ctx, const manidsdp_params* params);

/* Replace the ALM state: multiplier Xt (host or device N x N FP64, NULL = zero)
 * and penalty sigma.  Section 3, Algorithm 0. */
int manidsdp_set_state(manidsdp_ctx* ctx, const double* Xt, double sigma);

/* Direct formulation (params.direct = 1): set the frozen y_k of the subproblem
 * (host or device, m FP64), the y of Eq. (direct-ALM-subproblem) that
 * manidsdp_subproblem_eval and manidsdp_hessvec then use in place of y(S).
 * manidsdp_solve sets it itself (y(S0 + C) at the start, then each outer
 * iteration's y).  E_ARG for a complex context. */
int manidsdp_set_direct_y(manidsdp_ctx* ctx, const double* y);

/* Copy out the multiplier Xt (host or device N x N FP64). */
int manidsdp_get_multiplier(manidsdp_ctx* ctx, double* Xt);

/* Copy out Xt + D = X + Diag(z) (host or device N x N FP64): the primal matrix
 * of (PSDP) at the current multiplier and, after manidsdp_solve, the sensitivity
 * dV/dC of the optimal value (envelope theorem on (PSDP); Algorithm 1 steps 7-8). */
int manidsdp_get_dual_matrix(manidsdp_ctx* ctx, double* XD);

/*
 * manidsdp_subproblem_eval - value and Riemannian gradient of the ALM
 * subproblem Psi_k at Y (Section 4, Eq. (Sub-k), Proposition 4.2):
 *   Psi   = <D + Xt, S + C> + sigma/2 ||Q(S + C)||^2,  S = Y Y'
 *   G     = Xt + D - sigma R,  R = A*(y(S)) - S - C     (Lemma 3.1)
 *   z     = diag(G S),  rgrad = 2 (G Y - Diag(z) Y) = 2 X Y
 * Y: device N x p FP64 with unit rows.  Outputs (each may be NULL):
 *   psi, rnorm (= ||R||): host scalars; rgrad: device N x p; z: device N;
 *   y: device m (the per-class means y(S)).
 * Uses the context's multiplier and sigma.  The evaluated G is kept in the
 * context and used by later manidsdp_hessvec calls at the same Y.
 */
int manidsdp_subproblem_eval(manidsdp_ctx* ctx, const double* Y, int32_t p, double* psi,
                             double* rgrad, double* z, double* y, double* rnorm);

/*
 * manidsdp_hessvec - Riemannian Hessian of Psi_k at Y applied to U
 * (Proposition 4.2, Eq. (4.7)):
 *   W  = Y U' + U Y',  w = (AA*)^{-1} A(W)
 *   Ht = 2 G U + 2 sigma (Y (U'Y) + U (Y'Y) - A*(w) Y)      [= 2GU + 2 sigma Q(W) Y]
 *   HU = Ht - Diag(Ht Y') Y - 2 Diag(z) U
 * evaluated on P_Y(U) (equal to U for tangent U).  Requires a preceding
 * manidsdp_subproblem_eval at the same Y (same device pointer and contents).
 * Y, U, HU: device N x p FP64 (HU may not alias Y or U).  precision selects
 * MANIDSDP_PREC_FP64 or MANIDSDP_PREC_MIXED for this call.
 */
int manidsdp_hessvec(manidsdp_ctx* ctx, const double* Y, const double* U, int32_t p,
                     double* HU, int32_t precision);

/*
 * manidsdp_lanczos - extreme eigenpair of the certificate
 *   X = Xt + D - Diag(z),  z = diag((Xt + D) Y Y')          (Algorithm 1, steps 7-9)
 * at the context's multiplier and the factor Y (device N x p FP64).  Lanczos
 * with full FP64 reorthogonalisation, at most k steps (k <= N; k <= 0 uses
 * params.lanczos_k).  which: MANIDSDP_EIG_MIN or _MAX.  Outputs: *lambda
 * (host), v (device N, unit norm, first nonzero entry positive; may be NULL),
 * *steps (host, may be NULL).
 */
int manidsdp_lanczos(manidsdp_ctx* ctx, const double* Y, int32_t p, int32_t which, int32_t k,
                     double* lambda, double* v, int32_t* steps);

/*
 * manidsdp_lanczos_dense_noalloc - extreme eigenpair of X - Diag(d) for a dense
 * symmetric matrix the caller already holds, without allocating device memory.
 * The paper has no counterpart.  It computes what manidsdp_lanczos computes
 * (Lanczos with full FP64 reorthogonalisation, the same start vector and sign
 * convention), but without a context, for callers that cannot allocate at the
 * call site: a serving loop whose device memory is held by a caching allocator
 * (a cudaMalloc there can fail although the cache has free blocks), or code that
 * cannot take the device-wide synchronisation a cudaFree implies.  Its Krylov
 * basis lives in one static device array of the library (4.4 MiB, held by every
 * device that loads the library until the process exits).
 *   N       order of X, 1 <= N <= 16384.
 *   X       device N x N FP64, row-major, symmetric (only read).  Must be
 *           readable by the current device: its device memory, managed memory
 *           or registered host memory; anything else gives E_ARG.
 *   d       device N FP64 subtracted on the diagonal, or NULL for none; e.g.
 *           X = Xt + D and d = z = diag((Xt + D) Y Y') give the certificate.
 *   which   MANIDSDP_EIG_MIN or MANIDSDP_EIG_MAX.
 *   k       Lanczos steps at most (k <= 0: min(N, 64); capped at N).
 *           Limits: k <= 256 and k * N <= 524288; beyond them, or N > 16384,
 *           the call returns MANIDSDP_E_TOOLARGE and does nothing else.
 *   lambda  host: the Ritz value.  v: host or device N FP64, unit norm, first
 *           entry above 1e-14 in magnitude positive (may be NULL).
 *   steps   host, may be NULL.  stream: cudaStream_t as void* (NULL = legacy
 *           default stream); it must belong to the current device.
 * Stopping: every 10 steps, when the Ritz pair at the requested end has a
 * residual below 1e-10 and the one at the other end below 1e-6 (relative to the
 * larger extreme Ritz value), or after k steps.
 * The call returns after its work on the stream has finished.  Nothing in the
 * scratch needs to be zero beforehand: each call clears what it accumulates.
 * Calls on the same device share the scratch: two calls in flight at the same
 * time on one device (two streams or two host threads) corrupt each other, so
 * serialise them.  Each call looks up the scratch's device address with
 * cudaGetSymbolAddress in the current context; the first call on a device also
 * loads the library's module there, so make that first call before any stream
 * capture begins on the device.
 * Errors: E_ARG (bad arguments), E_TOOLARGE (limits above), E_NONFINITE,
 * E_CUDA (a CUDA call failed).
 */
int manidsdp_lanczos_dense_noalloc(int32_t N, const double* X, const double* d, int32_t which,
                                   int32_t k, double* lambda, double* v, int32_t* steps,
                                   void* stream);

/*
 * manidsdp_solve - Algorithm 1 from the starting matrix Y0 (host or device,
 * N x p0 FP64, rows normalised by the library) to eta_max <= params.tol or
 * params.max_outer outer iterations.
 * Outputs (host or device; each may be NULL):
 *   Y_out  capacity N x params.p_max FP64; receives the final N x (*p_out) factor
 *          row-major with leading dimension *p_out;
 *   y_out  m FP64 (y at the final S);   z_out N FP64;
 *   Xt_out N x N FP64 final multiplier; report: host struct.
 * Returns MANIDSDP_OK when eta_max <= tol, MANIDSDP_E_NOCONV otherwise.
 * The context's multiplier and sigma are reset to 0 and params.sigma0 at entry,
 * unless params.warm_start = 1 continues the previous solve on this context.
 * The report's counters and phase times cover this call only.
 */
int manidsdp_solve(manidsdp_ctx* ctx, const double* Y0, int32_t p0, double* Y_out,
                   int32_t* p_out, double* y_out, double* z_out, double* Xt_out,
                   manidsdp_report* report);

/*
 * manidsdp_bqp_index_map - host helper: the moment-relaxation data of a binary
 * quadratic program min x'Qx + c'x, x in {-1,1}^q (Section 3.1).
 *   order 1: basis [1, x_1..x_q]; order 2: [1, x, x_1x_2, ..., x_{q-1}x_q].
 *   The class of entry (b, g) is the square-free monomial of the symmetric
 *   difference of the two basis monomials (x_i^2 = 1), ranked by degree and
 *   then lexicographically.
 * Pass idx = NULL to query *N and *m only.  idx: host N x N int32 output.
 */
int manidsdp_bqp_index_map(int32_t q, int32_t order, int32_t* N, int64_t* m, int32_t* idx);

/* Right-hand side b (host, m FP64 output) of the BQP relaxation: the
 * coefficients of x'Qx + c'x modulo x_i^2 = 1 on the canonical monomials:
 * b[1] = trace(Q), b[x_i] = c_i, b[x_i x_j] = 2 Q_ij (i < j), 0 otherwise.
 * Q: host q x q symmetric FP64; c: host q FP64 (NULL = 0).  Section 3.1. */
int manidsdp_bqp_rhs(int32_t q, int32_t order, const double* Q, const double* c, double* b);

/*
 * manidsdp_ucqp_index_map - host helper: the real second-order relaxation of a
 * unit-modulus complex quadratic program min x*Qx + Re(c'x), |x_i| = 1, with real
 * Q, c (Section 3.1, UCQP paragraph).  Basis: the Laurent exponents delta with
 * ||delta||_1 <= 2 (x_i conj(x_i) = 1 removed), N = 2q^2 + 2q + 1, ordered by
 * ||delta||_1 and then by the list of nonzero (index, value) pairs; the class of
 * entry (b, g) is {beta - gamma, gamma - beta} (real moments of delta and -delta
 * coincide), m = (q^4 + 2q^3 + 5q^2 + 4q + 3)/3 classes ordered the same way.
 * Pass idx = NULL to query *N and *m only.  idx: host N x N int32 output.
 */
int manidsdp_ucqp_index_map(int32_t q, int32_t* N, int64_t* m, int32_t* idx);

/* Right-hand side b (host, m FP64 output) of the UCQP relaxation: on the unit
 * torus x*Qx = trace(Q) + sum_{i != j} Q_ij x^(e_j - e_i) and
 * Re(c'x) = sum_i c_i (x^{e_i} + x^{-e_i}) / 2, each class collecting the
 * coefficients of delta and -delta.  Q: host q x q real symmetric; c: host q or NULL. */
int manidsdp_ucqp_rhs(int32_t q, const double* Q, const double* c, double* b);

/*
 * manidsdp_sparse_bqp_index_map - host helper: the second-order relaxation of a
 * sparse BQP with overlapping variable blocks (Section 6, sparse BQPs):
 * min sum_k x_k'Q_k x_k + c_k'x_k over x in {-1,1}^{(q-2)t+2}, block k (0-based)
 * holding the q variables (q-2)k .. (q-2)k+q-1.  The multi-block moment matrix
 * (t blocks of order n_b = 1 + q + q(q-1)/2) is embedded in one symmetric matrix of
 * order N = t n_b whose diagonal blocks carry the monomial classes (a square-free
 * monomial of degree <= 4 inside one block, ordered by degree and then
 * lexicographically on the sorted variables; *m_mono of them) and whose every
 * off-block pair {(r,c), (c,r)} is a class of its own (numbered after the
 * monomials, row-major in r < c; right-hand side 0).  The embedding has the
 * optimal value of the multi-block relaxation: a block-diagonal solution
 * extended by zeros is feasible for it, and the diagonal blocks of any of its
 * solutions are feasible for the block problem with the same objective.
 * q >= 2, t >= 1, N <= 65535.  Pass idx = NULL to query the sizes.
 * idx: host N x N int32 output.  m_mono may be NULL.
 */
int manidsdp_sparse_bqp_index_map(int32_t q, int32_t t, int32_t* N, int64_t* m,
                                  int64_t* m_mono, int32_t* idx);

/* Right-hand side b (host, m FP64 output) of the sparse BQP relaxation: the
 * coefficients of the objective modulo x_i^2 = 1 on the monomial classes (the
 * constant: the traces of the Q_k summed block by block; x_i: the c_k entries;
 * x_i x_j: Q_k[i][j] + Q_k[j][i], summed over the blocks sharing the monomial in
 * block order), 0 on the off-block classes.  Qs: host t x q x q row-major (each
 * symmetric); cs: host t x q or NULL. */
int manidsdp_sparse_bqp_rhs(int32_t q, int32_t t, const double* Qs, const double* cs, double* b);

/* ---- batched solve: many small instances in one persistent launch --------- */

/* Per-instance result of a batched solve (KKT residuals of Section 6). */
typedef struct {
  double value;                /* b'y, the relaxation value */
  double eta_p, eta_d, eta_g;  /* KKT residuals at the returned point */
  double lambda_min;           /* smallest eigenvalue of the certificate X */
  int32_t status;              /* MANIDSDP_OK, E_NOCONV or E_NONFINITE */
  int32_t p;                   /* final factor width (1 after an accepted rounding) */
  int32_t outer, hessvecs;     /* outer iterations, Hessian-vector products */
  int64_t cycles[5];           /* params.profile = 1: SM clock cycles of the instance's
                                  CTA spent in the whole solve, the Hessian-vector
                                  products, the certificate's eigenpairs, the
                                  subproblem evaluations and the eigenpairs of Y'Y
                                  (0 otherwise) */
} manidsdp_batch_out;

typedef struct manidsdp_batch manidsdp_batch; /* opaque, owned by the library */

/*
 * manidsdp_batch_setup - prepare ninst independent instances of (DSDP) with
 * C = 0 and index-map operators (as manidsdp_setup), each solved by Algorithm 1
 * in the same readings as manidsdp_solve, for one persistent kernel launch in
 * which every CTA takes whole instances from a device-side counter and runs the
 * outer loop, RTR/tCG, the multiplier update, the certificate's eigenpairs (a
 * parallel Jacobi method: the certificate is the full N x N X, computed exactly
 * rather than by Lanczos), the rank update, the sigma rule (5.1), the rank-one
 * rounding and the carried negative-curvature direction (Theorem 4.5) on the
 * device, with no host round trip.
 *   N[i] in [1, 128]; m[i] in [1, N[i]^2]: host arrays of length ninst.
 *   idx: host, the ninst full N[i] x N[i] index maps concatenated (row-major,
 *        symmetric, every class in [0, m[i]) nonempty).
 *   b:   host, the ninst right-hand sides concatenated (sum m[i] FP64).
 *   params: NULL for the defaults with p_max = 32; p_max <= 32; precision_mode
 *        MANIDSDP_PREC_MIXED (FP32 Hessian-vector products) or _FP64 (all FP64);
 *        profile = 1 fills manidsdp_batch_out.cycles; lanczos_k, tcg_device,
 *        tensor_cores, warm_start, verbose and tc_lowprec_eta are ignored.
 * Every starting factor is N[i] x p0.  Errors: E_ARG (as manidsdp_setup, or a size
 * above the limits), E_NONFINITE (b), E_NOMEM, E_CUDA.  The launch shape is the
 * one tuned earlier in the process for the same (max N, p_max, precision), else
 * 256 threads per CTA at the occupancy limit.
 */
int manidsdp_batch_setup(manidsdp_batch** batch, int32_t ninst, const int32_t* N,
                         const int64_t* m, const int32_t* idx, const double* b,
                         const manidsdp_params* params, void* stream);

/* Solve every instance from the starting factors Y0 (host or device: the N[i] x p0
 * factors concatenated; rows are normalised on the device).  res: host array of
 * ninst results or NULL; y: host or device, the optimal multipliers y_i (sum m[i]
 * FP64, concatenated; dV_i/db_i = y_i) or NULL; ms: device time of the launch or
 * NULL.  Returns MANIDSDP_OK when every instance met eta_max <= tol, E_NONFINITE if
 * one met a non-finite value, E_NOCONV if one reached max_outer (res tells which),
 * E_CUDA. */
int manidsdp_batch_solve(manidsdp_batch* batch, const double* Y0, manidsdp_batch_out* res,
                         double* y, float* ms);

/* Launch-shape tuner: solves the batch once for each shape (128, 256 or 512 threads
 * per CTA; 1, 2, 4, ... CTAs per SM up to the occupancy limit), keeps the fastest for
 * this batch and records it for later batches with the same (max N, p_max,
 * precision).  threads, ctas_per_sm: host outputs or NULL. */
int manidsdp_batch_tune(manidsdp_batch* batch, const double* Y0, int32_t* threads,
                        int32_t* ctas_per_sm);

/* Fix the launch shape: threads in {128, 256, 512}; ctas_per_sm 0 = the occupancy limit. */
int manidsdp_batch_set_launch(manidsdp_batch* batch, int32_t threads, int32_t ctas_per_sm);

/* Release the batch (NULL is a no-op). */
void manidsdp_batch_destroy(manidsdp_batch* batch);

/* One call: manidsdp_batch_setup, manidsdp_batch_solve, manidsdp_batch_destroy. */
int manidsdp_solve_batched(int32_t ninst, const int32_t* N, const int64_t* m, const int32_t* idx,
                           const double* b, const double* Y0, const manidsdp_params* params,
                           manidsdp_batch_out* res, double* y, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MANIDSDP_H */
