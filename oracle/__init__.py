"""FP64 CPU oracle of ManiDSDP (arXiv 2512.04406) — TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct NumPy code that states the paper's formulas one
step at a time.  Only the tests, the smoke check and the benchmark's CPU-baseline
leg may import it; the library under ``paper_2512_04406_gb300`` never does, and
this package never imports the library.

Modules
  moment     BQP moment-relaxation data: basis, monomial ranks, index map,
             multiplicities, right-hand side b (Section 3.1, Eq. (BQP)).
  operators  A, A*, y(S), P, Q, D (Section 3 and Eq. (projection-operators)).
  subproblem Psi_k, grad, Hess, tangent projector, retraction (Section 4,
             Lemma 4.1, Proposition 4.2).
  rtr        Riemannian trust region with truncated CG (textbook RTR cited in
             Section 4).
  manidsdp   Algorithm 1 (ManiDSDP) with the one-step-delayed curvature carry
             (Section 5.1), the sigma rule (Eq. (5.1)), the KKT residuals of
             Section 6, rank-one rounding.
  lanczos    Lanczos with full reorthogonalisation for lambda_min / lambda_max
             of the certificate (Algorithm 1, step 9 and the remark on partial
             eigendecompositions).
  brute      Exhaustive BQP minimum over {-1,1}^q (weak-duality pin).

Parity status: every function here is pinned by a `-m "not gpu"` test against a
closed form, an invariant of the paper, brute force, or finite differences; none
is "parity unpinned".
"""
