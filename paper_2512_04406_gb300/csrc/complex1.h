// Internal interface of the first-order complex relaxation (complex1.cu):
//   min <Q, S>  over Hermitian S >= 0 with diag(S) = 1,  Q = Qre + i Qim Hermitian,
// the relaxation of min z^H Q z over |z_i| = 1.  Every off-diagonal entry is a
// class of its own, so the projector residual vanishes on the manifold and the
// ALM is a rank-adaptive Riemannian trust region on the complex oblique
// manifold {Y in C^{n x p}: |Y_i| = 1}, certified by X = Q - Diag(mu),
// mu_i = Re (Q Y Y^H)_ii (Lemma 4.1, Proposition 4.2 with G = Q, Theorem 4.5 for
// the escape direction).  A complex factor Y = A + iB is held as the real n x 2p
// array [A | B] (row-major): its rows are the rows of the real oblique manifold,
// and G Y = Qre [A | B] + Qim [-B | A].
#pragma once

#include "common.cuh"

namespace mds {

struct ComplexState;

int complex_setup(ComplexState** out, int n, const double* qre, const double* qim,
                  const manidsdp_params& prm, cudaStream_t s);
void complex_destroy(ComplexState* cs);
int complex_set_params(ComplexState* cs, const manidsdp_params& prm);
// p: complex columns (arrays n x 2p).  psi, rnorm host; rgrad, z device (may be NULL).
int complex_eval(ComplexState* cs, const double* Y, int p, double* psi, double* rgrad, double* z);
int complex_hessvec(ComplexState* cs, const double* Y, const double* U, int p, double* HU,
                    int precision);
int complex_lanczos(ComplexState* cs, const double* Y, int p, int which, int k, double* lambda,
                    double* v, int* steps);
int complex_solve(ComplexState* cs, const double* Y0, int p0, double* Y_out, int* p_out,
                  double* z_out, manidsdp_report* rep);

}  // namespace mds
