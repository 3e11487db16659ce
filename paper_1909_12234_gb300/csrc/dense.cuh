// Small dense linear algebra on device (see dense.cu).
#pragma once

#include "qd_internal.cuh"

namespace qd {

// G (ma x mb, row major) = X^H Y; X: n x ma with row stride ldx, Y: n x mb.
void blockdot(qd_ctx& ctx, int64_t n, const cplx* X, int ldx, int ma, const cplx* Y, int ldy, int mb,
              cplx* G);
// blockdot with caller-provided partial-sum space of `cap` complex numbers;
// allocates nothing; false if the space is too small.
bool blockdot_into(qd_ctx& ctx, int64_t n, const cplx* X, int ldx, int ma, const cplx* Y, int ldy, int mb,
                   cplx* G, cplx* partials, int64_t cap);
// Load blockdot_into's and blockmul's kernels on the current device.
void preload_projection_kernels();
// Y = alpha X S + beta Y; X: n x ma, S: ma x mb (row stride lds), Y: n x mb.
void blockmul(qd_ctx& ctx, int64_t n, const cplx* X, int ldx, int ma, const cplx* S, int lds, int mb,
              cplx* Y, int ldy, double alpha, double beta);
// Hermitian eigen-decomposition (one CTA): A overwritten, E eigenvectors
// (columns), w eigenvalues.  sweeps_dev (nullable) receives the sweep count.
void jacobi_eigh(qd_ctx& ctx, int m, cplx* A, cplx* E, double* w, int* sweeps_dev);
void sort_by_abs(qd_ctx& ctx, int m, const double* w, const cplx* E, double* wout, cplx* Eout, int* perm);
void hermitize(qd_ctx& ctx, int m, cplx* A);
// G = R^H R; G overwritten by R, Rinv = R^{-1}; flag set if not positive definite.
void cholesky_inverse(qd_ctx& ctx, int m, cplx* G, cplx* Rinv, int* flag_dev);
void scale_rows_inv(qd_ctx& ctx, int k, int s, const double* lam, cplx* Y);
void eig_residuals(qd_ctx& ctx, int64_t n, int m, const cplx* HX, const cplx* X, const double* theta,
                   cplx* out);

}  // namespace qd
