// Dense direct solves on the coarsest level (see direct.cu).
#pragma once

#include "qd_internal.cuh"

namespace qd {

// In-place inverse of an n x n complex matrix (row major, FP64 or FP32),
// Gauss-Jordan with partial pivoting.  Fails with QD_ERR_NONFINITE on a zero
// pivot.
template <class C> void gauss_jordan_inverse(qd_ctx& ctx, int n, C* A);
// lv.Cinvf = dense inverse of the level's stencil operator (FP32
// Gauss-Jordan), lv.Cinv = the same widened to FP64, lv.ndense = n.
void coarse_dense_inverse(qd_ctx& ctx, CoarseLevel& lv);
// y = C^{-1} x to FP64 accuracy on a level with a dense inverse: the stored
// inverse applied, then `steps` residual corrections with the FP64 stencil.
void coarsest_solve_refined(qd_ctx& ctx, const CoarseLevel& lv, int nrhs, const cplx* x, cplx* y, int steps);
// Y (n x s) = M (n x n) X (n x s), row major, complex, FP64 or FP32.
template <class C> void dense_apply(qd_ctx& ctx, int n, int s, const C* M, const C* X, C* Y);

}  // namespace qd
