// Dense direct solves on the coarsest level (see direct.cu).
#pragma once

#include "qd_internal.cuh"

namespace qd {

// In-place inverse of an n x n complex FP64 matrix (row major), Gauss-Jordan
// with partial pivoting.  Fails with QD_ERR_NONFINITE on a zero pivot.
void gauss_jordan_inverse(qd_ctx& ctx, int n, cplx* A);
// lv.Cinv = dense inverse of the level's stencil operator, lv.ndense = n.
void coarse_dense_inverse(qd_ctx& ctx, CoarseLevel& lv);
// Y (n x s) = M (n x n) X (n x s), row major, complex, FP64 or FP32.
template <class C> void dense_apply(qd_ctx& ctx, int n, int s, const C* M, const C* X, C* Y);

}  // namespace qd
