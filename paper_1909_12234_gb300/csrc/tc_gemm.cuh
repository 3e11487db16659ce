// Coarsest-level dense solve on tcgen05 tensor cores (see tc_gemm.cu).
#pragma once

#include "blas.cuh"

namespace qd {

inline int blas_grid(int64_t tot) { return blas::grid_1d(tot); }

// Build the BF16 operand [Re C^{-1} | Im C^{-1}] and its TMA map (setup).
void tc_prepare(qd_ctx& ctx, CoarseLevel& lv);
// Y = C^{-1} X (complex FP32, n x s, RHS innermost) with BF16 inputs and FP32
// accumulation on the tensor cores.
void tc_dense_apply(qd_ctx& ctx, CoarseLevel& lv, const cplxf* X, cplxf* Y, int s);
// Error flag of the last launches (1-3: a bounded wait timed out), 0 if none.
int tc_error(qd_ctx& ctx, CoarseLevel& lv);

}  // namespace qd
