// Tensor-core (tcgen05, BF16 operands, FP32 accumulation) form of the
// coarse-operator stencil used by the FP32 V-cycle (coarse_tc.cu).
#pragma once

#include "qd_internal.cuh"

namespace qd {

// Whether the tensor-core stencil handles this level and call: dof per site
// in {8, 16, 24, 32}, 16-byte aligned fields, an even nrhs above 128.
bool coarse_tc_supported(const CoarseLevel& lv, const void* in, const void* out, int s);
// Make the compact BF16 copy of the level's stencil (once).
void coarse_tc_prepare(qd_ctx& ctx, CoarseLevel& lv);
// out = C in for s right-hand sides (interleaved complex FP32 in and out);
// with b: out = b - C in (b may not alias out or in).
void coarse_apply_tc(qd_ctx& ctx, CoarseLevel& lv, const cplxf* in, cplxf* out, int s, const cplxf* b = nullptr);
// Error code recorded by a bounded wait of the kernel (0: none); synchronises.
int coarse_tc_error(qd_ctx& ctx, const CoarseLevel& lv);

}  // namespace qd
