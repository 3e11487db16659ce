// Tensor-core (tcgen05, split-BF16 operands, FP32 accumulation) form of the
// restriction W^H x used by the FP32 V-cycle (restrict_tc.cu).
#pragma once

#include "qd_internal.cuh"

namespace qd {

// Whether the tensor-core restriction handles this transfer and call: fine
// dof per site in {12, 16, 24, 32}, coarse dof in {16, 24, 32}, 16-byte
// aligned fields, an even nrhs above 128.
bool restrict_tc_supported(const Transfer& T, const void* in, const void* out, int s);
// Make the split-BF16 copy of W (once).
void restrict_tc_prepare(qd_ctx& ctx, Transfer& T);
// coarse = W^H fine for s right-hand sides (interleaved complex FP32).
void restrict_tc(qd_ctx& ctx, Transfer& T, const cplxf* fine, cplxf* coarse, int s);
// Error code recorded by a bounded wait of the kernel (0: none); synchronises.
int restrict_tc_error(qd_ctx& ctx, const Transfer& T);

}  // namespace qd
