// Restriction W^H x (Sec. 2 two-grid step 1) as a dense contraction on the
// tcgen05 tensor cores, for the FP32 V-cycle: k_block_tc (block_tc.cuh) with
// the aggregate's fine sites as its input blocks and b_m = W^H of site m
// (conj(W) restricted to the output's chirality).
#include <string>

#include "block_tc.cuh"
#include "restrict_tc.cuh"
#include "tune.cuh"

namespace qd {

namespace {

// Split-BF16 copy of W: Wb[s][0][a][v] = hi and [1][a][v] = lo of (Re, Im)
// W[s][a][v], each pair one 32-bit word (real part in the low half).
__global__ void k_build_wb(int64_t nsite, int DV, const cplx* __restrict__ W, uint32_t* __restrict__ Wb) {
  const int64_t n = nsite * DV;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t st = e / DV, i = e - st * DV;
    uint32_t hi, lo;
    blocktc::split_bf16x2((float)W[e].x, (float)W[e].y, hi, lo);
    Wb[st * 2 * DV + i] = hi;
    Wb[st * 2 * DV + DV + i] = lo;
  }
}

template <int DIN, int DOUT>
bool launch(qd_ctx& ctx, const Transfer& T, const cplxf* in, cplxf* out, int s, int* err, int NS) {
  return blocktc::launch<DIN, DOUT, blocktc::kRestrict>(ctx, T.ncoarse, T.bsites, T.members.as<int>(),
                                                        T.Wtc.as<uint32_t>(), in, out, s, err, NS);
}

template <int DIN>
bool launch_dout(qd_ctx& ctx, const Transfer& T, const cplxf* in, cplxf* out, int s, int* err, int NS) {
  switch (T.Dc) {
    case 16: return launch<DIN, 16>(ctx, T, in, out, s, err, NS);
    case 24: return launch<DIN, 24>(ctx, T, in, out, s, err, NS);
    default: return launch<DIN, 32>(ctx, T, in, out, s, err, NS);
  }
}

}  // namespace

bool restrict_tc_supported(const Transfer& T, const void* in, const void* out, int s) {
  if (!(T.Df == 12 || T.Df == 16 || T.Df == 24 || T.Df == 32)) return false;
  if (!(T.Dc == 16 || T.Dc == 24 || T.Dc == 32)) return false;
  return blocktc::fields_ok(in, out, s);
}

void restrict_tc_prepare(qd_ctx& ctx, Transfer& T) {
  if (T.Wtc.bytes() > 0) return;
  const int DV = T.Df * T.nv;
  const int64_t n = T.nfine * (int64_t)DV;
  T.Wtc.resize((size_t)2 * n * sizeof(uint32_t));
  k_build_wb<<<(int)std::min<int64_t>((n + 255) / 256, 32 * kNumSMs), 256, 0, ctx.stream>>>(T.nfine, DV, T.W.as<cplx>(),
                                                                                          T.Wtc.as<uint32_t>());
  QD_LAUNCH_CHECK();
  if (T.rtc_err.bytes() == 0) {
    T.rtc_err.resize(sizeof(int));
    QD_CUDA(cudaMemsetAsync(T.rtc_err.as<int>(), 0, sizeof(int), ctx.stream));
  }
}

void restrict_tc(qd_ctx& ctx, Transfer& T, const cplxf* fine, cplxf* coarse, int s) {
  QD_REQUIRE(restrict_tc_supported(T, fine, coarse, s), "tensor-core restriction: unsupported size or alignment");
  restrict_tc_prepare(ctx, T);
  ProfScope ps(ctx, QD_PROF_RESTRICT_TC, 8.0 * T.nv * (double)T.nfine * T.Df * s,
               8.0 * ((double)T.nfine * T.Df * T.nv + (double)T.nfine * T.Df * s + (double)T.ncoarse * T.Dc * s));
  int* err = T.rtc_err.as<int>();
  auto go = [&](int c) -> bool {
    const int NS = 2 + c;
    switch (T.Df) {
      case 12: return launch_dout<12>(ctx, T, fine, coarse, s, err, NS);
      case 16: return launch_dout<16>(ctx, T, fine, coarse, s, err, NS);
      case 24: return launch_dout<24>(ctx, T, fine, coarse, s, err, NS);
      default: return launch_dout<32>(ctx, T, fine, coarse, s, err, NS);
    }
  };
  const std::string key = "restrict_tc Df" + std::to_string(T.Df) + " Dc" + std::to_string(T.Dc) + " agg" +
                          std::to_string(T.ncoarse) + " rhs" + std::to_string(s);
  const int c = tune_pick(ctx, key, 3, go);
  if (c >= 0 && go(c)) return;
  for (int d = 0; d < 3; ++d)
    if (go(d)) return;
  fail(QD_ERR_INVALID, "tensor-core restriction: operand tiles do not fit in shared memory");
}

int restrict_tc_error(qd_ctx& ctx, const Transfer& T) {
  if (T.rtc_err.bytes() == 0) return 0;
  int h = 0;
  QD_CUDA(cudaMemcpyAsync(&h, T.rtc_err.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaStreamSynchronize(ctx.stream));
  return h;
}

}  // namespace qd
