// The coarse-operator stencil (Sec. 2: C = W^H A W, "much denser" than A,
// Sec. 3.2) as a dense contraction on the tcgen05 tensor cores, for the FP32
// V-cycle: k_block_tc (block_tc.cuh) with the nine directions of the
// stencil as its input blocks, b_j = C_dir(x).
#include <string>

#include "block_tc.cuh"
#include "coarse_tc.cuh"
#include "tune.cuh"

namespace qd {

namespace {

constexpr int kCoarseTcCandidates = 11;

// Compact split-BF16 copy of the stencil: for block (x, dir) of D x D
// entries, Cb[(x*9 + dir)][0][d][e] = hi and [1][d][e] = lo of (Re, Im) C,
// each pair one 32-bit word (real part in the low half).
__global__ void k_build_cb(int64_t nblk, int DD, const cplx* __restrict__ C, uint32_t* __restrict__ Cb) {
  const int64_t n = nblk * DD;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blk = e / DD, i = e - blk * DD;
    uint32_t hi, lo;
    blocktc::split_bf16x2((float)C[e].x, (float)C[e].y, hi, lo);
    Cb[blk * 2 * DD + i] = hi;
    Cb[blk * 2 * DD + DD + i] = lo;
  }
}

template <int D>
bool launch(qd_ctx& ctx, const CoarseLevel& lv, const cplxf* in, cplxf* out, int s, int* err, int NS,
            const cplxf* b) {
  return blocktc::launch<D, D, blocktc::kStencil>(ctx, lv.geo.nsites, 9, lv.sten_src.as<int>(),
                                                  lv.Cmb.as<uint32_t>(), in, out, s, err, NS, b);
}

template <int D>
bool launch_split(qd_ctx& ctx, const CoarseLevel& lv, const cplxf* in, cplxf* out, int s, int* err, int NA,
                  bool region_copies, bool two_per_sm, const cplxf* b) {
  const size_t need = (size_t)lv.geo.nsites * ((s + 127) / 128) * blocktc::split_tile_bytes<D>();
  if (lv.ctc_tiles.bytes() < need) lv.ctc_tiles.resize(need);
  return blocktc::launch_split<D>(ctx, lv.geo.nsites, lv.sten_src.as<int>(), lv.Cmb.as<uint32_t>(), in,
                                  lv.ctc_tiles.as<unsigned char>(), out, s, err, NA, region_copies, two_per_sm, b);
}

}  // namespace

bool coarse_tc_supported(const CoarseLevel& lv, const void* in, const void* out, int s) {
  const int D = lv.D;
  if (!(D == 8 || D == 16 || D == 24 || D == 32)) return false;
  return blocktc::fields_ok(in, out, s);
}

void coarse_tc_prepare(qd_ctx& ctx, CoarseLevel& lv) {
  if (lv.Cmb.bytes() > 0) return;
  const int64_t nblk = lv.geo.nsites * 9;
  const int DD = lv.D * lv.D;
  const int64_t n = nblk * DD;
  lv.Cmb.resize((size_t)2 * n * sizeof(uint32_t));
  k_build_cb<<<(int)std::min<int64_t>((n + 255) / 256, 32 * kNumSMs), 256, 0, ctx.stream>>>(
      nblk, DD, lv.Cm.as<cplx>(), lv.Cmb.as<uint32_t>());
  QD_LAUNCH_CHECK();
  // input block of direction j: the site itself (j = 0) and its neighbours
  std::vector<int> src((size_t)lv.geo.nsites * 9);
  for (int64_t x = 0; x < lv.geo.nsites; ++x) {
    src[x * 9] = (int)x;
    for (int h = 0; h < 8; ++h) src[x * 9 + 1 + h] = lv.geo.h_nbr[x * 8 + h];
  }
  lv.sten_src.resize(src.size() * sizeof(int));
  QD_CUDA(cudaMemcpyAsync(lv.sten_src.as<int>(), src.data(), src.size() * sizeof(int), cudaMemcpyHostToDevice,
                          ctx.stream));
  QD_CUDA(cudaStreamSynchronize(ctx.stream));  // the host table goes out of scope
  if (lv.ctc_err.bytes() == 0) {
    lv.ctc_err.resize(sizeof(int));
    QD_CUDA(cudaMemsetAsync(lv.ctc_err.as<int>(), 0, sizeof(int), ctx.stream));
  }
}

void coarse_apply_tc(qd_ctx& ctx, CoarseLevel& lv, const cplxf* in, cplxf* out, int s, const cplxf* b) {
  QD_REQUIRE(coarse_tc_supported(lv, in, out, s), "tensor-core coarse stencil: unsupported size or alignment");
  coarse_tc_prepare(ctx, lv);
  const double D = lv.D;
  ProfScope ps(ctx, QD_PROF_COARSE_TC, 72.0 * D * D * (double)lv.geo.nsites * s,
               (double)lv.geo.nsites * (9.0 * D * D * 8.0 + (b ? 3.0 : 2.0) * D * 8.0 * s));
  int* err = lv.ctc_err.as<int>();
  // candidates 0-3: the input split once into operand tiles first
  // (k_split_tiles), at most 8, 4, 3 or 2 operand slots, one bulk copy per
  // tile; 4-6: the input blocks converted inside the kernel with 2, 3 or 4
  // staging slots; 7-8: split tiles, at most 8 or 4 slots, one bulk copy per
  // 4 KB region of a tile; 9-10: split tiles with two CTAs of 256 threads per
  // SM (two pipelines), at most 8 or 2 slots each.  Every candidate forms the
  // same BF16 operands and issues the same MMAs in the same order.
  auto go = [&](int c) -> bool {
    if (c >= 4 && c <= 6) {
      const int NS = c - 2;
      switch (lv.D) {
        case 8: return launch<8>(ctx, lv, in, out, s, err, NS, b);
        case 16: return launch<16>(ctx, lv, in, out, s, err, NS, b);
        case 24: return launch<24>(ctx, lv, in, out, s, err, NS, b);
        default: return launch<32>(ctx, lv, in, out, s, err, NS, b);
      }
    }
    static const int kNA[11] = {8, 4, 3, 2, 0, 0, 0, 8, 4, 8, 2};
    const int NA = kNA[c];
    const bool rc = c == 7 || c == 8;
    const bool two = c >= 9;
    switch (lv.D) {
      case 8: return launch_split<8>(ctx, lv, in, out, s, err, NA, rc, two, b);
      case 16: return launch_split<16>(ctx, lv, in, out, s, err, NA, rc, two, b);
      case 24: return launch_split<24>(ctx, lv, in, out, s, err, NA, rc, two, b);
      default: return launch_split<32>(ctx, lv, in, out, s, err, NA, rc, two, b);
    }
  };
  const std::string key = "coarse_tc D" + std::to_string(lv.D) + " sites" + std::to_string(lv.geo.nsites) + " rhs" +
                          std::to_string(s) + (b ? " res" : "");
  const int c = tune_pick(ctx, key, kCoarseTcCandidates, go);
  if (c >= 0 && go(c)) return;
  for (int d = 0; d < kCoarseTcCandidates; ++d)
    if (go(d)) return;
  fail(QD_ERR_INVALID, "tensor-core coarse stencil: operand tiles do not fit in shared memory");
}

int coarse_tc_error(qd_ctx& ctx, const CoarseLevel& lv) {
  if (lv.ctc_err.bytes() == 0) return 0;
  int h = 0;
  QD_CUDA(cudaMemcpyAsync(&h, lv.ctc_err.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaStreamSynchronize(ctx.stream));
  return h;
}

}  // namespace qd
