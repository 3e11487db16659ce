// The coarse-operator stencil (Sec. 2: C = W^H A W, "much denser" than A,
// Sec. 3.2) as a dense contraction on the tcgen05 tensor cores, for the FP32
// V-cycle.  For a coarse site x and a chunk of up to 128 right-hand sides:
//
//   y(x)[d][r] = sum_{dir=0..8} sum_e C_dir(x)[d][e] in(nb(x, dir))[e][r]
//
// is one real GEMM, M = 128 right-hand sides, N = 2D, K = 9 x 2D:
//   A[r][dir, 2e+p] = component p (re, im) of in(nb(x, dir))[e][r]
//   B[n][dir, 2e+p] = (Re C[n][e], -Im C[n][e])        for n <  D
//                     (Im C[n-D][e], Re C[n-D][e])      for n >= D
//   acc[r][n] = Re y[n][r] (n < D), Im y[n-D][r] (n >= D).
// The coarse operator is ill-conditioned near the critical mass, so plain
// BF16 operands (8 significant bits) perturb its small singular values too
// much for the coarse solve; each operand is therefore split into two BF16
// terms, v = hi + lo with hi = bf16(v), lo = bf16(v - hi) (16 bits together),
// and the product is formed as A_hi [B_hi | B_lo] + A_lo B_hi with FP32
// accumulation (relative error ~3 2^-16 per term; the lo x lo term is left
// out).  Each direction is one 64-wide K atom of which 2D columns are used.
//
// One persistent CTA per SM walks (site, chunk) items with warp roles:
//   warp 0 lane 0   bulk copies (cp.async.bulk) of the 9 neighbour blocks
//                   in(nb)[0..D)[r0..r0+w) (FP32) and of C_dir(x) (split
//                   BF16, compact) into a staging ring;
//   warps 8-15      split a staged direction into the swizzled K-major BF16
//                   operand tiles A_hi, A_lo (128 x 64) and B = [B_hi; B_lo]
//                   (4D x 64);
//   warp 1 lane 0   issues tcgen05.mma (K = 16 per instruction): A_hi B with
//                   N = 4D into columns [0, 4D) and A_lo B_hi with N = 2D
//                   into columns [0, 2D) of one of two TMEM accumulators;
//   warps 4-7       read the finished accumulator (tcgen05.ld), add the
//                   B_lo columns to the rest and write y.
// Every wait is an mbarrier wait bounded by 2 s of %globaltimer; on timeout
// the CTA records an error, stops, drains its copies and MMAs and frees TMEM.
#include <cuda_bf16.h>

#include <string>

#include "coarse_tc.cuh"
#include "ptx.cuh"
#include "tune.cuh"

namespace qd {

namespace {

using namespace ptx;

constexpr int kThreads = 512;
constexpr int kMaxNS = 4;  // staging ring depth
constexpr int kMaxNA = 8;  // operand-tile ring depth
constexpr uint32_t kATile = 128 * 128;  // 128 rows x 64 BF16 (one of A_hi, A_lo)
constexpr uint32_t kAccStride = 128;    // TMEM columns per accumulator
constexpr uint32_t kTmemCols = 256;     // two accumulators

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}
// Split (a, b) into BF16 pairs hi = bf16(a, b) and lo = bf16(a - hi_a, b - hi_b).
__device__ __forceinline__ void split_bf16x2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Wait that ignores the abort flag (used to drain work already in flight).
__device__ __forceinline__ bool mbar_wait_drain(uint32_t a, uint32_t parity) {
  const uint64_t t0 = gtimer();
  while (!mbar_try(a, parity))
    if (gtimer() - t0 > kTimeoutNs) return false;
  return true;
}

template <int D>
__global__ void __launch_bounds__(kThreads, 1)
    k_coarse_tc(int64_t nsites, int s, int nchunks, int NS, int NA, uint32_t stage_bytes, uint32_t b_tile,
                const int* __restrict__ nbr, const uint32_t* __restrict__ Cb, const float2* __restrict__ in,
                float2* __restrict__ out, int* __restrict__ err) {
  static_assert(D % 8 == 0 && D <= 32, "2D must be a multiple of 16 and at most 64");
  constexpr int KSTEPS = 2 * D / 16;
  constexpr int NCOL = 2 * D;
  constexpr uint32_t kCBytes = 2u * D * D * 4u;  // C_dir(x): hi pairs then lo pairs
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t sfull[kMaxNS], sempty[kMaxNS], afull[kMaxNA], aempty[kMaxNA];
  __shared__ __align__(8) uint64_t accf[2], acce[2], drain;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // layout: NA (A_hi, A_lo) tile pairs, NA B tiles, NS staging slots (1024-aligned)
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - smem_u32(smem_raw));
  const uint32_t a_off = 0, b_off = (uint32_t)NA * 2u * kATile, s_off = b_off + (uint32_t)NA * b_tile;
  const int64_t total = nsites * (int64_t)nchunks;
  if (tid == 0) {
    abort_flag = 0;
    for (int i = 0; i < NS; ++i) {
      mbar_init(smem_u32(&sfull[i]), 1);
      mbar_init(smem_u32(&sempty[i]), 256);
    }
    for (int i = 0; i < NA; ++i) {
      mbar_init(smem_u32(&afull[i]), 256);
      mbar_init(smem_u32(&aempty[i]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&accf[b]), 1);
      mbar_init(smem_u32(&acce[b]), 128);
    }
    mbar_init(smem_u32(&drain), 1);
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(smem_u32(&tmem_base), kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // ---- bulk-copy producer ----
      int last_use[kMaxNS];
      for (int i = 0; i < kMaxNS; ++i) last_use[i] = -1;
      int64_t q = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < total && ok; it += gridDim.x) {
        const int64_t x = it / nchunks;
        const int r0 = (int)(it - x * nchunks) * 128;
        const int w = min(128, s - r0);
        const uint32_t vbytes = (uint32_t)D * w * 8u;
        for (int j = 0; j < 9; ++j, ++q) {
          const int ss = (int)(q % NS);
          const int us = (int)(q / NS);
          if (us > 0 && !mbar_wait(smem_u32(&sempty[ss]), (uint32_t)(us - 1) & 1u, &abort_flag)) {
            atomicExch(err, 11);
            abort_flag = 1;
            ok = false;
            break;
          }
          const int64_t nb = j == 0 ? x : (int64_t)nbr[x * 8 + j - 1];
          const uint32_t dst = base + s_off + (uint32_t)ss * stage_bytes;
          const uint32_t bar = smem_u32(&sfull[ss]);
          mbar_expect_tx(bar, vbytes + kCBytes);
          if (nchunks == 1) {
            bulk_g2s(dst, in + nb * D * (int64_t)s, vbytes, bar);
          } else {
            for (int e = 0; e < D; ++e)
              bulk_g2s(dst + (uint32_t)e * w * 8u, in + (nb * D + e) * (int64_t)s + r0, (uint32_t)w * 8u, bar);
          }
          bulk_g2s(dst + vbytes, Cb + (x * 9 + j) * (int64_t)(2 * D * D), kCBytes, bar);
          last_use[ss] = us;
        }
      }
      // copies still in flight land before the CTA may exit
      for (int i = 0; i < NS; ++i)
        if (last_use[i] >= 0 && !mbar_wait_drain(smem_u32(&sfull[i]), (uint32_t)last_use[i] & 1u)) atomicExch(err, 12);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer ----
      const uint32_t idesc2 = idesc_bf16(128, 2 * NCOL);  // A_hi x [B_hi; B_lo]
      const uint32_t idesc1 = idesc_bf16(128, NCOL);      // A_lo x B_hi
      int64_t q = 0;
      int li = 0;
      bool issued = false, ok = true;
      for (int64_t it = blockIdx.x; it < total && ok; it += gridDim.x, ++li) {
        const int b = li & 1, ub = li >> 1;
        if (ub > 0 && !mbar_wait(smem_u32(&acce[b]), (uint32_t)(ub - 1) & 1u, &abort_flag)) {
          atomicExch(err, 13);
          abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)b * kAccStride;
        for (int j = 0; j < 9; ++j, ++q) {
          const int as = (int)(q % NA);
          const int ua = (int)(q / NA);
          if (!mbar_wait(smem_u32(&afull[as]), (uint32_t)ua & 1u, &abort_flag)) {
            atomicExch(err, 14);
            abort_flag = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t at = base + a_off + (uint32_t)as * 2u * kATile;
          const uint32_t bt = base + b_off + (uint32_t)as * b_tile;
#pragma unroll
          for (int k = 0; k < KSTEPS; ++k) {
            const uint64_t bdesc = sdesc_sw128(bt + (uint32_t)k * 32u);
            mma_bf16(acc, sdesc_sw128(at + (uint32_t)k * 32u), bdesc, idesc2, (j > 0 || k > 0) ? 1u : 0u);
            mma_bf16(acc, sdesc_sw128(at + kATile + (uint32_t)k * 32u), bdesc, idesc1, 1u);
          }
          mma_commit(smem_u32(&aempty[as]));
          issued = true;
        }
        if (ok) mma_commit(smem_u32(&accf[b]));
      }
      if (issued) {
        mma_commit(smem_u32(&drain));
        if (!mbar_wait_drain(smem_u32(&drain), 0)) atomicExch(err, 15);
      }
    }
  } else if (warp >= 4 && warp < 8) {
    // ---- epilogue: TMEM -> y ----
    const int ew = warp - 4;
    const int r = ew * 32 + lane;
    int li = 0;
    for (int64_t it = blockIdx.x; it < total; it += gridDim.x, ++li) {
      const int64_t x = it / nchunks;
      const int r0 = (int)(it - x * nchunks) * 128;
      const int w = min(128, s - r0);
      const int b = li & 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&accf[b]), (uint32_t)(li >> 1) & 1u, &abort_flag));
      if (!ok) {
        if (lane == 0) atomicExch(err, 16);
        abort_flag = 1;
        break;
      }
      tc_fence_after();
      float v[NCOL];
      const uint32_t taddr = tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)b * kAccStride;
#pragma unroll
      for (int c0 = 0; c0 < NCOL; c0 += 16) {
        uint32_t u0[16], u1[16];
        tmem_ld16(taddr + (uint32_t)c0, u0);
        tmem_ld16(taddr + (uint32_t)(NCOL + c0), u1);
        tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 16; ++i) v[c0 + i] = __uint_as_float(u0[i]) + __uint_as_float(u1[i]);
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&acce[b]));
      if (r < w) {
        float2* o = out + x * D * (int64_t)s + r0 + r;
#pragma unroll
        for (int d = 0; d < D; ++d) o[(int64_t)d * s] = make_float2(v[d], v[D + d]);
      }
    }
  } else if (warp >= 8) {
    // ---- converters: staged FP32 / compact BF16 -> swizzled operand tiles ----
    const int ct = tid - 256;
    int64_t q = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < total && ok; it += gridDim.x) {
      const int64_t x = it / nchunks;
      const int r0 = (int)(it - x * nchunks) * 128;
      const int w = min(128, s - r0);
      for (int j = 0; j < 9; ++j, ++q) {
        const int ss = (int)(q % NS), us = (int)(q / NS);
        const int as = (int)(q % NA), ua = (int)(q / NA);
        if (!mbar_wait(smem_u32(&sfull[ss]), (uint32_t)us & 1u, &abort_flag) ||
            (ua > 0 && !mbar_wait(smem_u32(&aempty[as]), (uint32_t)(ua - 1) & 1u, &abort_flag))) {
          atomicExch(err, 17);
          abort_flag = 1;
          ok = false;
          break;
        }
        const unsigned char* stg = gbase + s_off + (size_t)ss * stage_bytes;
        const float2* sv = reinterpret_cast<const float2*>(stg);
        const uint4* sc = reinterpret_cast<const uint4*>(stg + (size_t)D * w * 8);
        unsigned char* at = gbase + a_off + (size_t)as * 2 * kATile;
        unsigned char* bt = gbase + b_off + (size_t)as * b_tile;
        // A_hi, A_lo: row r, chunk c = components 2e+p for e = 4c..4c+3
        for (int idx = ct; idx < 128 * (D / 4); idx += 256) {
          const int rr = idx & 127, c = idx >> 7;
          if (rr < w) {
            const float2 v0 = sv[(4 * c + 0) * w + rr], v1 = sv[(4 * c + 1) * w + rr];
            const float2 v2 = sv[(4 * c + 2) * w + rr], v3 = sv[(4 * c + 3) * w + rr];
            uint4 h, l;
            split_bf16x2(v0.x, v0.y, h.x, l.x);
            split_bf16x2(v1.x, v1.y, h.y, l.y);
            split_bf16x2(v2.x, v2.y, h.z, l.z);
            split_bf16x2(v3.x, v3.y, h.w, l.w);
            const uint32_t off = sw128_offset(rr, 8 * c);
            *reinterpret_cast<uint4*>(at + off) = h;
            *reinterpret_cast<uint4*>(at + kATile + off) = l;
          }
        }
        // B: compact (re, im) BF16 pairs of C_dir[d][4c..4c+3], hi then lo
        // -> rows d (re, -im) and D + d (im, re) of B_hi (rows 0..2D) and of
        // B_lo (rows 2D..4D)
        for (int idx = ct; idx < 2 * D * (D / 4); idx += 256) {
          const int part = idx / (D * (D / 4));  // 0: hi, 1: lo
          const int rem = idx - part * (D * (D / 4));
          const int d = rem / (D / 4), c = rem - d * (D / 4);
          const uint4 cv = sc[idx];
          uint4 re, im;
          re.x = cv.x ^ 0x80000000u;
          re.y = cv.y ^ 0x80000000u;
          re.z = cv.z ^ 0x80000000u;
          re.w = cv.w ^ 0x80000000u;
          im.x = __byte_perm(cv.x, 0, 0x1032);
          im.y = __byte_perm(cv.y, 0, 0x1032);
          im.z = __byte_perm(cv.z, 0, 0x1032);
          im.w = __byte_perm(cv.w, 0, 0x1032);
          *reinterpret_cast<uint4*>(bt + sw128_offset(part * 2 * D + d, 8 * c)) = re;
          *reinterpret_cast<uint4*>(bt + sw128_offset(part * 2 * D + D + d, 8 * c)) = im;
        }
        fence_proxy_async_smem();
        mbar_arrive(smem_u32(&afull[as]));
        mbar_arrive(smem_u32(&sempty[ss]));
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) {
    __syncwarp();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// Compact split-BF16 copy of the stencil: for block (x, dir) of D x D
// entries, Cb[(x*9 + dir)][0][d][e] = hi and [1][d][e] = lo of (Re, Im) C,
// each pair one 32-bit word (real part in the low half).
__global__ void k_build_cb(int64_t nblk, int DD, const cplx* __restrict__ C, uint32_t* __restrict__ Cb) {
  const int64_t n = nblk * DD;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blk = e / DD, i = e - blk * DD;
    uint32_t hi, lo;
    split_bf16x2((float)C[e].x, (float)C[e].y, hi, lo);
    Cb[blk * 2 * DD + i] = hi;
    Cb[blk * 2 * DD + DD + i] = lo;
  }
}

// Launch with NS staging slots and as many operand stages as fit (at most
// kMaxNA); false (nothing launched) when fewer than two operand stages fit.
template <int D>
bool launch(qd_ctx& ctx, const CoarseLevel& lv, const cplxf* in, cplxf* out, int s, int* err, int NS) {
  const int nchunks = (s + 127) / 128;
  const int w = s < 128 ? s : 128;
  const uint32_t b_tile = (uint32_t)((4 * D * 128 + 1023) / 1024 * 1024);
  const uint32_t stage = (uint32_t)(((size_t)D * w * 8 + (size_t)2 * D * D * 4 + 1023) / 1024 * 1024);
  const size_t budget = 220 * 1024;
  if (NS > kMaxNS || 1024 + (size_t)NS * stage + 2 * (2 * kATile + b_tile) > budget) return false;
  int NA = (int)((budget - 1024 - (size_t)NS * stage) / (2 * kATile + b_tile));
  if (NA > kMaxNA) NA = kMaxNA;
  const size_t smem = 1024 + (size_t)NA * (2 * kATile + b_tile) + (size_t)NS * stage;
  ensure_smem_limit(reinterpret_cast<const void*>(k_coarse_tc<D>), smem);
  const int64_t items = lv.geo.nsites * (int64_t)nchunks;
  const int grid = (int)(items < kNumSMs ? items : kNumSMs);
  k_coarse_tc<D><<<grid, kThreads, smem, ctx.stream>>>(lv.geo.nsites, s, nchunks, NS, NA, stage, b_tile,
                                                        lv.geo.nbr.as<int>(), lv.Cmb.as<uint32_t>(),
                                                        reinterpret_cast<const float2*>(in),
                                                        reinterpret_cast<float2*>(out), err);
  QD_LAUNCH_CHECK();
  return true;
}

}  // namespace

bool coarse_tc_supported(const CoarseLevel& lv, const void* in, const void* out, int s) {
  const int D = lv.D;
  if (!(D == 8 || D == 16 || D == 24 || D == 32)) return false;
  if (s < 1) return false;
  if (((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) != 0) return false;
  // more than one chunk: every row of a block is its own copy, which must
  // start on a 16-byte boundary
  if (s > 128 && (s & 1)) return false;
  return true;
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
  if (lv.ctc_err.bytes() == 0) {
    lv.ctc_err.resize(sizeof(int));
    QD_CUDA(cudaMemsetAsync(lv.ctc_err.as<int>(), 0, sizeof(int), ctx.stream));
  }
}

void coarse_apply_tc(qd_ctx& ctx, CoarseLevel& lv, const cplxf* in, cplxf* out, int s) {
  QD_REQUIRE(coarse_tc_supported(lv, in, out, s), "tensor-core coarse stencil: unsupported size or alignment");
  coarse_tc_prepare(ctx, lv);
  const double D = lv.D;
  ProfScope ps(ctx, QD_PROF_COARSE_TC, 72.0 * D * D * (double)lv.geo.nsites * s,
               (double)lv.geo.nsites * (9.0 * D * D * 8.0 + 2.0 * D * 8.0 * s));
  int* err = lv.ctc_err.as<int>();
  // candidates: 2, 3 or 4 staging slots (deeper prefetch against fewer
  // operand stages); every candidate computes the same sums in the same order
  auto go = [&](int c) -> bool {
    const int NS = 2 + c;
    switch (lv.D) {
      case 8: return launch<8>(ctx, lv, in, out, s, err, NS);
      case 16: return launch<16>(ctx, lv, in, out, s, err, NS);
      case 24: return launch<24>(ctx, lv, in, out, s, err, NS);
      default: return launch<32>(ctx, lv, in, out, s, err, NS);
    }
  };
  const std::string key = "coarse_tc D" + std::to_string(lv.D) + " sites" + std::to_string(lv.geo.nsites) + " rhs" +
                          std::to_string(s);
  const int c = tune_pick(ctx, key, 3, go);
  if (c >= 0 && go(c)) return;
  for (int d = 0; d < 3; ++d)
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
