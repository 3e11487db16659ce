// Block contractions on the tcgen05 tensor cores (sm_103a) shared by the
// coarse-operator stencil and the restriction of the FP32 V-cycle.
//
// For an output site x and a chunk of up to 128 right-hand sides,
//   y(x)[d][r] = sum_{j < nstep} sum_e b_j(x)[d][e] in(src(x, j))[e][r]
// (d < DOUT, e < DIN) is one real GEMM, M = 128 right-hand sides,
// N = 2 DOUT, K = nstep x 2 DIN:
//   A[r][j, 2e+p] = component p (re, im) of in(src(x, j))[e][r]
//   B[d][j, 2e+p] = (Re b, -Im b),  B[DOUT+d][j, 2e+p] = (Im b, Re b)
//   acc[r][n] = Re y[n][r] (n < DOUT), Im y[n-DOUT][r] (n >= DOUT).
// Coarse stencil (MODE kStencil): nstep = 9 directions, src = the site and
// its eight neighbours, b_j = C_dir(x).  Restriction (MODE kRestrict): nstep
// = the aggregate's fine sites, src = those sites, b_j[c nv + v][e] =
// conj(W[s][e][v]) for e of chirality c and 0 across chiralities (W^H of
// one site).
// Operands are split into two BF16 terms, v = hi + lo with hi = bf16(v),
// lo = bf16(v - hi) (16 significant bits together): the coarse operator is
// ill-conditioned near the critical mass and plain BF16 (8 bits) perturbs
// its small singular values too much.  The product is A_hi [B_hi | B_lo] +
// A_lo B_hi with FP32 accumulation (lo x lo left out; error ~3 2^-16 per
// term).  Each input block is one 64-wide K atom of which 2 DIN columns are
// used (zero padded to a multiple of 16).
//
// One persistent CTA per SM walks (x, chunk) items with warp roles:
//   warp 0 lane 0   bulk copies (cp.async.bulk) of the input blocks
//                   in(src)[0..DIN)[r0..r0+w) (FP32) and of b_j (compact
//                   split BF16) into a staging ring;
//   warps 8-15      split a staged block into the swizzled K-major BF16
//                   operand tiles A_hi, A_lo (128 x 64) and B = [B_hi; B_lo]
//                   (4 DOUT x 64);
//   warp 1 lane 0   issues tcgen05.mma (K = 16 per instruction): A_hi B with
//                   N = 4 DOUT into columns [0, 4 DOUT) and A_lo B_hi with
//                   N = 2 DOUT into columns [0, 2 DOUT) of one of two TMEM
//                   accumulators;
//   warps 4-7       read the finished accumulator (tcgen05.ld), add the B_lo
//                   columns to the rest and write y.
// Every wait is an mbarrier wait bounded by 2 s of %globaltimer; on timeout
// the CTA records an error, stops, drains its copies and MMAs and frees TMEM.
#pragma once

#include <cuda_bf16.h>

#include "ptx.cuh"
#include "qd_internal.cuh"

namespace qd {
namespace blocktc {

using namespace ptx;

enum { kStencil = 0, kRestrict = 1, kStencilSplit = 2 };

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

// Source indices the producer loads one item ahead.
constexpr int kPrefetch = 16;
__device__ __forceinline__ void prefetch_src(const int* __restrict__ src, int nstep, int nchunks, int64_t total,
                                             int64_t item, int pre[kPrefetch]) {
  const bool valid = item < total;
  const int64_t x = valid ? item / nchunks : 0;
#pragma unroll
  for (int j = 0; j < kPrefetch; ++j) pre[j] = (valid && j < nstep) ? src[x * nstep + j] : 0;
}

// Wait that ignores the abort flag (used to drain work already in flight).
__device__ __forceinline__ bool mbar_wait_drain(uint32_t a, uint32_t parity) {
  const uint64_t t0 = gtimer();
  while (!mbar_try(a, parity))
    if (gtimer() - t0 > kTimeoutNs) return false;
  return true;
}

// B tile of one input block from its compact split-BF16 coefficients sw
// (hi block, then lo): for output row d the complex coefficients b[d][e] of
// y[d] = sum_e b[d][e] in[e], as rows d (Re b, -Im b) and DOUT + d
// (Im b, Re b) of B_hi (rows 0..2 DOUT) and of B_lo (2 DOUT..4 DOUT), K-major
// with 128-byte swizzle; K chunks past DIN/4 that the MMAs read are zero.
template <int DIN, int DOUT, int MODE>
__device__ __forceinline__ void build_b_tile(int ct, int nct, const uint32_t* sw, unsigned char* bt) {
  constexpr int KSTEPS = (2 * DIN + 15) / 16;
  constexpr int KCH = 2 * KSTEPS;
  constexpr int NV = DOUT / 2;
  for (int idx = ct; idx < 2 * DOUT * KCH; idx += nct) {
    const int part = idx / (DOUT * KCH);  // 0: hi, 1: lo
    const int rem = idx - part * (DOUT * KCH);
    const int d = rem / KCH, c = rem - d * KCH;
    uint4 re = make_uint4(0u, 0u, 0u, 0u), im = re;
    if (c < DIN / 4) {
      uint32_t bw[4];
      if (MODE != kRestrict) {
        // b = C_dir[d][e], stored (Re, Im)
        const uint4 cv = *reinterpret_cast<const uint4*>(sw + part * DOUT * DIN + d * DIN + 4 * c);
        bw[0] = cv.x; bw[1] = cv.y; bw[2] = cv.z; bw[3] = cv.w;
#pragma unroll
        for (int i = 0; i < 4; ++i) bw[i] ^= 0x80000000u;  // (Re b, -Im b)
      } else {
        // b = conj(W[e][j]) on the output's chirality, 0 across:
        // (Re b, -Im b) = (Re W, Im W) as stored
        const int jv = d % NV, cout = d / NV;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int e = 4 * c + i;
          bw[i] = (e / (DIN / 2) == cout) ? sw[part * DIN * NV + e * NV + jv] : 0u;
        }
      }
      re = make_uint4(bw[0], bw[1], bw[2], bw[3]);
      // (Im b, Re b) from (Re b, -Im b): swap halves, negate the low one
      im.x = __byte_perm(bw[0], 0, 0x1032) ^ 0x00008000u;
      im.y = __byte_perm(bw[1], 0, 0x1032) ^ 0x00008000u;
      im.z = __byte_perm(bw[2], 0, 0x1032) ^ 0x00008000u;
      im.w = __byte_perm(bw[3], 0, 0x1032) ^ 0x00008000u;
    }
    *reinterpret_cast<uint4*>(bt + sw128_offset(part * 2 * DOUT + d, 8 * c)) = re;
    *reinterpret_cast<uint4*>(bt + sw128_offset(part * 2 * DOUT + DOUT + d, 8 * c)) = im;
  }
}

template <int DIN, int DOUT, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    k_block_tc(int64_t nout, int nstep, int s, int nchunks, int NS, int NA, uint32_t stage_bytes, uint32_t b_tile,
               const int* __restrict__ src, const uint32_t* __restrict__ Bsrc, const float2* __restrict__ in,
               float2* __restrict__ out, int* __restrict__ err, const float2* __restrict__ bres = nullptr) {
  static_assert(DOUT % 8 == 0 && DOUT <= 32, "2 DOUT must be a multiple of 16 and at most 64");
  static_assert(DIN % 4 == 0 && DIN <= 32, "DIN must be a multiple of 4 and at most 32");
  constexpr int KSTEPS = (2 * DIN + 15) / 16;  // MMA K steps of 16 per input block
  constexpr int KCH = 2 * KSTEPS;              // 16-byte chunks of a K row the MMAs read
  constexpr int NCOL = 2 * DOUT;
  constexpr int NV = DOUT / 2;
  constexpr uint32_t kBWords = MODE == kStencil ? 2u * DOUT * DIN : 2u * DIN * NV;  // hi block, then lo
  constexpr uint32_t kCBytes = kBWords * 4u;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t sfull[kMaxNS], sempty[kMaxNS], afull[kMaxNA], aempty[kMaxNA];
  __shared__ int s_src[kPrefetch];  // the producer's source indices of the current item
  __shared__ __align__(8) uint64_t accf[2], acce[2], drain;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // layout: NA (A_hi, A_lo) tile pairs, NA B tiles, NS staging slots (1024-aligned)
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - smem_u32(smem_raw));
  const uint32_t a_off = 0, b_off = (uint32_t)NA * 2u * kATile, s_off = b_off + (uint32_t)NA * b_tile;
  const int64_t total = nout * (int64_t)nchunks;
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
      // the first kPrefetch source indices of the next item are loaded while
      // the current item's copies are issued (no memory round trip per step)
      int pre[kPrefetch];
      prefetch_src(src, nstep, nchunks, total, (int64_t)blockIdx.x, pre);
      for (int64_t it = blockIdx.x; it < total && ok; it += gridDim.x) {
        const int64_t x = it / nchunks;
        const int r0 = (int)(it - x * nchunks) * 128;
        const int w = min(128, s - r0);
        const uint32_t vbytes = (uint32_t)DIN * w * 8u;
#pragma unroll
        for (int j = 0; j < kPrefetch; ++j) s_src[j] = pre[j];
        prefetch_src(src, nstep, nchunks, total, it + gridDim.x, pre);
        for (int j = 0; j < nstep; ++j, ++q) {
          const int ss = (int)(q % NS);
          const int us = (int)(q / NS);
          if (us > 0 && !mbar_wait(smem_u32(&sempty[ss]), (uint32_t)(us - 1) & 1u, &abort_flag)) {
            atomicExch(err, 11);
            abort_flag = 1;
            ok = false;
            break;
          }
          const int64_t nb = j < kPrefetch ? s_src[j] : src[x * nstep + j];
          const uint32_t dst = base + s_off + (uint32_t)ss * stage_bytes;
          const uint32_t bar = smem_u32(&sfull[ss]);
          mbar_expect_tx(bar, vbytes + kCBytes);
          if (nchunks == 1) {
            bulk_g2s(dst, in + nb * DIN * (int64_t)s, vbytes, bar);
          } else {
            for (int e = 0; e < DIN; ++e)
              bulk_g2s(dst + (uint32_t)e * w * 8u, in + (nb * DIN + e) * (int64_t)s + r0, (uint32_t)w * 8u, bar);
          }
          const int64_t bblk = MODE == kStencil ? x * nstep + j : nb;
          bulk_g2s(dst + vbytes, Bsrc + bblk * (int64_t)kBWords, kCBytes, bar);
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
        for (int j = 0; j < nstep; ++j, ++q) {
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
        const int64_t ob = x * DOUT * (int64_t)s + r0 + r;
        float2* o = out + ob;
        if (bres) {  // residual form: out = b - y
#pragma unroll
          for (int d = 0; d < DOUT; ++d) {
            const float2 bv = bres[ob + (int64_t)d * s];
            o[(int64_t)d * s] = make_float2(bv.x - v[d], bv.y - v[DOUT + d]);
          }
        } else {
#pragma unroll
          for (int d = 0; d < DOUT; ++d) o[(int64_t)d * s] = make_float2(v[d], v[DOUT + d]);
        }
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
      for (int j = 0; j < nstep; ++j, ++q) {
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
        const uint32_t* sw = reinterpret_cast<const uint32_t*>(stg + (size_t)DIN * w * 8);
        unsigned char* at = gbase + a_off + (size_t)as * 2 * kATile;
        unsigned char* bt = gbase + b_off + (size_t)as * b_tile;
        // A_hi, A_lo: row r, chunk c = components 2e+p for e = 4c..4c+3;
        // chunks past DIN/4 that the MMAs read are zero
        for (int idx = ct; idx < 128 * KCH; idx += 256) {
          const int rr = idx & 127, c = idx >> 7;
          if (rr < w) {
            uint4 h = make_uint4(0u, 0u, 0u, 0u), l = h;
            if (c < DIN / 4) {
              const float2 v0 = sv[(4 * c + 0) * w + rr], v1 = sv[(4 * c + 1) * w + rr];
              const float2 v2 = sv[(4 * c + 2) * w + rr], v3 = sv[(4 * c + 3) * w + rr];
              split_bf16x2(v0.x, v0.y, h.x, l.x);
              split_bf16x2(v1.x, v1.y, h.y, l.y);
              split_bf16x2(v2.x, v2.y, h.z, l.z);
              split_bf16x2(v3.x, v3.y, h.w, l.w);
            }
            const uint32_t off = sw128_offset(rr, 8 * c);
            *reinterpret_cast<uint4*>(at + off) = h;
            *reinterpret_cast<uint4*>(at + kATile + off) = l;
          }
        }
        build_b_tile<DIN, DOUT, MODE>(ct, 256, sw, bt);
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


// ---------------------------------------------------------------------------
// Stencil from pre-split input tiles.
//
// A coarse field is read by nine output sites, so converting each staged
// block to BF16 inside the stencil converts every value nine times.  Here
// k_split_tiles converts the field once into the operand tiles the MMAs read
// (split BF16, K-major, 32-byte swizzle): for site x and chunk of 128
// right-hand sides, part p (hi, lo) and K step k (complex components
// 8k..8k+7, re/im interleaved) one 4 KB region of 128 rows x 32 B, row r =
// column r of the chunk.  The same number of bytes as the FP32 field.  The
// stencil kernel then bulk-copies a neighbour's tile straight into an operand
// slot; its converter warps only build the B tiles from the coefficients.
// ---------------------------------------------------------------------------
constexpr uint32_t kSplitRegion = 4096;  // 128 rows x 32 B

template <int DIN>
__host__ __device__ constexpr uint32_t split_tile_bytes() {
  return 2u * (uint32_t)((2 * DIN + 15) / 16) * kSplitRegion;
}

template <int DIN>
__global__ void __launch_bounds__(256) k_split_tiles(int64_t nsites, int s, int nchunks, const float2* __restrict__ in,
                                                    unsigned char* __restrict__ tiles) {
  constexpr int KSTEPS = (2 * DIN + 15) / 16;
  const int64_t tot = nsites * nchunks * KSTEPS * 128;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t & 127);
    int64_t u = t >> 7;
    const int k = (int)(u % KSTEPS);
    u /= KSTEPS;
    const int ch = (int)(u % nchunks);
    const int64_t x = u / nchunks;
    const int rr = ch * 128 + r;
    uint32_t hi[8], lo[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int e = 8 * k + i;
      float2 v = make_float2(0.f, 0.f);
      if (e < DIN && rr < s) v = in[(x * DIN + e) * (int64_t)s + rr];
      split_bf16x2(v.x, v.y, hi[i], lo[i]);
    }
    unsigned char* tb = tiles + (size_t)(x * nchunks + ch) * split_tile_bytes<DIN>();
    unsigned char* ph = tb + (size_t)k * kSplitRegion;
    unsigned char* pl = tb + (size_t)(KSTEPS + k) * kSplitRegion;
    *reinterpret_cast<uint4*>(ph + sw32_offset(r, 0)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4*>(ph + sw32_offset(r, 1)) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
    *reinterpret_cast<uint4*>(pl + sw32_offset(r, 0)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    *reinterpret_cast<uint4*>(pl + sw32_offset(r, 1)) = make_uint4(lo[4], lo[5], lo[6], lo[7]);
  }
}

// y(x) = sum_dir C_dir(x) in(nb(x, dir)) from pre-split tiles.  One
// persistent CTA per SM; each operand slot holds one direction's A tile
// (bulk-copied), its compact coefficients (bulk-copied) and its B tile
// (built by the converter warps).  Roles as in k_block_tc; barriers per
// slot: full (copies landed), bready (B tile built), empty (MMAs done).
// NT = 512: converter warps 8-15 (256 threads), one CTA per SM; NT = 256:
// converter warps 2-3 (64 threads), two CTAs per SM (two pipelines).
template <int D, bool REGION_COPIES, int NT = kThreads>
__global__ void __launch_bounds__(NT, 512 / NT)
    k_stencil_tc_split(int64_t nout, int s, int nchunks, int NA, uint32_t slot_bytes, uint32_t b_tile,
                       const int* __restrict__ src, const uint32_t* __restrict__ Bsrc,
                       const unsigned char* __restrict__ tiles, float2* __restrict__ out, int* __restrict__ err,
                       const float2* __restrict__ bres) {
  constexpr int NSTEP = 9;
  constexpr int kConv = NT == 512 ? 256 : 64;      // converter threads
  constexpr int kConvBase = NT == 512 ? 256 : 64;  // their first thread
  constexpr int KSTEPS = (2 * D + 15) / 16;
  constexpr int NCOL = 2 * D;
  constexpr uint32_t kTile = split_tile_bytes<D>();
  constexpr uint32_t kBWords = 2u * D * D;
  constexpr uint32_t kCBytes = kBWords * 4u;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kMaxNA], bready[kMaxNA], empty[kMaxNA];
  __shared__ int s_src[kPrefetch];  // the producer's source indices of the current item
  __shared__ __align__(8) uint64_t accf[2], acce[2], drain;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // slot layout: A tile (kTile), B tile (b_tile), coefficients (kCBytes)
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - smem_u32(smem_raw));
  const uint32_t b_off = kTile, c_off = kTile + b_tile;
  const int64_t total = nout * (int64_t)nchunks;
  if (tid == 0) {
    abort_flag = 0;
    for (int i = 0; i < NA; ++i) {
      mbar_init(smem_u32(&full[i]), 1);
      mbar_init(smem_u32(&bready[i]), kConv);
      mbar_init(smem_u32(&empty[i]), 1);
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
      int last_use[kMaxNA];
      for (int i = 0; i < kMaxNA; ++i) last_use[i] = -1;
      int64_t q = 0;
      bool ok = true;
      // the next item's nine source indices load while this item's copies go out
      int pre[kPrefetch];
      prefetch_src(src, NSTEP, nchunks, total, (int64_t)blockIdx.x, pre);
      for (int64_t it = blockIdx.x; it < total && ok; it += gridDim.x) {
        const int64_t x = it / nchunks;
        const int ch = (int)(it - x * nchunks);
#pragma unroll
        for (int j = 0; j < NSTEP; ++j) s_src[j] = pre[j];
        prefetch_src(src, NSTEP, nchunks, total, it + gridDim.x, pre);
        for (int j = 0; j < NSTEP; ++j, ++q) {
          const int as = (int)(q % NA), ua = (int)(q / NA);
          if (ua > 0 && !mbar_wait(smem_u32(&empty[as]), (uint32_t)(ua - 1) & 1u, &abort_flag)) {
            atomicExch(err, 21);
            abort_flag = 1;
            ok = false;
            break;
          }
          const int64_t nb = s_src[j];
          const uint32_t slot = base + (uint32_t)as * slot_bytes;
          const uint32_t bar = smem_u32(&full[as]);
          mbar_expect_tx(bar, kTile + kCBytes);
          const unsigned char* tsrc = tiles + (size_t)(nb * nchunks + ch) * kTile;
          if (REGION_COPIES) {
            // one copy per 4 KB region (part, K step): more requests in flight
#pragma unroll
            for (int k = 0; k < 2 * KSTEPS; ++k)
              bulk_g2s(slot + (uint32_t)k * kSplitRegion, tsrc + (size_t)k * kSplitRegion, kSplitRegion, bar);
          } else {
            bulk_g2s(slot, tsrc, kTile, bar);
          }
          bulk_g2s(slot + c_off, Bsrc + (x * NSTEP + j) * (int64_t)kBWords, kCBytes, bar);
          last_use[as] = ua;
        }
      }
      // copies still in flight land before the CTA may exit
      for (int i = 0; i < NA; ++i)
        if (last_use[i] >= 0 && !mbar_wait_drain(smem_u32(&full[i]), (uint32_t)last_use[i] & 1u)) atomicExch(err, 22);
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
          atomicExch(err, 23);
          abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)b * kAccStride;
        for (int j = 0; j < NSTEP; ++j, ++q) {
          const int as = (int)(q % NA), ua = (int)(q / NA);
          if (!mbar_wait(smem_u32(&full[as]), (uint32_t)ua & 1u, &abort_flag) ||
              !mbar_wait(smem_u32(&bready[as]), (uint32_t)ua & 1u, &abort_flag)) {
            atomicExch(err, 24);
            abort_flag = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t at = base + (uint32_t)as * slot_bytes;
          const uint32_t bt = at + b_off;
#pragma unroll
          for (int k = 0; k < KSTEPS; ++k) {
            const uint64_t bdesc = sdesc_sw128(bt + (uint32_t)k * 32u);
            mma_bf16(acc, sdesc_sw32(at + (uint32_t)k * kSplitRegion), bdesc, idesc2, (j > 0 || k > 0) ? 1u : 0u);
            mma_bf16(acc, sdesc_sw32(at + (uint32_t)(KSTEPS + k) * kSplitRegion), bdesc, idesc1, 1u);
          }
          mma_commit(smem_u32(&empty[as]));
          issued = true;
        }
        if (ok) mma_commit(smem_u32(&accf[b]));
      }
      if (issued) {
        mma_commit(smem_u32(&drain));
        if (!mbar_wait_drain(smem_u32(&drain), 0)) atomicExch(err, 25);
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
        if (lane == 0) atomicExch(err, 26);
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
        const int64_t ob = x * D * (int64_t)s + r0 + r;
        float2* o = out + ob;
        if (bres) {  // residual form: out = b - y
#pragma unroll
          for (int d = 0; d < D; ++d) {
            const float2 bv = bres[ob + (int64_t)d * s];
            o[(int64_t)d * s] = make_float2(bv.x - v[d], bv.y - v[D + d]);
          }
        } else {
#pragma unroll
          for (int d = 0; d < D; ++d) o[(int64_t)d * s] = make_float2(v[d], v[D + d]);
        }
      }
    }
  } else if (NT == 512 ? warp >= 8 : (warp == 2 || warp == 3)) {
    // ---- converters: compact coefficients -> B tiles ----
    const int ct = tid - kConvBase;
    int64_t q = 0;
    for (int64_t it = blockIdx.x; it < total; it += gridDim.x) {
      bool ok = true;
      for (int j = 0; j < NSTEP; ++j, ++q) {
        const int as = (int)(q % NA), ua = (int)(q / NA);
        if (!mbar_wait(smem_u32(&full[as]), (uint32_t)ua & 1u, &abort_flag)) {
          atomicExch(err, 27);
          abort_flag = 1;
          ok = false;
          break;
        }
        unsigned char* slot = gbase + (size_t)as * slot_bytes;
        build_b_tile<D, D, kStencilSplit>(ct, kConv, reinterpret_cast<const uint32_t*>(slot + c_off), slot + b_off);
        fence_proxy_async_smem();
        mbar_arrive(smem_u32(&bready[as]));
      }
      if (!ok) break;
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

// Split `in` (nsites x D x s, FP32) into `tiles` and apply the stencil from
// them; false (nothing launched) when fewer than two operand slots fit.
template <int D>
bool launch_split(qd_ctx& ctx, int64_t nout, const int* src, const uint32_t* Bsrc, const cplxf* in, unsigned char* tiles,
                  cplxf* out, int s, int* err, int NA_max, bool region_copies, bool two_per_sm = false,
                  const cplxf* b = nullptr) {
  constexpr uint32_t kTile = split_tile_bytes<D>();
  constexpr int KSTEPS = (2 * D + 15) / 16;
  const int nchunks = (s + 127) / 128;
  const uint32_t b_tile = (uint32_t)((4 * D * 128 + 1023) / 1024 * 1024);
  const uint32_t c_bytes = (uint32_t)((2u * D * D * 4u + 1023) / 1024 * 1024);
  const uint32_t slot = kTile + b_tile + c_bytes;
  const size_t budget = two_per_sm ? 110 * 1024 : 220 * 1024;
  int NA = (int)((budget - 1024) / slot);
  if (NA > NA_max) NA = NA_max;
  if (NA > kMaxNA) NA = kMaxNA;
  if (NA < 2) return false;
  const int64_t st = nout * nchunks * KSTEPS * 128;
  const int sgrid = (int)(div_up(st, 256) < 16 * kNumSMs ? div_up(st, 256) : 16 * kNumSMs);
  k_split_tiles<D><<<sgrid, 256, 0, ctx.stream>>>(nout, s, nchunks, reinterpret_cast<const float2*>(in), tiles);
  QD_LAUNCH_CHECK();
  // two CTAs per SM at most (each holds 256 TMEM columns of the 512): the
  // shared-memory request keeps a third CTA off the SM
  size_t smem = 1024 + (size_t)NA * slot;
  if (two_per_sm && smem < 80 * 1024) smem = 80 * 1024;
  const int64_t items = nout * (int64_t)nchunks;
  const int ctas = two_per_sm ? 2 * kNumSMs : kNumSMs;
  const int grid = (int)(items < ctas ? items : ctas);
  auto kern = two_per_sm ? (region_copies ? k_stencil_tc_split<D, true, 256> : k_stencil_tc_split<D, false, 256>)
                         : (region_copies ? k_stencil_tc_split<D, true, 512> : k_stencil_tc_split<D, false, 512>);
  ensure_smem_limit(reinterpret_cast<const void*>(kern), smem);
  kern<<<grid, two_per_sm ? 256 : 512, smem, ctx.stream>>>(nout, s, nchunks, NA, slot, b_tile, src, Bsrc, tiles,
                                                              reinterpret_cast<float2*>(out), err, reinterpret_cast<const float2*>(b));
  QD_LAUNCH_CHECK();
  return true;
}

// Launch k_block_tc with NS staging slots and as many operand stages as fit
// (at most kMaxNA); false (nothing launched) when fewer than two fit.
template <int DIN, int DOUT, int MODE>
bool launch(qd_ctx& ctx, int64_t nout, int nstep, const int* src, const uint32_t* Bsrc, const cplxf* in, cplxf* out,
            int s, int* err, int NS, const cplxf* b = nullptr) {
  constexpr int NV = DOUT / 2;
  constexpr size_t kBBytes = (MODE == kStencil ? 2u * DOUT * DIN : 2u * DIN * NV) * 4u;
  const int nchunks = (s + 127) / 128;
  const int w = s < 128 ? s : 128;
  const uint32_t b_tile = (uint32_t)((4 * DOUT * 128 + 1023) / 1024 * 1024);
  const uint32_t stage = (uint32_t)(((size_t)DIN * w * 8 + kBBytes + 1023) / 1024 * 1024);
  const size_t budget = 220 * 1024;
  if (NS > kMaxNS || 1024 + (size_t)NS * stage + 2 * (2 * kATile + b_tile) > budget) return false;
  int NA = (int)((budget - 1024 - (size_t)NS * stage) / (2 * kATile + b_tile));
  if (NA > kMaxNA) NA = kMaxNA;
  const size_t smem = 1024 + (size_t)NA * (2 * kATile + b_tile) + (size_t)NS * stage;
  ensure_smem_limit(reinterpret_cast<const void*>(k_block_tc<DIN, DOUT, MODE>), smem);
  const int64_t items = nout * (int64_t)nchunks;
  const int grid = (int)(items < kNumSMs ? items : kNumSMs);
  k_block_tc<DIN, DOUT, MODE><<<grid, kThreads, smem, ctx.stream>>>(
      nout, nstep, s, nchunks, NS, NA, stage, b_tile, src, Bsrc, reinterpret_cast<const float2*>(in),
      reinterpret_cast<float2*>(out), err, reinterpret_cast<const float2*>(b));
  QD_LAUNCH_CHECK();
  return true;
}

// Alignment and size rules shared by both uses: 16-byte aligned fields and,
// above 128 right-hand sides (one bulk copy per block row), an even count.
inline bool fields_ok(const void* in, const void* out, int s) {
  if (s < 1) return false;
  if (((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) != 0) return false;
  if (s > 128 && (s & 1)) return false;
  return true;
}

}  // namespace blocktc
}  // namespace qd
