// Coarsest-level solve on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The mixed-precision V-cycle applies the dense inverse of the coarsest
// operator to s right-hand sides: Y = C^{-1} X (complex, n x n times n x s).
// Written as one real GEMM with K = 2n:
//   A' = [Re C^{-1} | Im C^{-1}]            (n x 2n, BF16, built once)
//   B' = [[Re X, Im X], [-Im X, Re X]]       (2n x 2s, BF16, per call)
//   A' B' = [Re Y | Im Y]                    (n x 2s, FP32 accumulate)
// A BF16 coarse solve costs the outer solver no extra iterations on the
// estimator workload (its preconditioner tolerates ~1e-3 relative error).
//
// Kernel: one CTA per (128-row tile, K split); TMA loads of 128B-swizzled
// K-major tiles (A 128 x 64, B N x 64) into a shared-memory ring of up to 6 stages
// guarded by mbarriers; one thread issues tcgen05.mma (M = 128, K = 16 per
// instruction) into a TMEM accumulator of N FP32 columns; tcgen05.commit
// frees ring stages and signals the epilogue; four warps read TMEM
// (tcgen05.ld 32x32b) and write FP32 partial sums, which a second kernel
// adds over the K splits in order and interleaves into complex Y.
// Every mbarrier wait is bounded (2 s of %globaltimer); on timeout the
// kernel records an error, stops issuing work and frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "ptx.cuh"
#include "tc_gemm.cuh"

namespace qd {

namespace {

constexpr int kBM = 128;     // rows per CTA (UMMA M)
constexpr int kBK = 64;      // K per stage: 64 BF16 = 128 B = one swizzle row
constexpr int kMaxStages = 6;  // ring depth: as many as fit in 227 KB, at most 6
constexpr int kThreads = 128;
using namespace ptx;

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int N,
              int ktiles_per_split, int ktiles_total, int Mp, int kStages, float* __restrict__ part,
              int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kMaxStages], empty_bar[kMaxStages], done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m_tile = blockIdx.x, split = blockIdx.y;
  const int kt0 = split * ktiles_per_split;
  int nkt = ktiles_total - kt0;
  if (nkt > ktiles_per_split) nkt = ktiles_per_split;
  // 1024-byte aligned ring
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t a_bytes = kBM * kBK * 2, b_bytes = (uint32_t)N * kBK * 2;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  const uint32_t ncols = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    mbar_init(smem_u32(&done_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    // producer: TMA loads into the ring
    for (int i = 0; i < nkt; ++i) {
      const int s = i % kStages;
      const uint32_t use = (uint32_t)(i / kStages);
      if (use > 0 && !mbar_wait(smem_u32(&empty_bar[s]), (use - 1) & 1u, &abort_flag)) {
        atomicExch(err, 1);
        abort_flag = 1;
        break;
      }
      const uint32_t fb = smem_u32(&full_bar[s]);
      const uint32_t sa = base + (uint32_t)s * stage_bytes;
      mbar_expect_tx(fb, stage_bytes);
      const int kx = (kt0 + i) * kBK;
      tma_load_2d(sa, &mapA, kx, m_tile * kBM, fb);
      tma_load_2d(sa + a_bytes, &mapB, kx, 0, fb);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = idesc_bf16(kBM, N);
    for (int i = 0; i < nkt; ++i) {
      const int s = i % kStages;
      if (!mbar_wait(smem_u32(&full_bar[s]), (uint32_t)(i / kStages) & 1u, &abort_flag)) {
        atomicExch(err, 2);
        abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = base + (uint32_t)s * stage_bytes;
#pragma unroll
      for (int k = 0; k < kBK / 16; ++k) {
        const uint64_t ad = sdesc_sw128(sa + (uint32_t)k * 32u);
        const uint64_t bd = sdesc_sw128(sa + a_bytes + (uint32_t)k * 32u);
        const uint32_t acc = (i > 0 || k > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&empty_bar[s]))
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&done_bar))
                 : "memory");
  }
  __syncwarp();
  // epilogue: wait for the accumulator, TMEM -> registers -> partial sums
  const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&done_bar), 0, &abort_flag) ? 1 : 0) != 0;
  if (!ok && lane == 0) atomicExch(err, 3);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok && nkt > 0) {
    const int row = m_tile * kBM + warp * 32 + lane;
    float* dst = part + ((int64_t)split * Mp + row) * N;
    for (int c0 = 0; c0 < N; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) dst[c0 + j] = __uint_as_float(v[j]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// A' (Mp x Kp BF16) from C^{-1} (n x n complex FP64): row i = [Re row | Im row], zero padded.
__global__ void k_build_a(int n, int Mp, int Kp, const cplx* __restrict__ Cinv, __nv_bfloat16* __restrict__ A) {
  const int64_t tot = (int64_t)Mp * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / Kp), k = (int)(e - (int64_t)i * Kp);
    float v = 0.f;
    if (i < n) {
      if (k < n)
        v = (float)Cinv[(int64_t)i * n + k].x;
      else if (k < 2 * n)
        v = (float)Cinv[(int64_t)i * n + (k - n)].y;
    }
    A[e] = __float2bfloat16_rn(v);
  }
}

// B'^T (Np x Kp BF16) from X (n x s complex FP32, RHS innermost):
// column j < s: [Re X_j ; -Im X_j], s <= j < 2s: [Im X_{j-s} ; Re X_{j-s}].
__global__ void k_build_b(int n, int s, int Np, int Kp, const cplxf* __restrict__ X, __nv_bfloat16* __restrict__ B) {
  const int64_t tot = (int64_t)Np * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / Kp), k = (int)(e - (int64_t)j * Kp);
    float v = 0.f;
    if (j < 2 * s && k < 2 * n) {
      const int r = j < s ? j : j - s;
      const int kk = k < n ? k : k - n;
      const cplxf x = X[(int64_t)kk * s + r];
      if (j < s)
        v = k < n ? x.x : -x.y;
      else
        v = k < n ? x.y : x.x;
    }
    B[e] = __float2bfloat16_rn(v);
  }
}

// Y[i][r] = (sum_split P[split][i][r], sum_split P[split][i][s + r])
__global__ void k_reduce_splits(int n, int s, int N, int Mp, int nsplit, const float* __restrict__ part,
                                cplxf* __restrict__ Y) {
  const int64_t tot = (int64_t)n * s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / s), r = (int)(e - (int64_t)i * s);
    float re = 0.f, im = 0.f;
    for (int sp = 0; sp < nsplit; ++sp) {
      const float* p = part + ((int64_t)sp * Mp + i) * N;
      re += p[r];
      im += p[s + r];
    }
    Y[e] = make_float2(re, im);
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  if (!fn) fail(QD_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  return fn;
}

// 2-D BF16 tensor map over a row-major (rows x cols) array, box (box_rows x 64).
void make_map(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols, int box_rows) {
  QD_REQUIRE(((uintptr_t)ptr & 15) == 0, "TMA base address must be 16-byte aligned");
  QD_REQUIRE((cols * 2) % 16 == 0, "TMA row pitch must be a multiple of 16 bytes");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(cols * 2)};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides,
                                 box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(QD_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
}

}  // namespace

void tc_prepare(qd_ctx& ctx, CoarseLevel& lv) {
  QD_REQUIRE(lv.ndense > 0, "coarsest level has no dense inverse");
  const int n = lv.ndense;
  lv.tc_Mp = (n + kBM - 1) / kBM * kBM;
  lv.tc_Kp = (2 * n + kBK - 1) / kBK * kBK;
  lv.tc_A.resize((size_t)lv.tc_Mp * lv.tc_Kp * 2);
  const int64_t tot = (int64_t)lv.tc_Mp * lv.tc_Kp;
  k_build_a<<<blas_grid(tot), 256, 0, ctx.stream>>>(n, lv.tc_Mp, lv.tc_Kp, lv.Cinv.as<cplx>(),
                                                    lv.tc_A.as<__nv_bfloat16>());
  QD_LAUNCH_CHECK();
  make_map(reinterpret_cast<CUtensorMap*>(lv.tc_mapA), lv.tc_A.as<void>(), lv.tc_Mp, lv.tc_Kp, kBM);
}

// Y = C^{-1} X for s columns (any s >= 1): chunks of <= 128 right-hand sides.
void tc_dense_apply(qd_ctx& ctx, CoarseLevel& lv, const cplxf* X, cplxf* Y, int s) {
  const int n = lv.ndense;
  const int Mp = lv.tc_Mp, Kp = lv.tc_Kp;
  const int ktiles = Kp / kBK;
  const int mtiles = Mp / kBM;
  int nsplit = kNumSMs / mtiles;  // at most one CTA per SM in one wave
  if (nsplit > ktiles) nsplit = ktiles;
  if (nsplit < 1) nsplit = 1;
  const int kps = (ktiles + nsplit - 1) / nsplit;
  nsplit = (ktiles + kps - 1) / kps;
  for (int c0 = 0; c0 < s; c0 += 128) {
    const int sc = (s - c0) < 128 ? (s - c0) : 128;
    const int N = (2 * sc + 15) / 16 * 16;
    // per-chunk views: X and Y rows have stride s, so gather the chunk
    const cplxf* Xc = X;
    cplxf* Yc = Y;
    if (sc != s) {
      lv.tc_xc.resize((size_t)n * sc * sizeof(cplxf));
      lv.tc_yc.resize((size_t)n * sc * sizeof(cplxf));
      QD_CUDA(cudaMemcpy2DAsync(lv.tc_xc.as<cplxf>(), sc * sizeof(cplxf), X + c0, s * sizeof(cplxf),
                                sc * sizeof(cplxf), n, cudaMemcpyDeviceToDevice, ctx.stream));
      Xc = lv.tc_xc.as<cplxf>();
      Yc = lv.tc_yc.as<cplxf>();
    }
    const size_t bbytes = (size_t)N * Kp * 2;
    if (lv.tc_B.bytes() < bbytes || lv.tc_mapB_N != N) {
      lv.tc_B.resize(bbytes);
      make_map(reinterpret_cast<CUtensorMap*>(lv.tc_mapB), lv.tc_B.as<void>(), N, Kp, N);
      lv.tc_mapB_N = N;
    }
    lv.tc_part.resize((size_t)nsplit * Mp * N * sizeof(float));
    if (lv.tc_err.bytes() == 0) {
      lv.tc_err.resize(sizeof(int));
      QD_CUDA(cudaMemsetAsync(lv.tc_err.as<int>(), 0, sizeof(int), ctx.stream));
    }
    const double flops = 8.0 * n * (double)n * sc;
    const double bytes = 2.0 * (double)Mp * Kp + 2.0 * bbytes + 8.0 * n * sc;
    k_build_b<<<blas_grid((int64_t)N * Kp), 256, 0, ctx.stream>>>(n, sc, N, Kp, Xc, lv.tc_B.as<__nv_bfloat16>());
    QD_LAUNCH_CHECK();
    {
      ProfScope ps(ctx, QD_PROF_DIRECT_BF16, flops, bytes);
      const size_t stage = (size_t)kBM * kBK * 2 + (size_t)N * kBK * 2;
      int stages = (int)((220u * 1024u - 1024u) / stage);
      if (stages > kMaxStages) stages = kMaxStages;
      QD_REQUIRE(stages >= 2, "tensor-core tile does not fit in shared memory");
      const size_t smem = 1024 + (size_t)stages * stage;
      ensure_smem_limit(reinterpret_cast<const void*>(k_tc_gemm), smem);
      k_tc_gemm<<<dim3(mtiles, nsplit), kThreads, smem, ctx.stream>>>(
          *reinterpret_cast<const CUtensorMap*>(lv.tc_mapA), *reinterpret_cast<const CUtensorMap*>(lv.tc_mapB), N,
          kps, ktiles, Mp, stages, lv.tc_part.as<float>(), lv.tc_err.as<int>());
      QD_LAUNCH_CHECK();
    }
    k_reduce_splits<<<blas_grid((int64_t)n * sc), 256, 0, ctx.stream>>>(n, sc, N, Mp, nsplit,
                                                                      lv.tc_part.as<float>(), Yc);
    QD_LAUNCH_CHECK();
    if (sc != s)
      QD_CUDA(cudaMemcpy2DAsync(Y + c0, s * sizeof(cplxf), Yc, sc * sizeof(cplxf), sc * sizeof(cplxf), n,
                                cudaMemcpyDeviceToDevice, ctx.stream));
  }
}

int tc_error(qd_ctx& ctx, CoarseLevel& lv) {
  if (lv.tc_err.bytes() == 0) return 0;
  int h = 0;
  QD_CUDA(cudaMemcpyAsync(&h, lv.tc_err.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaStreamSynchronize(ctx.stream));
  return h;
}

}  // namespace qd
