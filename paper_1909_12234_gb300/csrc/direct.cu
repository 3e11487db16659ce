// Direct solves on the coarsest level.
//
// The coarsest operator C (a few thousand dofs on the lattices this library
// targets) is inverted once in FP64 by Gauss-Jordan elimination with partial
// (row) pivoting, in place (Golub & Van Loan, "Matrix Computations", the
// Gauss-Jordan variant of Sec. 3.2; row swaps undone as column swaps at the
// end).  Every coarse solve is then one dense complex product C^{-1} R,
// R = n x s right-hand sides, done by a shared-memory tiled GEMM in FP64 or
// FP32.
#include <algorithm>

#include "blas.cuh"
#include "direct.cuh"

namespace qd {

// ---------------------------------------------------------------------------
// Gauss-Jordan step k, part 1 (one CTA): pivot search in column k over rows
// i >= k, row swap, copy of column k into f, scaling of the pivot row.
// ---------------------------------------------------------------------------
template <class C>
__global__ void __launch_bounds__(1024) k_gj_pivot(int n, int k, C* __restrict__ A, C* __restrict__ f,
                                                   int* __restrict__ perm, int* __restrict__ flag) {
  typedef typename CTraits<C>::R R;
  __shared__ double sv[1024];
  __shared__ int si[1024];
  __shared__ C s_inv;
  const int tid = threadIdx.x, nth = blockDim.x;
  double best = -1.0;
  int bi = k;
  for (int i = k + tid; i < n; i += nth) {
    const double v = (double)cnorm2(A[(int64_t)i * n + k]);
    if (v > best) { best = v; bi = i; }
  }
  sv[tid] = best;
  si[tid] = bi;
  __syncthreads();
  for (int h = nth / 2; h > 0; h >>= 1) {
    if (tid < h) {
      // ties resolved towards the smaller row index (deterministic)
      if (sv[tid + h] > sv[tid] || (sv[tid + h] == sv[tid] && si[tid + h] < si[tid])) {
        sv[tid] = sv[tid + h];
        si[tid] = si[tid + h];
      }
    }
    __syncthreads();
  }
  const int p = si[0];
  if (tid == 0) {
    perm[k] = p;
    if (!(sv[0] > 0.0) && flag) *flag = 1;
  }
  if (p != k) {
    for (int j = tid; j < n; j += nth) {
      const C a = A[(int64_t)k * n + j];
      A[(int64_t)k * n + j] = A[(int64_t)p * n + j];
      A[(int64_t)p * n + j] = a;
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += nth) f[i] = A[(int64_t)i * n + k];
  if (tid == 0) {
    const C piv = A[(int64_t)k * n + k];
    const R d = cnorm2(piv);
    s_inv = d > (R)0 ? mk<C>(piv.x / d, -piv.y / d) : mk<C>((R)0, (R)0);
  }
  __syncthreads();
  const C inv = s_inv;
  for (int j = tid; j < n; j += nth) {
    const C a = (j == k) ? mk<C>((R)1, (R)0) : A[(int64_t)k * n + j];
    A[(int64_t)k * n + j] = cmul(a, inv);
  }
}

// Part 2: for rows i != k: A[i][j] -= f[i] * A[k][j] (A[i][k] taken as 0).
template <class C>
__global__ void k_gj_update(int n, int k, C* __restrict__ A, const C* __restrict__ f) {
  typedef typename CTraits<C>::R R;
  const int64_t tot = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e - (int64_t)i * n);
    if (i == k) continue;
    const C fi = f[i];
    C a = (j == k) ? mk<C>((R)0, (R)0) : A[e];
    cfma(a, mk<C>(-fi.x, -fi.y), A[(int64_t)k * n + j]);
    A[e] = a;
  }
}

// Undo the row interchanges as column interchanges, last step first.
template <class C>
__global__ void k_gj_unswap(int n, C* __restrict__ A, const int* __restrict__ perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  C* row = A + (int64_t)i * n;
  for (int k = n - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k) {
      const C t = row[k];
      row[k] = row[p];
      row[p] = t;
    }
  }
}

template <class C> void gauss_jordan_inverse(qd_ctx& ctx, int n, C* A) {
  DevBuf f((size_t)n * sizeof(C)), perm((size_t)n * sizeof(int)), flag(sizeof(int));
  QD_CUDA(cudaMemsetAsync(flag.as<int>(), 0, sizeof(int), ctx.stream));
  const int64_t tot = (int64_t)n * n;
  int blocks = div_up(tot, 256);
  if (blocks > 16 * kNumSMs) blocks = 16 * kNumSMs;
  for (int k = 0; k < n; ++k) {
    k_gj_pivot<C><<<1, 1024, 0, ctx.stream>>>(n, k, A, f.as<C>(), perm.as<int>(), flag.as<int>());
    QD_LAUNCH_CHECK();
    k_gj_update<C><<<blocks, 256, 0, ctx.stream>>>(n, k, A, f.as<C>());
    QD_LAUNCH_CHECK();
  }
  k_gj_unswap<C><<<div_up(n, 128), 128, 0, ctx.stream>>>(n, A, perm.as<int>());
  QD_LAUNCH_CHECK();
  int h = 0;
  QD_CUDA(cudaMemcpyAsync(&h, flag.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaStreamSynchronize(ctx.stream));
  if (h) fail(QD_ERR_NONFINITE, "coarsest operator is singular (zero pivot in Gauss-Jordan)");
}
template void gauss_jordan_inverse<cplx>(qd_ctx&, int, cplx*);
template void gauss_jordan_inverse<cplxf>(qd_ctx&, int, cplxf*);

// ---------------------------------------------------------------------------
// Blocked Gauss-Jordan (FP32): the same eliminations, grouped into panels of
// w <= 64 columns.  A panel is factored on its own (a contiguous n x w copy,
// column major, so each pivot search reads one contiguous column); the
// panel's row interchanges are then applied to the whole matrix, and its
// accumulated transformation M (identity except in the panel columns, which
// the in-place factorisation leaves holding M's columns) is applied to the
// other columns as one rank-w update A += (M - I)[:, panel] B, with B the
// panel's rows of A and its panel columns zeroed.  The matrix is read and
// written once per panel instead of once per column.
// ---------------------------------------------------------------------------
constexpr int kGJPanel = 64;

__global__ void k_panel_extract(int n, int k0, int w, const cplxf* __restrict__ A, cplxf* __restrict__ P) {
  const int64_t tot = (int64_t)n * w;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / w), c = (int)(e - (int64_t)i * w);
    P[(int64_t)c * n + i] = A[(int64_t)i * n + k0 + c];
  }
}

// Step k of the panel (column c = k - k0): pivot among rows >= k, swap in
// the panel, f = column c, scale the pivot row.  One CTA.
__global__ void __launch_bounds__(1024) k_pgj_pivot(int n, int k, int c, int w, cplxf* __restrict__ P,
                                                    cplxf* __restrict__ f, int* __restrict__ perm,
                                                    int* __restrict__ flag) {
  __shared__ float sv[1024];
  __shared__ int si[1024];
  __shared__ cplxf s_inv;
  const int tid = threadIdx.x, nth = blockDim.x;
  const cplxf* col = P + (int64_t)c * n;
  float best = -1.0f;
  int bi = k;
  for (int i = k + tid; i < n; i += nth) {
    const float v = cnorm2(col[i]);
    if (v > best) { best = v; bi = i; }
  }
  sv[tid] = best;
  si[tid] = bi;
  __syncthreads();
  for (int h = nth / 2; h > 0; h >>= 1) {
    if (tid < h) {
      if (sv[tid + h] > sv[tid] || (sv[tid + h] == sv[tid] && si[tid + h] < si[tid])) {
        sv[tid] = sv[tid + h];
        si[tid] = si[tid + h];
      }
    }
    __syncthreads();
  }
  const int p = si[0];
  if (tid == 0) {
    perm[k] = p;
    if (!(sv[0] > 0.0f) && flag) *flag = 1;
  }
  if (p != k)
    for (int cc = tid; cc < w; cc += nth) {
      const cplxf a = P[(int64_t)cc * n + k];
      P[(int64_t)cc * n + k] = P[(int64_t)cc * n + p];
      P[(int64_t)cc * n + p] = a;
    }
  __syncthreads();
  for (int i = tid; i < n; i += nth) f[i] = col[i];
  if (tid == 0) {
    const cplxf piv = col[k];
    const float d = cnorm2(piv);
    s_inv = d > 0.0f ? make_float2(piv.x / d, -piv.y / d) : make_float2(0.0f, 0.0f);
  }
  __syncthreads();
  const cplxf inv = s_inv;
  for (int cc = tid; cc < w; cc += nth) {
    const cplxf a = (cc == c) ? make_float2(1.0f, 0.0f) : P[(int64_t)cc * n + k];
    P[(int64_t)cc * n + k] = cmul(a, inv);
  }
}

// Rows i != k of the panel: P[i][cc] -= f[i] P[k][cc] (P[i][c] taken as 0).
__global__ void k_pgj_update(int n, int k, int c, int w, cplxf* __restrict__ P, const cplxf* __restrict__ f) {
  const int64_t tot = (int64_t)n * w;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int cc = (int)(e / n), i = (int)(e - (int64_t)cc * n);
    if (i == k) continue;
    const cplxf fi = f[i];
    cplxf a = (cc == c) ? make_float2(0.0f, 0.0f) : P[e];
    cfma(a, make_float2(-fi.x, -fi.y), P[(int64_t)cc * n + k]);
    P[e] = a;
  }
}

// The panel's interchanges, in order, on every column of A (one thread per
// column).
__global__ void k_apply_swaps(int n, int k0, int k1, cplxf* __restrict__ A, const int* __restrict__ perm) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int k = k0; k < k1; ++k) {
    const int p = perm[k];
    if (p != k) {
      const cplxf t = A[(int64_t)k * n + j];
      A[(int64_t)k * n + j] = A[(int64_t)p * n + j];
      A[(int64_t)p * n + j] = t;
    }
  }
}

// A[:, panel] = P; Tm = P - I (on the panel's diagonal); B = rows k0..k1 of
// A with the panel columns zeroed.
__global__ void k_panel_finish(int n, int k0, int w, const cplxf* __restrict__ P, cplxf* __restrict__ A,
                               cplxf* __restrict__ Tm) {
  const int64_t tot = (int64_t)n * w;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / w), c = (int)(e - (int64_t)i * w);
    const cplxf v = P[(int64_t)c * n + i];
    A[(int64_t)i * n + k0 + c] = v;
    Tm[(int64_t)i * w + c] = (i == k0 + c) ? make_float2(v.x - 1.0f, v.y) : v;
  }
}
__global__ void k_panel_rows(int n, int k0, int w, const cplxf* __restrict__ A, cplxf* __restrict__ B) {
  const int64_t tot = (int64_t)w * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / n), j = (int)(e - (int64_t)r * n);
    B[e] = (j >= k0 && j < k0 + w) ? make_float2(0.0f, 0.0f) : A[(int64_t)(k0 + r) * n + j];
  }
}

// C (m x n, ldc) += A (m x K, lda) B (K x n, ldb), FP32 complex, K <= 64:
// 64 x 64 output tile per CTA (256 threads, 4 x 4 each), operands staged in
// shared memory in K-slices of 16.
__global__ void __launch_bounds__(256) k_cgemm_acc(int m, int n, int K, const cplxf* __restrict__ A, int lda,
                                                   const cplxf* __restrict__ B, int ldb, cplxf* __restrict__ C,
                                                   int ldc) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ cplxf sa[BK][BM + 1];
  __shared__ cplxf sb[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tr = tid / 16, tc = tid % 16;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  cplxf acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.0f, 0.0f);
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += 256) {
      const int mm = e / BK, kk = e % BK;
      const int gr = row0 + mm, gk = k0 + kk;
      sa[kk][mm] = (gr < m && gk < K) ? A[(int64_t)gr * lda + gk] : make_float2(0.0f, 0.0f);
    }
    for (int e = tid; e < BK * BN; e += 256) {
      const int kk = e / BN, cc = e % BN;
      const int gk = k0 + kk, gc = col0 + cc;
      sb[kk][cc] = (gk < K && gc < n) ? B[(int64_t)gk * ldb + gc] : make_float2(0.0f, 0.0f);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      cplxf a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sa[kk][tr + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sb[kk][tc + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gr = row0 + tr + 16 * i;
    if (gr >= m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gc = col0 + tc + 16 * j;
      if (gc < n) C[(int64_t)gr * ldc + gc] = cadd(C[(int64_t)gr * ldc + gc], acc[i][j]);
    }
  }
}

void gauss_jordan_inverse_blocked(qd_ctx& ctx, int n, cplxf* A) {
  const int W = kGJPanel;
  DevBuf P((size_t)n * W * sizeof(cplxf)), Tm((size_t)n * W * sizeof(cplxf)), B((size_t)W * n * sizeof(cplxf)),
      f((size_t)n * sizeof(cplxf)), perm((size_t)n * sizeof(int)), flag(sizeof(int));
  QD_CUDA(cudaMemsetAsync(flag.as<int>(), 0, sizeof(int), ctx.stream));
  auto grid = [](int64_t tot) { return (int)std::min<int64_t>(div_up(tot, 256), 16 * kNumSMs); };
  for (int k0 = 0; k0 < n; k0 += W) {
    const int w = std::min(W, n - k0);
    k_panel_extract<<<grid((int64_t)n * w), 256, 0, ctx.stream>>>(n, k0, w, A, P.as<cplxf>());
    QD_LAUNCH_CHECK();
    for (int c = 0; c < w; ++c) {
      const int k = k0 + c;
      k_pgj_pivot<<<1, 1024, 0, ctx.stream>>>(n, k, c, w, P.as<cplxf>(), f.as<cplxf>(), perm.as<int>(),
                                              flag.as<int>());
      QD_LAUNCH_CHECK();
      k_pgj_update<<<grid((int64_t)n * w), 256, 0, ctx.stream>>>(n, k, c, w, P.as<cplxf>(), f.as<cplxf>());
      QD_LAUNCH_CHECK();
    }
    k_apply_swaps<<<div_up(n, 256), 256, 0, ctx.stream>>>(n, k0, k0 + w, A, perm.as<int>());
    QD_LAUNCH_CHECK();
    k_panel_finish<<<grid((int64_t)n * w), 256, 0, ctx.stream>>>(n, k0, w, P.as<cplxf>(), A, Tm.as<cplxf>());
    QD_LAUNCH_CHECK();
    k_panel_rows<<<grid((int64_t)w * n), 256, 0, ctx.stream>>>(n, k0, w, A, B.as<cplxf>());
    QD_LAUNCH_CHECK();
    dim3 g2(div_up(n, 64), div_up(n, 64));
    k_cgemm_acc<<<g2, 256, 0, ctx.stream>>>(n, n, w, Tm.as<cplxf>(), w, B.as<cplxf>(), n, A, n);
    QD_LAUNCH_CHECK();
  }
  k_gj_unswap<cplxf><<<div_up(n, 128), 128, 0, ctx.stream>>>(n, A, perm.as<int>());
  QD_LAUNCH_CHECK();
  int h = 0;
  QD_CUDA(cudaMemcpyAsync(&h, flag.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaStreamSynchronize(ctx.stream));
  if (h) fail(QD_ERR_NONFINITE, "coarsest operator is singular (zero pivot in Gauss-Jordan)");
}

// ---------------------------------------------------------------------------
// Dense stencil -> matrix: D[(x*Dd + d)][(y*Dd + e)] += C[x][dir][d][e] for
// y = nb(x, dir) (aliased neighbours on small lattices are summed; the sum
// is formed in FP64 and rounded once to the output type).
// ---------------------------------------------------------------------------
template <class C>
__global__ void k_stencil_to_dense(int64_t nsites, int D, const int* __restrict__ nbr, const cplx* __restrict__ mat,
                                   C* __restrict__ dense) {
  typedef typename CTraits<C>::R R;
  const int64_t n = nsites * D;
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n;
       row += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = row / D;
    const int d = (int)(row - x * D);
    C* drow = dense + row * n;
    for (int dir = 0; dir < 9; ++dir) {
      const int64_t y = (dir == 0) ? x : (int64_t)nbr[x * 8 + dir - 1];
      for (int e = 0; e < D; ++e) {
        // sum every block that lands on (row, y*D + e), in direction order
        cplx acc = mkc(0.0, 0.0);
        bool first = true;
        for (int d2 = 0; d2 < dir && first; ++d2) {
          const int64_t y2 = (d2 == 0) ? x : (int64_t)nbr[x * 8 + d2 - 1];
          if (y2 == y) first = false;  // an earlier direction already wrote this column block
        }
        if (!first) continue;
        for (int d2 = dir; d2 < 9; ++d2) {
          const int64_t y2 = (d2 == 0) ? x : (int64_t)nbr[x * 8 + d2 - 1];
          if (y2 == y) acc = cadd(acc, mat[((x * 9 + d2) * D + d) * D + e]);
        }
        drow[y * D + e] = mk<C>((R)acc.x, (R)acc.y);
      }
    }
  }
}

// The dense inverse of the coarsest operator, computed by Gauss-Jordan in
// FP32 (FP64 runs at 1/60 of the FP32 rate on this part) and kept in both
// precisions; solves that need FP64 accuracy add residual corrections
// (coarsest_solve_refined).
void coarse_dense_inverse(qd_ctx& ctx, CoarseLevel& lv) {
  const int64_t n64 = lv.geo.nsites * (int64_t)lv.D;
  QD_REQUIRE(n64 <= 16384, "coarsest level too large for a dense direct solve");
  const int n = (int)n64;
  lv.Cinvf.resize((size_t)n * n * sizeof(cplxf));
  QD_CUDA(cudaMemsetAsync(lv.Cinvf.as<cplxf>(), 0, (size_t)n * n * sizeof(cplxf), ctx.stream));
  k_stencil_to_dense<cplxf><<<div_up(n, 128), 128, 0, ctx.stream>>>(lv.geo.nsites, lv.D, lv.geo.nbr.as<int>(),
                                                                   lv.Cm.as<cplx>(), lv.Cinvf.as<cplxf>());
  QD_LAUNCH_CHECK();
  if (n >= 4 * kGJPanel)
    gauss_jordan_inverse_blocked(ctx, n, lv.Cinvf.as<cplxf>());
  else
    gauss_jordan_inverse<cplxf>(ctx, n, lv.Cinvf.as<cplxf>());
  lv.Cinv.resize((size_t)n * n * sizeof(cplx));
  to_f64(ctx, lv.Cinvf.as<cplxf>(), lv.Cinv.as<cplx>(), (int64_t)n * n);
  lv.ndense = n;
}

// y = C^{-1} x to FP64 accuracy: y = X x with the FP32 inverse X, then
// `steps` corrections y += X (x - C y), the residual formed with the FP64
// stencil C and rounded to FP32 for the product (each correction gains the
// digits of ||I - C X||, about four here, at FP32 speed).
void coarsest_solve_refined(qd_ctx& ctx, const CoarseLevel& lv, int nrhs, const cplx* x, cplx* y, int steps) {
  const int n = lv.ndense;
  QD_REQUIRE(n > 0 && lv.Cinvf.bytes() > 0, "no dense inverse on this level");
  const int64_t tot = (int64_t)n * nrhs;
  // scratch kept on the level (grow-only) so repeated solves allocate nothing
  DevBuf& rf = lv.rs_f[0];
  DevBuf& ef = lv.rs_f[1];
  DevBuf& r = lv.rs_d[0];
  DevBuf& e = lv.rs_d[1];
  rf.resize((size_t)tot * sizeof(cplxf));
  ef.resize((size_t)tot * sizeof(cplxf));
  to_f32(ctx, x, rf.as<cplxf>(), tot);
  dense_apply<cplxf>(ctx, n, nrhs, lv.Cinvf.as<cplxf>(), rf.as<cplxf>(), ef.as<cplxf>());
  to_f64(ctx, ef.as<cplxf>(), y, tot);
  if (steps <= 0) return;
  r.resize((size_t)tot * sizeof(cplx));
  e.resize((size_t)tot * sizeof(cplx));
  for (int it = 0; it < steps; ++it) {
    coarse_apply<cplx>(ctx, lv, lv.Cm.as<cplx>(), y, r.as<cplx>(), nrhs);
    blas::sub(ctx, tot, x, r.as<cplx>(), r.as<cplx>());
    to_f32(ctx, r.as<cplx>(), rf.as<cplxf>(), tot);
    dense_apply<cplxf>(ctx, n, nrhs, lv.Cinvf.as<cplxf>(), rf.as<cplxf>(), ef.as<cplxf>());
    to_f64(ctx, ef.as<cplxf>(), e.as<cplx>(), tot);
    blas::add(ctx, tot, e.as<cplx>(), y);
  }
}

// ---------------------------------------------------------------------------
// Tiled complex GEMM, Y (n x s) = M (n x n) X (n x s), all row major, FP64
// or FP32.  64 x 64 output tile per CTA (256 threads, 4 x 4 per thread),
// k-tiles of 16 staged in shared memory.
// ---------------------------------------------------------------------------
template <class C, int BM = 64, int BN = 64>
__global__ void __launch_bounds__(256) k_zgemm(int n, int s, const C* __restrict__ M, const C* __restrict__ X,
                                               C* __restrict__ Y) {
  typedef typename CTraits<C>::R R;
  constexpr int BK = 16, TM = BM / 16, TN = BN / 16;  // 16 x 16 threads, TM x TN outputs each
  __shared__ C sa[BK][BM + 1];
  __shared__ C sb[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tr = tid / 16, tc = tid % 16;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  C acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = mk<C>((R)0, (R)0);
  for (int k0 = 0; k0 < n; k0 += BK) {
    // load M[row0 .. +64][k0 .. +16] -> sa[k][m] and X[k0 .. +16][col0 .. +64] -> sb[k][c]
    for (int e = tid; e < BM * BK; e += 256) {
      const int m = e / BK, kk = e % BK;
      const int gr = row0 + m, gk = k0 + kk;
      sa[kk][m] = (gr < n && gk < n) ? M[(int64_t)gr * n + gk] : mk<C>((R)0, (R)0);
    }
    for (int e = tid; e < BK * BN; e += 256) {
      const int kk = e / BN, c = e % BN;
      const int gk = k0 + kk, gc = col0 + c;
      sb[kk][c] = (gk < n && gc < s) ? X[(int64_t)gk * s + gc] : mk<C>((R)0, (R)0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      C a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = sa[kk][tr + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = sb[kk][tc + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) cfma(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gr = row0 + tr + 16 * i;
    if (gr >= n) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gc = col0 + tc + 16 * j;
      if (gc < s) Y[(int64_t)gr * s + gc] = acc[i][j];
    }
  }
}

// Few right-hand sides (s <= S <= 16): one warp per row of M, which is read
// once and contiguously; lanes take every 32nd column, then a fixed shuffle
// tree adds the lanes (deterministic).  The 64 x 64 tile above would leave
// most of each tile idle here.
template <class C, int S>
__global__ void __launch_bounds__(256) k_dense_small(int n, int s, const C* __restrict__ M, const C* __restrict__ X,
                                                     C* __restrict__ Y) {
  typedef typename CTraits<C>::R R;
  const int row = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  C acc[S];
#pragma unroll
  for (int c = 0; c < S; ++c) acc[c] = mk<C>((R)0, (R)0);
  const C* mrow = M + (int64_t)row * n;
  for (int k = lane; k < n; k += 32) {
    const C m = mrow[k];
    const C* xk = X + (int64_t)k * s;
#pragma unroll
    for (int c = 0; c < S; ++c)
      if (c < s) cfma(acc[c], m, xk[c]);
  }
#pragma unroll
  for (int c = 0; c < S; ++c) {
    R re = acc[c].x, im = acc[c].y;
    for (int off = 16; off > 0; off >>= 1) {
      re += __shfl_down_sync(0xffffffffu, re, off);
      im += __shfl_down_sync(0xffffffffu, im, off);
    }
    if (lane == 0 && c < s) Y[(int64_t)row * s + c] = mk<C>(re, im);
  }
}

template <class C> void dense_apply(qd_ctx& ctx, int n, int s, const C* M, const C* X, C* Y) {
  const double cb = (double)sizeof(C);
  ProfScope ps(ctx, sizeof(C) == 16 ? QD_PROF_DIRECT_F64 : QD_PROF_DIRECT_F32, 8.0 * n * (double)n * s,
               cb * ((double)n * n + 2.0 * n * s));
  if (s <= 16) {
    const int blocks = div_up((int64_t)n * 32, 256);
    if (s <= 4)
      k_dense_small<C, 4><<<blocks, 256, 0, ctx.stream>>>(n, s, M, X, Y);
    else if (s <= 8)
      k_dense_small<C, 8><<<blocks, 256, 0, ctx.stream>>>(n, s, M, X, Y);
    else
      k_dense_small<C, 16><<<blocks, 256, 0, ctx.stream>>>(n, s, M, X, Y);
    QD_LAUNCH_CHECK();
    return;
  }
  if (s <= 48) {
    // narrow blocks of right-hand sides (the eigensolver's 40): 32 x 48
    // tiles waste less of each tile and give twice the blocks
    dim3 grid(div_up(s, 48), div_up(n, 32));
    k_zgemm<C, 32, 48><<<grid, 256, 0, ctx.stream>>>(n, s, M, X, Y);
    QD_LAUNCH_CHECK();
    return;
  }
  dim3 grid(div_up(s, 64), div_up(n, 64));
  k_zgemm<C><<<grid, 256, 0, ctx.stream>>>(n, s, M, X, Y);
  QD_LAUNCH_CHECK();
}
template void dense_apply<cplx>(qd_ctx&, int, int, const cplx*, const cplx*, cplx*);
template void dense_apply<cplxf>(qd_ctx&, int, int, const cplxf*, const cplxf*, cplxf*);

}  // namespace qd
