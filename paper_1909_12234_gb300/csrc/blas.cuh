// Batched level-1 kernels on multi-RHS fields (RHS innermost).  Every
// right-hand side is an independent vector: reductions return one value per
// column.  Reductions are deterministic: a fixed grid writes per-block
// partial sums (fixed tree order inside a block) and a second kernel adds the
// partials in block order.
#pragma once

#include "qd_internal.cuh"

namespace qd {
namespace blas {

constexpr int kThreads = 256;
constexpr int kDotK = 8;  // dot products per reduction launch

// Thread tile for an (n rows) x (nrhs columns) sweep: RT lanes along the
// columns (coalesced), RY = 256 / RT rows per block.
struct Sweep {
  int RT, RY;
  dim3 block, grid;
};

inline Sweep sweep(int64_t n, int nrhs, int max_row_blocks = 4 * kNumSMs) {
  Sweep s;
  int rt = 1;
  while (rt < nrhs && rt < 32) rt <<= 1;
  s.RT = rt;
  s.RY = kThreads / rt;
  int gy = div_up(nrhs, rt);
  int64_t want = (n + s.RY - 1) / s.RY;
  int cap = max_row_blocks / gy;
  if (cap < 1) cap = 1;
  int gx = (int)(want < cap ? want : cap);
  if (gx < 1) gx = 1;
  s.block = dim3(s.RT, s.RY);
  s.grid = dim3(gx, gy);
  return s;
}

// Up to kDotK (X_k, Y_k) vector pairs for one reduction launch.
template <class C> struct DotPairs {
  const C* x[kDotK];
  const C* y[kDotK];
};

// partials[(blk*K + k)*nrhs + r] = sum over this block's rows of conj(X_k) Y_k
// KK: the pair count as a compile-time bound (1, 2 or kDotK).  The loop over
// pairs is unrolled to KK, so a launch with one pair carries no predicated-off
// multiply-adds: for FP64, whose pipe is narrow on this GPU, those cost as
// much issue time as live ones.
template <class C, int KK = kDotK>
__global__ void k_dots(int K, int64_t n, int nrhs, DotPairs<C> pr, cplx* __restrict__ partials) {
  typedef typename CTraits<C>::R R;
  __shared__ cplx sm[KK][kThreads];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int r = blockIdx.y * blockDim.x + tx;
  C acc[KK];
#pragma unroll
  for (int k = 0; k < KK; ++k) acc[k] = mk<C>((R)0, (R)0);
  if (r < nrhs) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.y + ty; i < n; i += (int64_t)gridDim.x * blockDim.y) {
      const int64_t e = i * nrhs + r;
#pragma unroll
      for (int k = 0; k < KK; ++k)
        if (KK == 1 || k < K) cfmac(acc[k], pr.x[k][e], pr.y[k][e]);
    }
  }
  const int t = ty * blockDim.x + tx;
#pragma unroll
  for (int k = 0; k < KK; ++k) sm[k][t] = mkc((double)acc[k].x, (double)acc[k].y);
  __syncthreads();
  for (int h = blockDim.y / 2; h > 0; h >>= 1) {
    if (ty < h) {
#pragma unroll
      for (int k = 0; k < KK; ++k)
        if (k < K) sm[k][t] = cadd(sm[k][t], sm[k][t + h * blockDim.x]);
    }
    __syncthreads();
  }
  if (ty == 0 && r < nrhs) {
    for (int k = 0; k < K; ++k) partials[((int64_t)blockIdx.x * K + k) * nrhs + r] = sm[k][tx];
  }
}

// out[k*nrhs + r] = sum_b partials[b][k][r]: one warp per output; lane l
// adds blocks l, l + 32, ... in order, then a fixed shuffle tree (the
// result does not depend on scheduling).
static __global__ void k_dots_final(int K, int nrhs, int nblk, const cplx* __restrict__ partials,
                                    cplx* __restrict__ out) {
  const int idx = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (idx >= K * nrhs) return;
  const int k = idx / nrhs, r = idx - k * nrhs;
  cplx s = mkc(0.0, 0.0);
  for (int b = lane; b < nblk; b += 32) s = cadd(s, partials[((int64_t)b * K + k) * nrhs + r]);
  for (int off = 16; off > 0; off >>= 1) {
    s.x += __shfl_down_sync(0xffffffffu, s.x, off);
    s.y += __shfl_down_sync(0xffffffffu, s.y, off);
  }
  if (lane == 0) out[idx] = s;
}

// One reduction launch (+ final pass) for K <= kDotK pairs: out[k][r].
template <class C>
void dots_launch(qd_ctx& ctx, int K, int64_t n, int nrhs, const DotPairs<C>& pr, cplx* out) {
  Sweep s = sweep(n, nrhs);
  ctx.red_partials.resize((size_t)s.grid.x * K * nrhs * sizeof(cplx));
  {
    ProfScope ps(ctx, sizeof(C) == 16 ? QD_PROF_BLAS_F64 : QD_PROF_DOTS_F32, 8.0 * K * n * nrhs,
                 (double)sizeof(C) * 2.0 * K * n * nrhs);
    if (K == 1)
      k_dots<C, 1><<<s.grid, s.block, 0, ctx.stream>>>(K, n, nrhs, pr, ctx.red_partials.as<cplx>());
    else if (K == 2)
      k_dots<C, 2><<<s.grid, s.block, 0, ctx.stream>>>(K, n, nrhs, pr, ctx.red_partials.as<cplx>());
    else
      k_dots<C><<<s.grid, s.block, 0, ctx.stream>>>(K, n, nrhs, pr, ctx.red_partials.as<cplx>());
    QD_LAUNCH_CHECK();
  }
  const int tot = K * nrhs;  // one warp each, 8 warps per block
  k_dots_final<<<div_up(tot, 8), 256, 0, ctx.stream>>>(K, nrhs, s.grid.x, ctx.red_partials.as<cplx>(), out);
  QD_LAUNCH_CHECK();
}

// out[k][r] = <X_k, Y_k>_r for k < K (any K), X_k = X + k*xs, Y_k = Y + k*ys
// (strides in complex elements; ys may be 0).  out: device cplx [K][nrhs].
template <class C>
void dots(qd_ctx& ctx, int K, int64_t n, int nrhs, const C* X, int64_t xs, const C* Y, int64_t ys,
          cplx* out) {
  if (K <= 0) return;
  for (int k0 = 0; k0 < K; k0 += kDotK) {
    const int kk = (K - k0) < kDotK ? (K - k0) : kDotK;
    DotPairs<C> pr;
    for (int k = 0; k < kDotK; ++k) {
      const int kc = k < kk ? k : 0;
      pr.x[k] = X + (k0 + kc) * xs;
      pr.y[k] = Y + (k0 + kc) * ys;
    }
    dots_launch<C>(ctx, kk, n, nrhs, pr, out + (int64_t)k0 * nrhs);
  }
}

// out[0][r] = <x0, y0>_r, out[1][r] = <x1, y1>_r in one launch.
template <class C>
void dots2(qd_ctx& ctx, int64_t n, int nrhs, const C* x0, const C* y0, const C* x1, const C* y1, cplx* out) {
  DotPairs<C> pr;
  for (int k = 0; k < kDotK; ++k) {
    pr.x[k] = (k == 1) ? x1 : x0;
    pr.y[k] = (k == 1) ? y1 : y0;
  }
  dots_launch<C>(ctx, 2, n, nrhs, pr, out);
}

// out[0][r] = <q,q>_r, out[1][r] = <q,r>_r reading q once (smoother steps).
template <class C>
__global__ void k_dots_qq_qr(int64_t n, int nrhs, const C* __restrict__ q, const C* __restrict__ rv,
                             cplx* __restrict__ partials) {
  typedef typename CTraits<C>::R R;
  __shared__ cplx sm[2][kThreads];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int col = blockIdx.y * blockDim.x + tx;
  R qq = 0;
  C qr = mk<C>((R)0, (R)0);
  if (col < nrhs) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.y + ty; i < n; i += (int64_t)gridDim.x * blockDim.y) {
      const int64_t e = i * nrhs + col;
      const C a = q[e];
      qq += cnorm2(a);
      cfmac(qr, a, rv[e]);
    }
  }
  const int t = ty * blockDim.x + tx;
  sm[0][t] = mkc((double)qq, 0.0);
  sm[1][t] = mkc((double)qr.x, (double)qr.y);
  __syncthreads();
  for (int h = blockDim.y / 2; h > 0; h >>= 1) {
    if (ty < h) {
      sm[0][t] = cadd(sm[0][t], sm[0][t + h * blockDim.x]);
      sm[1][t] = cadd(sm[1][t], sm[1][t + h * blockDim.x]);
    }
    __syncthreads();
  }
  if (ty == 0 && col < nrhs) {
    partials[((int64_t)blockIdx.x * 2 + 0) * nrhs + col] = sm[0][tx];
    partials[((int64_t)blockIdx.x * 2 + 1) * nrhs + col] = sm[1][tx];
  }
}

template <class C> void dots_qq_qr(qd_ctx& ctx, int64_t n, int nrhs, const C* q, const C* r, cplx* out) {
  Sweep s = sweep(n, nrhs);
  ctx.red_partials.resize((size_t)s.grid.x * 2 * nrhs * sizeof(cplx));
  {
    ProfScope ps(ctx, sizeof(C) == 16 ? QD_PROF_BLAS_F64 : QD_PROF_DOTS_F32, 12.0 * n * nrhs,
                 (double)sizeof(C) * 2.0 * n * nrhs);
    k_dots_qq_qr<C><<<s.grid, s.block, 0, ctx.stream>>>(n, nrhs, q, r, ctx.red_partials.as<cplx>());
    QD_LAUNCH_CHECK();
  }
  k_dots_final<<<div_up(2 * nrhs, 8), 256, 0, ctx.stream>>>(2, nrhs, s.grid.x, ctx.red_partials.as<cplx>(), out);
  QD_LAUNCH_CHECK();
}

// Y_j[i,r] -= sum_k coef[k][r] X_k[i,r] for (Y, X) and, when Y2 != null,
// (Y2, X2) with the same coefficients; columns with active[r] == 0 untouched.
template <class C>
__global__ void k_multi_axpy(int K, int64_t n, int nrhs, const cplx* __restrict__ coef,
                             const int* __restrict__ active, const C* __restrict__ X, int64_t xs,
                             C* __restrict__ Y, const C* __restrict__ X2, C* __restrict__ Y2) {
  typedef typename CTraits<C>::R R;
  const int64_t tot = n * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % nrhs);
    if (active && !active[r]) continue;
    C y = Y[e];
    C y2 = Y2 ? Y2[e] : mk<C>((R)0, (R)0);
    for (int k = 0; k < K; ++k) {
      const cplx cd = coef[(int64_t)k * nrhs + r];
      const C c = mk<C>((R)(-cd.x), (R)(-cd.y));
      cfma(y, c, X[k * xs + e]);
      if (Y2) cfma(y2, c, X2[k * xs + e]);
    }
    Y[e] = y;
    if (Y2) Y2[e] = y2;
  }
}

inline int grid_1d(int64_t tot, int threads = kThreads) {
  int64_t b = (tot + threads - 1) / threads;
  const int64_t cap = 32LL * kNumSMs;
  return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

template <class C>
void multi_axpy(qd_ctx& ctx, int K, int64_t n, int nrhs, const cplx* coef, const int* active,
                const C* X, int64_t xs, C* Y, const C* X2 = nullptr, C* Y2 = nullptr) {
  if (K <= 0) return;
  ProfScope ps(ctx, sizeof(C) == 16 ? QD_PROF_BLAS_F64 : QD_PROF_AXPY_F32, 8.0 * K * n * nrhs * (Y2 ? 2 : 1),
               (double)sizeof(C) * (K + 2.0) * n * nrhs * (Y2 ? 2 : 1));
  k_multi_axpy<C><<<grid_1d(n * nrhs), kThreads, 0, ctx.stream>>>(K, n, nrhs, coef, active, X, xs, Y,
                                                                 X2, Y2);
  QD_LAUNCH_CHECK();
}

// y = a x + b y with per-column complex a, b (device arrays; nullptr a -> 1,
// nullptr b -> 0).  Columns with active[r] == 0 untouched.
template <class C>
__global__ void k_axpby(int64_t n, int nrhs, const cplx* __restrict__ a, const C* __restrict__ x,
                        const cplx* __restrict__ b, C* __restrict__ y, const int* __restrict__ active) {
  typedef typename CTraits<C>::R R;
  const int64_t tot = n * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % nrhs);
    if (active && !active[r]) continue;
    C v = x[e];
    if (a) v = cmul(mk<C>((R)a[r].x, (R)a[r].y), v);
    if (b) cfma(v, mk<C>((R)b[r].x, (R)b[r].y), y[e]);
    y[e] = v;
  }
}

template <class C>
void axpby(qd_ctx& ctx, int64_t n, int nrhs, const cplx* a, const C* x, const cplx* b, C* y,
           const int* active = nullptr) {
  k_axpby<C><<<grid_1d(n * nrhs), kThreads, 0, ctx.stream>>>(n, nrhs, a, x, b, y, active);
  QD_LAUNCH_CHECK();
}

// z = x - y (elementwise, all columns)
template <class C>
__global__ void k_sub(int64_t tot, const C* x, const C* y, C* z) {  // z may alias x or y
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x)
    z[e] = csub(x[e], y[e]);
}
template <class C> void sub(qd_ctx& ctx, int64_t tot, const C* x, const C* y, C* z) {
  k_sub<C><<<grid_1d(tot), kThreads, 0, ctx.stream>>>(tot, x, y, z);
  QD_LAUNCH_CHECK();
}

// y += x (elementwise)
template <class C>
__global__ void k_add(int64_t tot, const C* __restrict__ x, C* __restrict__ y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] = cadd(y[e], x[e]);
}
template <class C> void add(qd_ctx& ctx, int64_t tot, const C* x, C* y) {
  k_add<C><<<grid_1d(tot), kThreads, 0, ctx.stream>>>(tot, x, y);
  QD_LAUNCH_CHECK();
}

// gamma5 on a field with `dof` per site: negate the second half of each site.
template <class C>
__global__ void k_gamma5(int64_t nsites, int dof, int nrhs, const C* __restrict__ x, C* __restrict__ y) {
  const int64_t tot = nsites * dof * nrhs;
  const int half = dof / 2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int d = (int)((e / nrhs) % dof);
    C v = x[e];
    if (d >= half) { v.x = -v.x; v.y = -v.y; }
    y[e] = v;
  }
}
template <class C> void gamma5(qd_ctx& ctx, int64_t nsites, int dof, int nrhs, const C* x, C* y) {
  k_gamma5<C><<<grid_1d(nsites * dof * nrhs), kThreads, 0, ctx.stream>>>(nsites, dof, nrhs, x, y);
  QD_LAUNCH_CHECK();
}

template <class C> void copy(qd_ctx& ctx, int64_t tot, const C* x, C* y) {
  QD_CUDA(cudaMemcpyAsync(y, x, tot * sizeof(C), cudaMemcpyDeviceToDevice, ctx.stream));
}
template <class C> void zero(qd_ctx& ctx, int64_t tot, C* y) {
  QD_CUDA(cudaMemsetAsync(y, 0, tot * sizeof(C), ctx.stream));
}

}  // namespace blas
}  // namespace qd
