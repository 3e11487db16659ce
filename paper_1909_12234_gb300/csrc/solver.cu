// Krylov solvers and multigrid: flexible GCR (Sec. 1 inexact solves A^{-1}_xi
// with the true-residual stopping rule; Sec. 2 and Sec. 3 use GCR on every
// level), minimal-residual smoothing and null vectors, the V-cycle of the
// two-grid method (Sec. 2) and the adaptive setup (Sec. 2, Sec. 4
// tolerance 1e-2 / 200 iterations).
#include "blas.cuh"
#include "direct.cuh"
#include "mg.cuh"
#include "tc_gemm.cuh"

namespace qd {

template <class C> void Op<C>::residual(qd_ctx& ctx, const C* b, const C* x, C* r, int nrhs) const {
  apply(ctx, x, r, nrhs);
  blas::sub(ctx, n() * nrhs, b, r, r);
}
template struct Op<cplx>;
template struct Op<cplxf>;

// ---------------------------------------------------------------------------
// Fused update kernels with a per-column |r|^2 reduction (deterministic).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void rows_reduce(double v, cplx* partials, int nrhs) {
  __shared__ double sm[blas::kThreads];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int t = ty * blockDim.x + tx;
  sm[t] = v;
  __syncthreads();
  for (int h = blockDim.y / 2; h > 0; h >>= 1) {
    if (ty < h) sm[t] += sm[t + h * blockDim.x];
    __syncthreads();
  }
  const int r = blockIdx.y * blockDim.x + tx;
  if (ty == 0 && r < nrhs) partials[(int64_t)blockIdx.x * nrhs + r] = mkc(sm[tx], 0.0);
}

// GCR step for active columns, with s2[0][r] = <q,q>, s2[1][r] = <q,r>:
//   a = <q,r>/<q,q>;  x += a p;  r -= a q;  q, p scaled to ||q|| = 1.
template <class C>
__global__ void k_gcr_update(int64_t n, int nrhs, const cplx* __restrict__ s2,
                             const int* __restrict__ active, C* __restrict__ q, C* __restrict__ p,
                             C* __restrict__ x, C* __restrict__ r, cplx* __restrict__ partials) {
  typedef typename CTraits<C>::R R;
  const int col = blockIdx.y * blockDim.x + threadIdx.x;
  R acc = 0;
  if (col < nrhs && active[col]) {
    const double qq = s2[col].x;
    const cplx qr = s2[nrhs + col];
    const double inv = qq > 0.0 ? 1.0 / sqrt(qq) : 0.0;
    const double ar = qq > 0.0 ? qr.x / qq : 0.0, ai = qq > 0.0 ? qr.y / qq : 0.0;
    const C a = mk<C>((R)ar, (R)ai), na = mk<C>((R)(-ar), (R)(-ai));
    const R ri = (R)inv;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i < n;
         i += (int64_t)gridDim.x * blockDim.y) {
      const int64_t e = i * nrhs + col;
      const C qv = q[e], pv = p[e];
      C xv = x[e], rv = r[e];
      cfma(xv, a, pv);
      cfma(rv, na, qv);
      x[e] = xv;
      r[e] = rv;
      q[e] = cscale(ri, qv);
      p[e] = cscale(ri, pv);
      acc += cnorm2(rv);
    }
  }
  rows_reduce((double)acc, partials, nrhs);
}

// Minimal-residual step: a = <q,r>/<q,q>; x += a r; r -= a q.
template <class C>
__global__ void k_mr_update(int64_t n, int nrhs, const cplx* __restrict__ s2,
                            const int* __restrict__ active, C* __restrict__ q, C* __restrict__ x,
                            C* __restrict__ r, cplx* __restrict__ partials, const C* __restrict__ rin = nullptr,
                            C* __restrict__ Az = nullptr, bool write_r = true) {
  typedef typename CTraits<C>::R R;
  const int col = blockIdx.y * blockDim.x + threadIdx.x;
  R acc = 0;
  if (col < nrhs && (!active || active[col])) {
    const double qq = s2[col].x;
    const cplx qr = s2[nrhs + col];
    const double ar = qq > 0.0 ? qr.x / qq : 0.0, ai = qq > 0.0 ? qr.y / qq : 0.0;
    const C a = mk<C>((R)ar, (R)ai), na = mk<C>((R)(-ar), (R)(-ai));
    for (int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i < n;
         i += (int64_t)gridDim.x * blockDim.y) {
      const int64_t e = i * nrhs + col;
      const C qv = q[e];
      C xv = x[e], rv = r[e];
      cfma(xv, a, rv);
      cfma(rv, na, qv);
      x[e] = xv;
      if (write_r) r[e] = rv;
      if (Az) {
        // A x = rin - res once res is the residual of x
        const C bv = rin[e];
        Az[e] = mk<C>(bv.x - rv.x, bv.y - rv.y);
      }
      acc += cnorm2(rv);
    }
  }
  if (partials) rows_reduce((double)acc, partials, nrhs);
}

// rn2[c] = sum of partials; active columns stay active while
// rn2 > tol2 * ref2; counts active columns and non-finite norms.
// One warp per column (fixed lane order and shuffle tree: deterministic).
__global__ void k_resid_final(int nrhs, int nblk, const cplx* __restrict__ partials, cplx* __restrict__ rn2,
                              const cplx* __restrict__ ref2, double tol2, int* __restrict__ active,
                              int* __restrict__ count, int* __restrict__ nonfin, int* __restrict__ iters) {
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= nrhs) return;
  if (!active[c]) return;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += partials[(int64_t)b * nrhs + c].x;
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane != 0) return;
  rn2[c] = mkc(s, 0.0);
  if (iters) iters[c] += 1;
  if (!isfinite(s)) {
    atomicAdd(nonfin, 1);
    active[c] = 0;
    return;
  }
  if (s > tol2 * ref2[c].x) {
    atomicAdd(count, 1);
  } else {
    active[c] = 0;
  }
}

// active[c] = (rn2 > tol2 * ref2), counting active and non-finite columns.
__global__ void k_set_active(int nrhs, const cplx* __restrict__ rn2, const cplx* __restrict__ ref2, double tol2,
                             int* __restrict__ active, int* __restrict__ count, int* __restrict__ nonfin) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nrhs) return;
  const double s = rn2[c].x;
  if (!isfinite(s) || !isfinite(ref2[c].x)) {
    atomicAdd(nonfin, 1);
    active[c] = 0;
    return;
  }
  const int a = s > tol2 * ref2[c].x ? 1 : 0;
  active[c] = a;
  if (a) atomicAdd(count, 1);
}

// ---------------------------------------------------------------------------
// One-pass (classical) Gram-Schmidt GCR with a deferred solution update, for
// FP32 fields.  The preconditioned directions Pt_i = M r are never rewritten:
// P_i = Pt_i - sum_{k<i} beta_ik P_k is kept implicit, Q_i = A Pt_i is
// orthogonalised in place (unnormalised, nu_i = <Q_i, Q_i>), and the solution
// x += sum_i a_i P_i = sum_k d_k Pt_k is formed once per cycle with
// d_k = a_k - sum_{i>k} beta_ik d_i.  Per iteration this reads the basis once
// for the projections and once for the update, instead of also updating P
// and rewriting q, p, x every iteration.
// ---------------------------------------------------------------------------
constexpr int kMaxMdot = 16;

// partials[(blk*K + k)*nrhs + c] = sum over this block's rows of conj(Q_k) y
// for k < K <= 16, reading y once (K a template argument so that the
// accumulators stay in registers).
template <int K>
__global__ void k_mdot_f32(int64_t n, int nrhs, const float2* __restrict__ Q, int64_t qs,
                           const float2* __restrict__ y, cplx* __restrict__ partials) {
  __shared__ float2 sm[K][blas::kThreads];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int c = blockIdx.y * blockDim.x + tx;
  float2 acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = make_float2(0.f, 0.f);
  if (c < nrhs) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.y + ty; i < n; i += (int64_t)gridDim.x * blockDim.y) {
      const int64_t e = i * nrhs + c;
      const float2 yv = y[e];
#pragma unroll
      for (int k = 0; k < K; ++k) cfmac(acc[k], Q[k * qs + e], yv);
    }
  }
  const int t = ty * blockDim.x + tx;
#pragma unroll
  for (int k = 0; k < K; ++k) sm[k][t] = acc[k];
  __syncthreads();
  for (int h = blockDim.y / 2; h > 0; h >>= 1) {
    if (ty < h) {
#pragma unroll
      for (int k = 0; k < K; ++k) sm[k][t] = cadd(sm[k][t], sm[k][t + h * blockDim.x]);
    }
    __syncthreads();
  }
  if (ty == 0 && c < nrhs)
#pragma unroll
    for (int k = 0; k < K; ++k)
      partials[((int64_t)blockIdx.x * K + k) * nrhs + c] = mkc((double)sm[k][tx].x, (double)sm[k][tx].y);
}

// Q_i -= sum_{k<i} (beta'_k / nu_k) Q_k for active columns, with the partial
// sums of <Q_i, Q_i> and <Q_i, r> (two values per column).  The coefficients
// are recorded in btab[k][c] (0 for inactive columns).
template <int I>
__global__ void k_orth_f32(int64_t n, int nrhs, float2* __restrict__ Q, int64_t qs,
                           const float2* __restrict__ r, const cplx* __restrict__ braw,
                           const cplx* __restrict__ ngtab, const int* __restrict__ active,
                           cplx* __restrict__ btab, cplx* __restrict__ partials) {
  constexpr int i = I;
  __shared__ double smr[2][blas::kThreads];
  __shared__ double smi[blas::kThreads];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int c = blockIdx.y * blockDim.x + tx;
  const bool act = c < nrhs && active[c];
  float2 coef[I > 0 ? I : 1];
#pragma unroll
  for (int k = 0; k < I; ++k) {
    coef[k] = make_float2(0.f, 0.f);
    if (act) {
      const double nu = ngtab[(int64_t)(2 * k) * nrhs + c].x;
      const cplx b = braw[(int64_t)k * nrhs + c];
      if (nu > 0.0) coef[k] = make_float2((float)(b.x / nu), (float)(b.y / nu));
    }
  }
  if (blockIdx.x == 0 && ty == 0 && c < nrhs)
#pragma unroll
    for (int k = 0; k < I; ++k) btab[(int64_t)k * nrhs + c] = mkc((double)coef[k].x, (double)coef[k].y);
  float nn = 0.f;
  float2 nr = make_float2(0.f, 0.f);
  float2* Qi = Q + (int64_t)i * qs;
  if (act) {
    for (int64_t row = (int64_t)blockIdx.x * blockDim.y + ty; row < n; row += (int64_t)gridDim.x * blockDim.y) {
      const int64_t e = row * nrhs + c;
      float2 q = Qi[e];
#pragma unroll
      for (int k = 0; k < I; ++k) cfma(q, make_float2(-coef[k].x, -coef[k].y), Q[k * qs + e]);
      Qi[e] = q;
      nn += cnorm2(q);
      cfmac(nr, q, r[e]);
    }
  }
  const int t = ty * blockDim.x + tx;
  smr[0][t] = (double)nn;
  smr[1][t] = (double)nr.x;
  smi[t] = (double)nr.y;
  __syncthreads();
  for (int h = blockDim.y / 2; h > 0; h >>= 1) {
    if (ty < h) {
      smr[0][t] += smr[0][t + h * blockDim.x];
      smr[1][t] += smr[1][t + h * blockDim.x];
      smi[t] += smi[t + h * blockDim.x];
    }
    __syncthreads();
  }
  if (ty == 0 && c < nrhs) {
    partials[((int64_t)blockIdx.x * 2 + 0) * nrhs + c] = mkc(smr[0][tx], 0.0);
    partials[((int64_t)blockIdx.x * 2 + 1) * nrhs + c] = mkc(smr[1][tx], smi[tx]);
  }
}

// a = <Q_i, r> / <Q_i, Q_i>; r -= a Q_i for active columns (a recorded in
// atab[c], 0 for inactive ones), with the partial sums of |r|^2.
__global__ void k_rupd_f32(int64_t n, int nrhs, const float2* __restrict__ Qi, float2* __restrict__ r,
                           const cplx* __restrict__ ng, const int* __restrict__ active, cplx* __restrict__ atab,
                           cplx* __restrict__ partials) {
  const int col = blockIdx.y * blockDim.x + threadIdx.x;
  float acc = 0.f;
  const bool act = col < nrhs && active[col];
  double ar = 0.0, ai = 0.0;
  if (act) {
    const double nu = ng[col].x;
    const cplx g = ng[nrhs + col];
    if (nu > 0.0) {
      ar = g.x / nu;
      ai = g.y / nu;
    }
  }
  if (blockIdx.x == 0 && threadIdx.y == 0 && col < nrhs) atab[col] = mkc(ar, ai);
  if (act) {
    const float2 na = make_float2((float)(-ar), (float)(-ai));
    for (int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i < n; i += (int64_t)gridDim.x * blockDim.y) {
      const int64_t e = i * nrhs + col;
      float2 rv = r[e];
      cfma(rv, na, Qi[e]);
      r[e] = rv;
      acc += cnorm2(rv);
    }
  }
  rows_reduce((double)acc, partials, nrhs);
}

// Per column: d_{m-1} = a_{m-1}, d_k = a_k - sum_{i>k} beta_ik d_i; writes
// coef[k][c] = -d_k (multi_axpy subtracts).
__global__ void k_backsub(int m, int nrhs, const cplx* __restrict__ atab, const cplx* __restrict__ btab,
                          cplx* __restrict__ coef) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nrhs) return;
  cplx d[kMaxMdot];
  for (int k = m - 1; k >= 0; --k) {
    cplx v = atab[(int64_t)k * nrhs + c];
    for (int i = k + 1; i < m; ++i)
      cfma(v, cscale(-1.0, btab[((int64_t)i * kMaxMdot + k) * nrhs + c]), d[i]);
    d[k] = v;
    coef[(int64_t)k * nrhs + c] = mkc(-v.x, -v.y);
  }
}

// Launch k_mdot_f32<K> / k_orth_f32<I> for a run-time count (1..16 / 0..15).
template <int K>
static void launch_mdot(int k, dim3 g, dim3 b, cudaStream_t st, int64_t n, int nrhs, const float2* Q, int64_t qs,
                        const float2* y, cplx* partials) {
  if constexpr (K <= kMaxMdot) {
    if (k == K) {
      k_mdot_f32<K><<<g, b, 0, st>>>(n, nrhs, Q, qs, y, partials);
      return;
    }
    launch_mdot<K + 1>(k, g, b, st, n, nrhs, Q, qs, y, partials);
  }
}
template <int I>
static void launch_orth(int i, dim3 g, dim3 b, cudaStream_t st, int64_t n, int nrhs, float2* Q, int64_t qs,
                        const float2* r, const cplx* braw, const cplx* ngtab, const int* active, cplx* btab,
                        cplx* partials) {
  if constexpr (I < kMaxMdot) {
    if (i == I) {
      k_orth_f32<I><<<g, b, 0, st>>>(n, nrhs, Q, qs, r, braw, ngtab, active, btab, partials);
      return;
    }
    launch_orth<I + 1>(i, g, b, st, n, nrhs, Q, qs, r, braw, ngtab, active, btab, partials);
  }
}

static void read_flags(qd_ctx& ctx, const int* dev, int n, int* host) {
  QD_CUDA(cudaMemcpyAsync(ctx.host_pinned, dev, n * sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaStreamSynchronize(ctx.stream));
  for (int i = 0; i < n; ++i) host[i] = ctx.host_pinned[i];
}

// ---------------------------------------------------------------------------
// GCR
// ---------------------------------------------------------------------------
template <class C> void GCR<C>::buffers(std::vector<const void*>& v) const {
  for (const DevBuf* b : {&P_, &Q_, &r_, &t_, &sc_, &act_, &tab_}) v.push_back(b->as<void>());
}

template <class C> bool GCR<C>::embeds(int restart) const {
  return embed > 0 && orth_passes == 1 && sizeof(C) == sizeof(cplxf) && restart <= kMaxMdot;
}

template <class C> void GCR<C>::ensure(int64_t n, int nrhs, int m, int64_t emb) {
  if (n == cap_n_ && nrhs <= cap_rhs_ && m <= cap_m_ && emb == cap_emb_) return;
  const size_t vec = (size_t)n * nrhs * sizeof(C);
  const size_t slot = vec + (size_t)emb * sizeof(C);
  P_.release();
  Q_.release();
  P_.resize(slot * m);
  Q_.resize(vec * m);
  r_.resize(slot);
  t_.resize(vec);
  cap_emb_ = emb;
  sc_.resize((size_t)(4 + m) * nrhs * sizeof(cplx));
  act_.resize((size_t)(2 * nrhs + 4) * sizeof(int));
  cap_n_ = n;
  cap_rhs_ = nrhs;
  cap_m_ = m;
}

template <class C>
void GCR<C>::solve(qd_ctx& ctx, const Op<C>& A, Precond<C>* M, const C* b, C* x, int nrhs, double tol,
                   int maxit, int restart, SolveInfo* info) {
  QD_REQUIRE(restart >= 1 && restart <= 256, "GCR restart length must be in [1, 256]");
  QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
  const int64_t n = A.n();
  const int64_t tot = n * nrhs;
  // FP32 with one Gram-Schmidt pass: the fused form with a deferred update
  const bool fused = orth_passes == 1 && sizeof(C) == sizeof(cplxf) && restart <= kMaxMdot;
  const int64_t emb = embeds(restart) ? embed : 0;
  QD_REQUIRE(emb == 0 || emb >= tot, "GCR embedding shorter than a vector");
  ensure(n, nrhs, restart, emb);
  const int64_t pst = tot + emb;  // stride of the directions P_i
  tab_.resize((size_t)(2 * kMaxMdot + kMaxMdot * kMaxMdot + 3 * kMaxMdot) * nrhs * sizeof(cplx));
  cplx* ngtab = tab_.as<cplx>();                          // [m][2][nrhs]: nu_i, gamma_i
  cplx* btab = ngtab + (int64_t)2 * kMaxMdot * nrhs;      // [m][16][nrhs]: beta_ik
  cplx* atab = btab + (int64_t)kMaxMdot * kMaxMdot * nrhs;  // [m][nrhs]: a_i
  cplx* coefx = atab + (int64_t)kMaxMdot * nrhs;           // [m][nrhs]: -d_k
  cplx* braw = coefx + (int64_t)kMaxMdot * nrhs;           // [m][nrhs]: <Q_k, Q_i>
  C* P = P_.as<C>() + emb;
  C* Q = Q_.as<C>();
  C* r = r_.as<C>() + emb;
  C* t = t_.as<C>();
  if (emb) QD_CUDA(cudaMemsetAsync(r_.as<C>(), 0, (size_t)emb * sizeof(C), ctx.stream));  // the leading part of r
  cplx* bn2 = sc_.as<cplx>();
  cplx* rn2 = bn2 + nrhs;
  cplx* s2 = bn2 + 2 * nrhs;
  cplx* beta = bn2 + 4 * nrhs;
  int* act = act_.as<int>();
  int* iters = act + nrhs;
  int* flags = act + 2 * nrhs;  // [0] count, [1] non-finite
  const double tol2 = tol * tol;
  blas::zero(ctx, tot, x);
  blas::copy(ctx, tot, b, r);
  blas::dots(ctx, 1, n, nrhs, b, 0, b, 0, bn2);
  QD_CUDA(cudaMemcpyAsync(rn2, bn2, nrhs * sizeof(cplx), cudaMemcpyDeviceToDevice, ctx.stream));
  QD_CUDA(cudaMemsetAsync(iters, 0, nrhs * sizeof(int), ctx.stream));
  const blas::Sweep sw = blas::sweep(n, nrhs);
  // room for the largest Gram-Schmidt reduction of a cycle up front, so that
  // the buffer keeps its address through the solve
  ctx.red_partials.resize((size_t)sw.grid.x * (restart > 2 ? restart : 2) * nrhs * sizeof(cplx));
  int its = 0;
  int hflags[2];
  // tol <= 0: exactly maxit iterations and no host synchronisation (columns
  // with a zero residual are masked on the device)
  const bool check = tol > 0.0;
  // stagnation test: residual norms of the active columns every stag_window
  // iterations against the previous snapshot
  bool stag = false;
  std::vector<cplx> snap, now(nrhs);
  std::vector<int> hact(nrhs);
  auto stagnating = [&]() -> bool {
    if (!check || stag_window <= 0 || its == 0 || its % stag_window != 0) return false;
    QD_CUDA(cudaMemcpyAsync(now.data(), rn2, nrhs * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
    QD_CUDA(cudaMemcpyAsync(hact.data(), act, nrhs * sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
    QD_CUDA(cudaStreamSynchronize(ctx.stream));
    bool st = false;
    if (!snap.empty())
      for (int c = 0; c < nrhs; ++c)
        if (hact[c] && now[c].x > stag_ratio * stag_ratio * snap[c].x) st = true;
    snap = now;
    return st;
  };
  while (true) {
    if (!check && its >= maxit) break;
    QD_CUDA(cudaMemsetAsync(flags, 0, 2 * sizeof(int), ctx.stream));
    k_set_active<<<div_up(nrhs, 128), 128, 0, ctx.stream>>>(nrhs, rn2, bn2, tol2, act, flags, flags + 1);
    QD_LAUNCH_CHECK();
    if (check) {
      read_flags(ctx, flags, 2, hflags);
      if (hflags[1]) fail(QD_ERR_NONFINITE, "non-finite residual in GCR");
      if (hflags[0] == 0 || its >= maxit) break;
    }
    if (fused) {
      // one-pass Gram-Schmidt, deferred solution update (see k_orth_f32)
      float2* Pf = reinterpret_cast<float2*>(P);
      float2* Qf = reinterpret_cast<float2*>(Q);
      float2* rf = reinterpret_cast<float2*>(r);
      int mi = 0;
      for (int i = 0; i < restart; ++i) {
        C* Pi = P + i * pst;
        C* Qi = Q + i * tot;
        bool have_q = false;
        if (M)
          have_q = M->apply_az(ctx, A, r, Pi, Qi, nrhs);
        else
          blas::copy(ctx, tot, r, Pi);
        if (!have_q) A.apply(ctx, Pi, Qi, nrhs);
        if (i > 0) {
          {
            ProfScope ps(ctx, QD_PROF_DOTS_F32, 8.0 * i * n * nrhs, 8.0 * (i + 1.0) * n * nrhs);
            launch_mdot<1>(i, sw.grid, sw.block, ctx.stream, n, nrhs, Qf, tot, Qf + i * tot,
                           ctx.red_partials.as<cplx>());
            QD_LAUNCH_CHECK();
          }
          blas::k_dots_final<<<div_up(i * nrhs, 8), 256, 0, ctx.stream>>>(i, nrhs, sw.grid.x, ctx.red_partials.as<cplx>(),
                                                                    braw);
          QD_LAUNCH_CHECK();
        }
        {
          ProfScope ps(ctx, QD_PROF_AXPY_F32, 8.0 * (i + 2.0) * n * nrhs, 8.0 * (i + 3.0) * n * nrhs);
          launch_orth<0>(i, sw.grid, sw.block, ctx.stream, n, nrhs, Qf, tot, rf, braw, ngtab, act,
                         btab + (int64_t)i * kMaxMdot * nrhs, ctx.red_partials.as<cplx>());
          QD_LAUNCH_CHECK();
        }
        blas::k_dots_final<<<div_up(2 * nrhs, 8), 256, 0, ctx.stream>>>(2, nrhs, sw.grid.x, ctx.red_partials.as<cplx>(),
                                                                  ngtab + (int64_t)2 * i * nrhs);
        QD_LAUNCH_CHECK();
        {
          ProfScope ps(ctx, QD_PROF_UPDATE_F32, 8.0 * n * nrhs, 8.0 * 3.0 * n * nrhs);
          k_rupd_f32<<<sw.grid, sw.block, 0, ctx.stream>>>(n, nrhs, Qf + i * tot, rf, ngtab + (int64_t)2 * i * nrhs, act,
                                                            atab + (int64_t)i * nrhs, ctx.red_partials.as<cplx>());
          QD_LAUNCH_CHECK();
        }
        QD_CUDA(cudaMemsetAsync(flags, 0, 2 * sizeof(int), ctx.stream));
        k_resid_final<<<div_up(nrhs, 8), 256, 0, ctx.stream>>>(nrhs, sw.grid.x, ctx.red_partials.as<cplx>(), rn2,
                                                              bn2, tol2, act, flags, flags + 1, iters);
        QD_LAUNCH_CHECK();
        ++its;
        ++mi;
        if (check) {
          read_flags(ctx, flags, 2, hflags);
          if (hflags[1]) fail(QD_ERR_NONFINITE, "non-finite residual in GCR");
          if (hflags[0] == 0) break;
          if (stagnating()) {
            stag = true;
            break;
          }
        }
        if (its >= maxit) break;
      }
      // x += sum_k d_k Pt_k
      k_backsub<<<div_up(nrhs, 128), 128, 0, ctx.stream>>>(mi, nrhs, atab, btab, coefx);
      QD_LAUNCH_CHECK();
      blas::multi_axpy(ctx, mi, n, nrhs, coefx, nullptr, P, pst, x);
      (void)Pf;
      if (!check && its >= maxit) break;
      A.residual(ctx, b, x, r, nrhs);
      blas::dots(ctx, 1, n, nrhs, r, 0, r, 0, rn2);
      if (stag) break;
      continue;
    }
    for (int i = 0; i < restart; ++i) {
      C* Pi = P + i * tot;
      C* Qi = Q + i * tot;
      bool have_q = false;
      if (M)
        have_q = M->apply_az(ctx, A, r, Pi, Qi, nrhs);
      else
        blas::copy(ctx, tot, r, Pi);
      if (!have_q) A.apply(ctx, Pi, Qi, nrhs);
      for (int pass = 0; pass < orth_passes && i > 0; ++pass) {
        blas::dots(ctx, i, n, nrhs, Q, tot, Qi, 0, beta);
        blas::multi_axpy(ctx, i, n, nrhs, beta, act, Q, tot, Qi, P, Pi);
      }
      blas::dots2(ctx, n, nrhs, Qi, Qi, Qi, r, s2);
      ctx.red_partials.resize((size_t)sw.grid.x * nrhs * sizeof(cplx));
      {
        ProfScope ps(ctx, sizeof(C) == 16 ? QD_PROF_BLAS_F64 : QD_PROF_UPDATE_F32, 16.0 * n * nrhs,
                     (double)sizeof(C) * 8.0 * n * nrhs);
        k_gcr_update<C><<<sw.grid, sw.block, 0, ctx.stream>>>(n, nrhs, s2, act, Qi, Pi, x, r,
                                                              ctx.red_partials.as<cplx>());
        QD_LAUNCH_CHECK();
      }
      QD_CUDA(cudaMemsetAsync(flags, 0, 2 * sizeof(int), ctx.stream));
      k_resid_final<<<div_up(nrhs, 8), 256, 0, ctx.stream>>>(nrhs, sw.grid.x, ctx.red_partials.as<cplx>(), rn2,
                                                            bn2, tol2, act, flags, flags + 1, iters);
      QD_LAUNCH_CHECK();
      ++its;
      if (check) {
        read_flags(ctx, flags, 2, hflags);
        if (hflags[1]) fail(QD_ERR_NONFINITE, "non-finite residual in GCR");
        if (hflags[0] == 0) break;
        if (stagnating()) {
          stag = true;
          break;
        }
      }
      if (its >= maxit) break;
    }
    if (!check && its >= maxit) break;  // no further cycle reads the residual
    // true residual r = b - A x
    A.residual(ctx, b, x, r, nrhs);
    blas::dots(ctx, 1, n, nrhs, r, 0, r, 0, rn2);
    if (stag) break;
  }
  if (info) {
    info->stagnated = stag;
    std::vector<cplx> hb(nrhs), hr(nrhs);
    info->iters.assign(nrhs, 0);
    QD_CUDA(cudaMemcpyAsync(hb.data(), bn2, nrhs * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
    QD_CUDA(cudaMemcpyAsync(hr.data(), rn2, nrhs * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
    QD_CUDA(cudaMemcpyAsync(info->iters.data(), iters, nrhs * sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
    QD_CUDA(cudaStreamSynchronize(ctx.stream));
    info->iterations = its;
    info->true_rel.assign(nrhs, 0.0);
    info->converged = 0;
    info->max_rel = 0.0;
    for (int c = 0; c < nrhs; ++c) {
      const double rel = hb[c].x > 0.0 ? std::sqrt(hr[c].x / hb[c].x) : 0.0;
      info->true_rel[c] = rel;
      if (rel <= tol) info->converged++;
      if (rel > info->max_rel || rel != rel) info->max_rel = rel;
    }
  }
}

template class GCR<cplx>;
template class GCR<cplxf>;

// ---------------------------------------------------------------------------
// Minimal-residual steps
// ---------------------------------------------------------------------------
template <class C>
void mr_steps(qd_ctx& ctx, const Op<C>& A, const C* b, C* x, bool x_is_zero, int nrhs, int nsteps,
              double tol, C* r, C* q, int* steps_dev, DevBuf& scratch) {
  const int64_t n = A.n(), tot = n * nrhs;
  scratch.resize((size_t)4 * nrhs * sizeof(cplx) + (size_t)(nrhs + 4) * sizeof(int));
  cplx* s2 = scratch.as<cplx>();
  cplx* r0n2 = s2 + 2 * nrhs;
  cplx* rn2 = s2 + 3 * nrhs;
  int* act = reinterpret_cast<int*>(s2 + 4 * nrhs);
  int* flags = act + nrhs;
  if (x_is_zero) {
    blas::zero(ctx, tot, x);
    blas::copy(ctx, tot, b, r);
  } else {
    A.residual(ctx, b, x, r, nrhs);
  }
  const bool check = tol > 0.0;
  const blas::Sweep sw = blas::sweep(n, nrhs);
  int hflags[2];
  if (check) {
    blas::dots(ctx, 1, n, nrhs, r, 0, r, 0, r0n2);
    QD_CUDA(cudaMemsetAsync(flags, 0, 2 * sizeof(int), ctx.stream));
    k_set_active<<<div_up(nrhs, 128), 128, 0, ctx.stream>>>(nrhs, r0n2, r0n2, 0.0, act, flags, flags + 1);
    QD_LAUNCH_CHECK();
  }
  for (int k = 0; k < nsteps; ++k) {
    A.apply(ctx, r, q, nrhs);
    blas::dots2(ctx, n, nrhs, q, q, q, r, s2);
    ctx.red_partials.resize((size_t)sw.grid.x * nrhs * sizeof(cplx));
    k_mr_update<C><<<sw.grid, sw.block, 0, ctx.stream>>>(n, nrhs, s2, check ? act : nullptr, q, x, r,
                                                         check ? ctx.red_partials.as<cplx>() : nullptr);
    QD_LAUNCH_CHECK();
    if (check) {
      QD_CUDA(cudaMemsetAsync(flags, 0, 2 * sizeof(int), ctx.stream));
      k_resid_final<<<div_up(nrhs, 8), 256, 0, ctx.stream>>>(nrhs, sw.grid.x, ctx.red_partials.as<cplx>(), rn2,
                                                            r0n2, tol * tol, act, flags, flags + 1, steps_dev);
      QD_LAUNCH_CHECK();
      read_flags(ctx, flags, 2, hflags);
      if (hflags[1]) fail(QD_ERR_NONFINITE, "non-finite residual in minimal-residual iteration");
      if (hflags[0] == 0) break;
    }
  }
}

// nsteps minimal-residual steps on A e = res that add to x and update res
// in place (no convergence checks, no host synchronisation).
template <class C>
void mr_smooth(qd_ctx& ctx, const Op<C>& A, C* x, C* res, C* q, int nrhs, int nsteps, DevBuf& scratch,
               const C* rin, C* Az, bool keep_res) {
  const int64_t n = A.n();
  scratch.resize((size_t)2 * nrhs * sizeof(cplx));
  cplx* s2 = scratch.as<cplx>();
  const blas::Sweep sw = blas::sweep(n, nrhs);
  for (int k = 0; k < nsteps; ++k) {
    A.apply(ctx, res, q, nrhs);
    blas::dots_qq_qr(ctx, n, nrhs, q, res, s2);
    const bool last = k == nsteps - 1;
    const bool last_az = Az && last;
    // the residual of the last step is not written when res is not kept
    const bool write_r = !last || keep_res;
    ProfScope ps(ctx, sizeof(C) == 16 ? QD_PROF_BLAS_F64 : QD_PROF_UPDATE_F32, 8.0 * n * nrhs,
                 (double)sizeof(C) * ((last_az ? 6.0 : 4.0) + (write_r ? 1.0 : 0.0)) * n * nrhs);
    k_mr_update<C><<<sw.grid, sw.block, 0, ctx.stream>>>(n, nrhs, s2, nullptr, q, x, res, nullptr,
                                                         last_az ? rin : nullptr, last_az ? Az : nullptr, write_r);
    QD_LAUNCH_CHECK();
  }
}
template void mr_smooth<cplx>(qd_ctx&, const Op<cplx>&, cplx*, cplx*, cplx*, int, int, DevBuf&, const cplx*,
                              cplx*, bool);
template void mr_smooth<cplxf>(qd_ctx&, const Op<cplxf>&, cplxf*, cplxf*, cplxf*, int, int, DevBuf&,
                               const cplxf*, cplxf*, bool);

template void mr_steps<cplx>(qd_ctx&, const Op<cplx>&, const cplx*, cplx*, bool, int, int, double, cplx*,
                             cplx*, int*, DevBuf&);
template void mr_steps<cplxf>(qd_ctx&, const Op<cplxf>&, const cplxf*, cplxf*, bool, int, int, double,
                              cplxf*, cplxf*, int*, DevBuf&);

// ---------------------------------------------------------------------------
// V-cycle
// ---------------------------------------------------------------------------
template <class C>
MGPrecond<C>::MGPrecond(qd_mg* mg, int level) : mg_(mg), level_(level) {
  if (level + 1 < mg->nlevels) next_.reset(new MGPrecond<C>(mg, level + 1));
  // FP32 coarse GCR: one Gram-Schmidt pass in the fused form (a handful of
  // iterations of a preconditioner lose little orthogonality); FP64 keeps two
  if (sizeof(C) == sizeof(cplxf)) coarse_.orth_passes = 1;
}

template <class C> MGPrecond<C>::~MGPrecond() {
  drop_graphs();
  if (cap_stream_) cudaStreamDestroy(cap_stream_);
}

template <class C> void MGPrecond<C>::drop_graphs() {
  for (Graph& g : graphs_) cudaGraphExecDestroy(g.exec);
  graphs_.clear();
  seen_.clear();
}

// No host synchronisation anywhere below this level: the next level has a
// dense inverse, or its GCR runs a fixed number of iterations (tol <= 0)
// with a V-cycle that is itself free of synchronisation.
template <class C> bool MGPrecond<C>::sync_free() const {
  if (mg_->Cinv<C>(level_ + 1)) return true;
  if (mg_->p.coarse_tol > 0.0 || !next_) return false;
  return next_->sync_free();
}

// Every device buffer the V-cycle below this level reads or writes and that
// can be reallocated after a first call (grow-only buffers: the same address
// means the same, large-enough buffer).
template <class C> void MGPrecond<C>::buffers(std::vector<const void*>& v) const {
  for (const DevBuf* b : {&rc_, &ec_, &t_, &res_, &q_, &d_, &scratch_}) v.push_back(b->as<void>());
  coarse_.buffers(v);
  const CoarseLevel& cl = *mg_->L[level_];
  for (const DevBuf* b : std::initializer_list<const DevBuf*>{&cl.tc_xc, &cl.tc_yc, &cl.tc_B, &cl.tc_part, &cl.tc_err,
                                                                &cl.Cinvf, &cl.Cmf, &cl.Cmb, &cl.ctc_err, &cl.sten_src,
                                                                &cl.ctc_tiles})
    v.push_back(b->as<void>());
  const Transfer& tr = *mg_->T[level_];
  for (const DevBuf* b : std::initializer_list<const DevBuf*>{&tr.Wf, &tr.Wtc, &tr.rtc_err}) v.push_back(b->as<void>());
  if (next_) next_->buffers(v);
}

// The V-cycle ends on minimal-residual smoothing, whose residual gives A z.
template <class C> bool MGPrecond<C>::ends_on_residual() const {
  const LearnedSmoother* ls = level_ == 0 ? mg_->ls.get() : nullptr;
  if (ls && ls->enabled) return ls->mr_steps > 0;
  const int nu = (level_ > 0 && mg_->p.coarse_smoother_steps >= 0) ? mg_->p.coarse_smoother_steps
                                                                    : mg_->p.smoother_steps;
  return nu > 0;
}

template <class C> void MGPrecond<C>::apply(qd_ctx& ctx, const C* r, C* z, int nrhs) { run(ctx, r, z, nullptr, nrhs); }

template <class C> bool MGPrecond<C>::apply_az(qd_ctx& ctx, const Op<C>& A, const C* r, C* z, C* Az, int nrhs) {
  if (!Az || !ends_on_residual() || !A.same(*mg_->op<C>(level_))) {
    run(ctx, r, z, nullptr, nrhs);
    return false;
  }
  run(ctx, r, z, Az, nrhs);
  return true;
}

template <class C> void MGPrecond<C>::run(qd_ctx& ctx, const C* r, C* z, C* Az, int nrhs) {
  if (level_ != 0 || !mg_->p.use_graphs || ctx.prof || !sync_free()) {
    body(ctx, r, z, Az, nrhs);
    return;
  }
  std::vector<const void*> cur;
  buffers(cur);
  cur.push_back(ctx.red_partials.as<void>());
  cur.push_back(reinterpret_cast<const void*>(ctx.red_partials.bytes()));
  cur.push_back(reinterpret_cast<const void*>(ctx.stream));
  // the V-cycle's shape: learned smoother on or off, its MR steps
  const LearnedSmoother* ls = mg_->ls.get();
  cur.push_back(reinterpret_cast<const void*>((uintptr_t)(ls && ls->enabled ? 1 + ls->mr_steps : 0)));
  if (ls) {
    cur.push_back(ls->w64.as<void>());
    cur.push_back(ls->w32.as<void>());
    cur.push_back(reinterpret_cast<const void*>((uintptr_t)ls->layers));
    cur.push_back(ls->t[0].as<void>());
    cur.push_back(ls->t[1].as<void>());
  }
  if (!graphs_.empty() && (graphs_.front().ptrs != cur || graphs_.front().nrhs != nrhs)) {
    // another context or a reallocated buffer: run eagerly once more first
    drop_graphs();
    warm_nrhs_ = -1;
  }
  for (Graph& g : graphs_) {
    if (g.r == r && g.z == z && g.Az == Az) {
      QD_CUDA(cudaGraphLaunch(g.exec, ctx.stream));
      launch_counter().fetch_add(g.kernels, std::memory_order_relaxed);
      return;
    }
  }
  if (warm_nrhs_ != nrhs) {
    // first call at this size: eager, so that every buffer reaches its size
    body(ctx, r, z, Az, nrhs);
    warm_nrhs_ = nrhs;
    seen_.clear();
    return;
  }
  // capture an (input, output) pair only when it comes back: one-shot
  // solves (setup, training) run eagerly and pay no capture
  bool again = false;
  for (const Seen& sn : seen_)
    if (sn.r == r && sn.z == z && sn.Az == Az) again = true;
  if (!again) {
    if (seen_.size() < 64) seen_.push_back({r, z, Az});
    body(ctx, r, z, Az, nrhs);
    return;
  }
  // capture on a private stream (the caller's may be the legacy default
  // stream, which cannot be captured); the graph is then launched on the
  // caller's stream
  if (!cap_stream_) QD_CUDA(cudaStreamCreateWithFlags(&cap_stream_, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  const long long c0 = launch_counter().load();
  const cudaStream_t user = ctx.stream;
  ctx.stream = cap_stream_;
  cudaError_t ce = cudaStreamBeginCapture(cap_stream_, cudaStreamCaptureModeThreadLocal);
  if (ce != cudaSuccess) {
    ctx.stream = user;
    QD_CUDA(ce);
  }
  try {
    body(ctx, r, z, Az, nrhs);
  } catch (...) {
    cudaStreamEndCapture(cap_stream_, &graph);
    if (graph) cudaGraphDestroy(graph);
    ctx.stream = user;
    throw;
  }
  ce = cudaStreamEndCapture(cap_stream_, &graph);
  ctx.stream = user;
  QD_CUDA(ce);
  // kernels captured, not launched: take them off the counter; they count
  // each time the graph is launched
  size_t nn = 0;
  QD_CUDA(cudaGraphGetNodes(graph, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) QD_CUDA(cudaGraphGetNodes(graph, nodes.data(), &nn));
  long long kernels = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType ty;
    QD_CUDA(cudaGraphNodeGetType(nd, &ty));
    if (ty == cudaGraphNodeTypeKernel) ++kernels;
  }
  launch_counter().fetch_sub(launch_counter().load() - c0 >= kernels ? kernels : 0, std::memory_order_relaxed);
  Graph g;
  g.r = r;
  g.z = z;
  g.Az = Az;
  g.nrhs = nrhs;
  g.ptrs = cur;
  g.kernels = kernels;
  const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  QD_CUDA(ie);
  graphs_.push_back(g);
  QD_CUDA(cudaGraphLaunch(g.exec, ctx.stream));
  launch_counter().fetch_add(kernels, std::memory_order_relaxed);
}

template <class C> void MGPrecond<C>::ensure_buffers(int nrhs) {
  const int64_t nf = mg_->geom(level_).nsites * (int64_t)mg_->dof(level_);
  const int64_t nc = mg_->geom(level_ + 1).nsites * (int64_t)mg_->dof(level_ + 1);
  if (nrhs > cap_) {
    rc_.resize(nc * nrhs * sizeof(C));
    ec_.resize(nc * nrhs * sizeof(C));
    t_.resize(nf * nrhs * sizeof(C));
    res_.resize(nf * nrhs * sizeof(C));
    q_.resize(nf * nrhs * sizeof(C));
    d_.resize(nf * nrhs * sizeof(C));
    cap_ = nrhs;
  }
}

// z = W C^{-1} W^H r: the coarse-grid correction
template <class C> void MGPrecond<C>::coarse_correction(qd_ctx& ctx, const C* r, C* z, int nrhs) {
  ensure_buffers(nrhs);
  const Transfer& T = *mg_->T[level_];
  const int64_t nc = mg_->geom(level_ + 1).nsites * (int64_t)mg_->dof(level_ + 1);
  const C* W = mg_->W<C>(level_);
  restrict_<C>(ctx, T, W, r, rc_.as<C>(), nrhs);
  const C* inv = mg_->Cinv<C>(level_ + 1);
  CoarseLevel& cl = *mg_->L[level_];
  if (inv && sizeof(C) == sizeof(cplxf) && cl.tc) {
    tc_dense_apply(ctx, cl, reinterpret_cast<const cplxf*>(rc_.as<C>()), reinterpret_cast<cplxf*>(ec_.as<C>()), nrhs);
  } else if (inv) {
    dense_apply<C>(ctx, (int)nc, nrhs, inv, rc_.as<C>(), ec_.as<C>());
  } else {
    auto Ac = mg_->op<C>(level_ + 1);
    coarse_.solve(ctx, *Ac, next_.get(), rc_.as<C>(), ec_.as<C>(), nrhs, mg_->p.coarse_tol,
                  mg_->p.coarse_maxit, mg_->p.coarse_restart, nullptr);
  }
  prolongate<C>(ctx, T, W, ec_.as<C>(), z, nrhs);
}

template <class C> void MGPrecond<C>::body(qd_ctx& ctx, const C* r, C* z, C* Az, int nrhs) {
  coarse_correction(ctx, r, z, nrhs);
  // smoothing: z += M^{-1} (r - A z).  Plain: M^{-1} = minimal-residual
  // steps from 0, which update z in place with the residual res = r - A z.
  // With a learned smoother on the fine level: z += S (r - A z), then the
  // smoother's own minimal-residual steps.
  auto Af = mg_->op<C>(level_);
  const LearnedSmoother* ls = level_ == 0 ? mg_->ls.get() : nullptr;
  if (ls && ls->enabled) {
    Af->residual(ctx, r, z, res_.as<C>(), nrhs);
    smoother_apply<C>(ctx, *mg_, nrhs, res_.as<C>(), z, true);
    if (ls->mr_steps > 0) {
      Af->residual(ctx, r, z, res_.as<C>(), nrhs);
      mr_smooth<C>(ctx, *Af, z, res_.as<C>(), q_.as<C>(), nrhs, ls->mr_steps, scratch_, r, Az, false);
    }
    return;
  }
  const int nu = (level_ > 0 && mg_->p.coarse_smoother_steps >= 0) ? mg_->p.coarse_smoother_steps
                                                                    : mg_->p.smoother_steps;
  if (nu > 0) {
    Af->residual(ctx, r, z, res_.as<C>(), nrhs);
    mr_smooth<C>(ctx, *Af, z, res_.as<C>(), q_.as<C>(), nrhs, nu, scratch_, r, Az, false);
  }
}

template class MGPrecond<cplx>;
template class MGPrecond<cplxf>;

// ---------------------------------------------------------------------------
// Even-odd (Schur complement) solves
// ---------------------------------------------------------------------------
namespace {
// M = 4 + m0 + i tau gamma5 on the upper (gamma5 = +1) and lower spins, and
// its inverse
void diag_m(double m0, double tau, cplx M[2], cplx Minv[2]) {
  const double m = 4.0 + m0, d = m * m + tau * tau;
  M[0] = mkc(m, tau);
  M[1] = mkc(m, -tau);
  Minv[0] = mkc(m / d, -tau / d);
  Minv[1] = mkc(m / d, tau / d);
}
}  // namespace

template <class C> int64_t SchurOp<C>::nsites() const { return g->geo.nsites / 2; }

template <class C> void SchurOp<C>::apply(qd_ctx& ctx, const C* in, C* out, int nrhs) const {
  const int64_t Vh = g->geo.nsites / 2;
  t.resize((size_t)Vh * 12 * nrhs * sizeof(C));
  cplx M[2], Minv[2];
  diag_m(m0, tau, M, Minv);
  const cplx zero[2] = {mkc(0.0, 0.0), mkc(0.0, 0.0)};
  const cplx quarter[2] = {mkc(-0.25, 0.0), mkc(-0.25, 0.0)};
  // t_e = M^{-1} H_eo in_o, then out_o = M in_o - (1/4) H_oe t_e
  wilson_eo<C>(ctx, g->geo, links, 0, zero, Minv, in, nullptr, t.as<C>(), nrhs);
  wilson_eo<C>(ctx, g->geo, links, 1, M, quarter, t.as<C>(), in, out, nrhs);
}

template <class C> void SchurPrecond<C>::apply(qd_ctx& ctx, const C* r, C* z, int nrhs) {
  QD_REQUIRE(mg && geo, "Schur preconditioner without a V-cycle");
  const int64_t Vh = geo->nsites / 2;
  const size_t half = (size_t)Vh * 12 * nrhs * sizeof(C);
  if (embedded) {
    // r and z are the odd halves of full fields (the even half of r zero)
    const int64_t hn = Vh * 12 * (int64_t)nrhs;
    mg->apply(ctx, r - hn, z - hn, nrhs);
    return;
  }
  if (nrhs != cap_) {
    R_.resize(2 * half);
    Z_.resize(2 * half);
    QD_CUDA(cudaMemsetAsync(R_.as<void>(), 0, half, ctx.stream));  // the even half stays zero
    cap_ = nrhs;
  }
  unsigned char* Rb = R_.as<unsigned char>();
  QD_CUDA(cudaMemcpyAsync(Rb + half, r, half, cudaMemcpyDeviceToDevice, ctx.stream));
  mg->apply(ctx, R_.as<C>(), Z_.as<C>(), nrhs);
  QD_CUDA(cudaMemcpyAsync(z, Z_.as<unsigned char>() + half, half, cudaMemcpyDeviceToDevice, ctx.stream));
}

template <class C>
void schur_solve(qd_ctx& ctx, const qd_gauge& g, const C* links, double m0, double tau, SchurPrecond<C>* pre,
                 GCR<C>& gcr, DevBuf& scratch, const C* b, C* x, int nrhs, double tol, int maxit, int restart,
                 SolveInfo* info) {
  QD_REQUIRE(g.geo.eo, "even-odd solve on a lattice without even-odd ordering");
  const int64_t Vh = g.geo.nsites / 2;
  const int64_t hn = Vh * 12 * (int64_t)nrhs;
  scratch.resize((size_t)2 * hn * sizeof(C));
  C* u = scratch.as<C>();
  C* bh = u + hn;
  cplx M[2], Minv[2];
  diag_m(m0, tau, M, Minv);
  const cplx one[2] = {mkc(1.0, 0.0), mkc(1.0, 0.0)};
  const cplx half2[2] = {mkc(0.5, 0.0), mkc(0.5, 0.0)};
  const cplx halfMinv[2] = {mkc(0.5 * Minv[0].x, 0.5 * Minv[0].y), mkc(0.5 * Minv[1].x, 0.5 * Minv[1].y)};
  // b_o' = b_o + (1/2) H_oe M^{-1} b_e
  spin_diag<C>(ctx, Vh, nrhs, Minv, b, u);
  wilson_eo<C>(ctx, g.geo, links, 1, one, half2, u, b + hn, bh, nrhs);
  SchurOp<C> S(&g, links, m0, tau);
  // the GCR's residual and directions as odd halves of full fields: the
  // preconditioner runs the V-cycle on them in place
  gcr.embed = hn;
  if (pre) pre->embedded = gcr.embeds(restart);
  gcr.solve(ctx, S, pre, bh, x + hn, nrhs, tol, maxit, restart, info);
  if (pre) pre->embedded = false;
  // x_e = M^{-1} b_e + (1/2) M^{-1} H_eo x_o
  wilson_eo<C>(ctx, g.geo, links, 0, Minv, halfMinv, x + hn, b, x, nrhs);
}

template struct SchurOp<cplx>;
template struct SchurOp<cplxf>;
template class SchurPrecond<cplx>;
template class SchurPrecond<cplxf>;
template void schur_solve<cplx>(qd_ctx&, const qd_gauge&, const cplx*, double, double, SchurPrecond<cplx>*,
                                GCR<cplx>&, DevBuf&, const cplx*, cplx*, int, double, int, int, SolveInfo*);
template void schur_solve<cplxf>(qd_ctx&, const qd_gauge&, const cplxf*, double, double, SchurPrecond<cplxf>*,
                                 GCR<cplxf>&, DevBuf&, const cplxf*, cplxf*, int, double, int, int, SolveInfo*);

}  // namespace qd

// ---------------------------------------------------------------------------
// qd_mg helpers
// ---------------------------------------------------------------------------
template <>
std::unique_ptr<qd::Op<qd::cplx>> qd_mg::op<qd::cplx>(int level) {
  if (level == 0)
    return std::unique_ptr<qd::Op<qd::cplx>>(
        new qd::WilsonOp<qd::cplx>(gauge, gauge->links.as<qd::cplx>(), m0, tau, false));
  return std::unique_ptr<qd::Op<qd::cplx>>(new qd::CoarseOp<qd::cplx>(L[level - 1].get(), L[level - 1]->Cm.as<qd::cplx>()));
}

template <>
std::unique_ptr<qd::Op<qd::cplxf>> qd_mg::op<qd::cplxf>(int level) {
  if (level == 0)
    return std::unique_ptr<qd::Op<qd::cplxf>>(
        new qd::WilsonOp<qd::cplxf>(gauge, const_cast<qd_gauge*>(gauge)->links_f32(), m0, tau, false));
  qd::CoarseLevel& lv = *L[level - 1];
  if (lv.Cmf.bytes() == 0) {
    const int64_t n = lv.geo.nsites * 9 * (int64_t)lv.D * lv.D;
    lv.Cmf.resize(n * sizeof(qd::cplxf));
    qd::to_f32(*ctx, lv.Cm.as<qd::cplx>(), lv.Cmf.as<qd::cplxf>(), n);
  }
  return std::unique_ptr<qd::Op<qd::cplxf>>(new qd::CoarseOp<qd::cplxf>(&lv, lv.Cmf.as<qd::cplxf>()));
}

template <> const qd::cplx* qd_mg::W<qd::cplx>(int level) { return T[level]->W.as<qd::cplx>(); }
template <> const qd::cplxf* qd_mg::W<qd::cplxf>(int level) {
  qd::Transfer& t = *T[level];
  if (t.Wf.bytes() == 0) {
    const int64_t n = t.nfine * t.Df * (int64_t)t.nv;
    t.Wf.resize(n * sizeof(qd::cplxf));
    qd::to_f32(*ctx, t.W.as<qd::cplx>(), t.Wf.as<qd::cplxf>(), n);
  }
  return t.Wf.as<qd::cplxf>();
}

template <> const qd::cplx* qd_mg::Cinv<qd::cplx>(int level) {
  const qd::CoarseLevel& lv = *L[level - 1];
  return lv.ndense > 0 ? lv.Cinv.as<qd::cplx>() : nullptr;
}
template <> const qd::cplxf* qd_mg::Cinv<qd::cplxf>(int level) {
  qd::CoarseLevel& lv = *L[level - 1];
  if (lv.ndense <= 0) return nullptr;
  if (lv.Cinvf.bytes() == 0) {
    const int64_t n = (int64_t)lv.ndense * lv.ndense;
    lv.Cinvf.resize(n * sizeof(qd::cplxf));
    qd::to_f32(*ctx, lv.Cinv.as<qd::cplx>(), lv.Cinvf.as<qd::cplxf>(), n);
  }
  return lv.Cinvf.as<qd::cplxf>();
}
