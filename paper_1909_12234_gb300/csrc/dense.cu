// Small dense linear algebra for the deflation space (Algorithms 1 and 2):
// tall-skinny products X^H Y and X S on multi-column fields, a one-CTA
// cyclic Jacobi eigensolver for Hermitian matrices (Golub & Van Loan,
// "Matrix Computations", Sec. 8.5, with the round-robin parallel ordering),
// and a one-CTA Cholesky factorisation with triangular inverse.
#include "dense.cuh"

namespace qd {

// ---------------------------------------------------------------------------
// G[a][b] = sum_i conj(X[i][a]) Y[i][b]; X: n x ma (row stride ldx), Y: n x mb.
// 16 x 16 output tile per CTA, rows split into chunks; partials summed in
// chunk order by a second kernel.
// ---------------------------------------------------------------------------
__global__ void k_blockdot(int64_t n, const cplx* __restrict__ X, int ldx, int ma, const cplx* __restrict__ Y,
                           int ldy, int mb, int64_t rows_per_chunk, cplx* __restrict__ partials) {
  __shared__ cplx sx[16][17], sy[16][17];
  const int tx = threadIdx.x, ty = threadIdx.y;  // tx -> b, ty -> a
  const int a0 = blockIdx.y * 16, b0 = blockIdx.x * 16;
  const int64_t r0 = blockIdx.z * rows_per_chunk;
  int64_t r1 = r0 + rows_per_chunk;
  if (r1 > n) r1 = n;
  cplx acc = mkc(0, 0);
  for (int64_t i0 = r0; i0 < r1; i0 += 16) {
    // load 16 rows: thread (ty, tx) loads X[i0+ty][a0+tx] and Y[i0+ty][b0+tx]
    const int64_t i = i0 + ty;
    sx[ty][tx] = (i < r1 && a0 + tx < ma) ? X[i * ldx + a0 + tx] : mkc(0, 0);
    sy[ty][tx] = (i < r1 && b0 + tx < mb) ? Y[i * ldy + b0 + tx] : mkc(0, 0);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) cfmac(acc, sx[k][ty], sy[k][tx]);
    __syncthreads();
  }
  const int a = a0 + ty, b = b0 + tx;
  if (a < ma && b < mb) partials[((int64_t)blockIdx.z * ma + a) * mb + b] = acc;
}

__global__ void k_chunk_sum(int nchunk, int64_t m, const cplx* __restrict__ partials, cplx* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m) return;
  cplx s = mkc(0, 0);
  for (int c = 0; c < nchunk; ++c) s = cadd(s, partials[c * m + e]);
  out[e] = s;
}

void blockdot(qd_ctx& ctx, int64_t n, const cplx* X, int ldx, int ma, const cplx* Y, int ldy, int mb,
              cplx* G) {
  const int ta = div_up(ma, 16), tb = div_up(mb, 16);
  int64_t chunks = (2 * kNumSMs + ta * tb - 1) / (ta * tb);
  const int64_t max_chunks = (n + 255) / 256;
  if (chunks > max_chunks) chunks = max_chunks;
  if (chunks < 1) chunks = 1;
  int64_t rpc = (n + chunks - 1) / chunks;
  rpc = (rpc + 15) / 16 * 16;
  chunks = (n + rpc - 1) / rpc;
  if (chunks < 1) chunks = 1;
  ctx.red_partials.resize((size_t)chunks * ma * mb * sizeof(cplx));
  k_blockdot<<<dim3(tb, ta, (unsigned)chunks), dim3(16, 16), 0, ctx.stream>>>(n, X, ldx, ma, Y, ldy, mb, rpc,
                                                                            ctx.red_partials.as<cplx>());
  QD_LAUNCH_CHECK();
  const int64_t m = (int64_t)ma * mb;
  k_chunk_sum<<<div_up(m, 128), 128, 0, ctx.stream>>>((int)chunks, m, ctx.red_partials.as<cplx>(), G);
  QD_LAUNCH_CHECK();
}

// Same product with caller-provided partial-sum space of `cap` complex
// numbers (no allocation).  Uses as few row chunks as the space allows, at
// most the number blockdot() would use.  Returns false if even one chunk
// does not fit.
bool blockdot_into(qd_ctx& ctx, int64_t n, const cplx* X, int ldx, int ma, const cplx* Y, int ldy, int mb,
                   cplx* G, cplx* partials, int64_t cap) {
  const int64_t m = (int64_t)ma * mb;
  if (m > cap) return false;
  const int ta = div_up(ma, 16), tb = div_up(mb, 16);
  int64_t chunks = (2 * kNumSMs + ta * tb - 1) / (ta * tb);
  const int64_t max_chunks = (n + 255) / 256;
  if (chunks > max_chunks) chunks = max_chunks;
  if (chunks > cap / m) chunks = cap / m;
  if (chunks < 1) chunks = 1;
  int64_t rpc = (n + chunks - 1) / chunks;
  rpc = (rpc + 15) / 16 * 16;
  chunks = (n + rpc - 1) / rpc;
  if (chunks < 1) chunks = 1;
  if (chunks * m > cap) return false;
  k_blockdot<<<dim3(tb, ta, (unsigned)chunks), dim3(16, 16), 0, ctx.stream>>>(n, X, ldx, ma, Y, ldy, mb, rpc,
                                                                            partials);
  QD_LAUNCH_CHECK();
  k_chunk_sum<<<div_up(m, 128), 128, 0, ctx.stream>>>((int)chunks, m, partials, G);
  QD_LAUNCH_CHECK();
  return true;
}

// Y[i][b] = alpha sum_a X[i][a] S[a][b] + beta Y[i][b]
__global__ void k_blockmul(int64_t n, const cplx* __restrict__ X, int ldx, int ma, const cplx* __restrict__ S,
                           int lds, int mb, cplx* __restrict__ Y, int ldy, double alpha, double beta);

// Load the kernels of blockdot_into and blockmul on the current device now
// (with lazy module loading a kernel is otherwise loaded, and its module's
// memory taken, at its first launch).
void preload_projection_kernels() {
  cudaFuncAttributes a;
  QD_CUDA(cudaFuncGetAttributes(&a, reinterpret_cast<const void*>(k_blockdot)));
  QD_CUDA(cudaFuncGetAttributes(&a, reinterpret_cast<const void*>(k_chunk_sum)));
  QD_CUDA(cudaFuncGetAttributes(&a, reinterpret_cast<const void*>(k_blockmul)));
}

__global__ void k_blockmul(int64_t n, const cplx* __restrict__ X, int ldx, int ma, const cplx* __restrict__ S,
                           int lds, int mb, cplx* __restrict__ Y, int ldy, double alpha, double beta) {
  const int64_t tot = n * mb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e % mb);
    const int64_t i = e / mb;
    const cplx* x = X + i * ldx;
    cplx acc = mkc(0, 0);
    for (int a = 0; a < ma; ++a) cfma(acc, x[a], S[(int64_t)a * lds + b]);
    cplx* y = Y + i * ldy + b;
    cplx v = cscale(alpha, acc);
    if (beta != 0.0) v = cadd(v, cscale(beta, *y));
    *y = v;
  }
}

void blockmul(qd_ctx& ctx, int64_t n, const cplx* X, int ldx, int ma, const cplx* S, int lds, int mb,
              cplx* Y, int ldy, double alpha, double beta) {
  const int64_t tot = n * mb;
  int blocks = div_up(tot, 256);
  if (blocks > 32 * kNumSMs) blocks = 32 * kNumSMs;
  k_blockmul<<<blocks, 256, 0, ctx.stream>>>(n, X, ldx, ma, S, lds, mb, Y, ldy, alpha, beta);
  QD_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// Hermitian Jacobi eigensolver, one CTA.  A (m x m, row major, overwritten),
// E (m x m) receives eigenvectors as columns, w the eigenvalues (unsorted).
// Each round rotates M/2 disjoint pairs (M = m rounded up to even; indices
// >= m are idle), chosen by the round-robin schedule: position 0 fixed, the
// others cycle; pair i joins positions i and M-1-i.
// Rotation for a pair (p, q), a_pq = |a_pq| e: with D = diag(1, conj(e)) the
// pair entry becomes real and the real symmetric 2x2 rotation
// [[c, s], [-s, c]] with t = sign(z) / (|z| + sqrt(1 + z^2)),
// z = (a_qq - a_pp) / (2 |a_pq|) annihilates it.  V = D J:
//   V_pp = c, V_pq = s, V_qp = -s conj(e), V_qq = c conj(e).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_jacobi(int m, cplx* __restrict__ A, cplx* __restrict__ E,
                                                 double* __restrict__ w, int max_sweeps, double rel_tol,
                                                 int* __restrict__ sweeps_out) {
  extern __shared__ double shj[];
  const int M = (m + 1) & ~1;
  const int half = M / 2;
  int* P = reinterpret_cast<int*>(shj);
  int* Qi = P + half;
  double* cs = reinterpret_cast<double*>(Qi + half);  // c, s, er, ei per pair (2*half ints: aligned)
  double* red = cs + 4 * half;
  __shared__ double s_off, s_fro;
  const int tid = threadIdx.x, nth = blockDim.x;
  // E = I
  for (int e = tid; e < m * m; e += nth) E[e] = mkc((e / m) == (e % m) ? 1.0 : 0.0, 0.0);
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    // convergence test: off-diagonal Frobenius norm vs total
    double off = 0.0, fro = 0.0;
    for (int e = tid; e < m * m; e += nth) {
      const double v = cnorm2(A[e]);
      fro += v;
      if ((e / m) != (e % m)) off += v;
    }
    red[tid] = off;
    red[nth + tid] = fro;
    __syncthreads();
    for (int h = nth / 2; h > 0; h >>= 1) {
      if (tid < h) {
        red[tid] += red[tid + h];
        red[nth + tid] += red[nth + tid + h];
      }
      __syncthreads();
    }
    if (tid == 0) {
      s_off = red[0];
      s_fro = red[nth];
    }
    __syncthreads();
    if (s_off <= rel_tol * rel_tol * s_fro || s_off == 0.0) break;
    for (int round = 0; round < M - 1; ++round) {
      for (int i = tid; i < half; i += nth) {
        const int pa = i, pb = M - 1 - i;
        const int ia = (pa == 0) ? 0 : ((pa - 1 + round) % (M - 1)) + 1;
        const int ib = (pb == 0) ? 0 : ((pb - 1 + round) % (M - 1)) + 1;
        const int p = ia < ib ? ia : ib, q = ia < ib ? ib : ia;
        P[i] = p;
        Qi[i] = q;
        double c = 1.0, s = 0.0, er = 1.0, ei = 0.0;
        if (q < m) {
          const cplx apq = A[p * m + q];
          const double g = sqrt(cnorm2(apq));
          const double app = A[p * m + p].x, aqq = A[q * m + q].x;
          if (g > 1e-300 && g > 1e-18 * sqrt(fabs(app * aqq))) {
            er = apq.x / g;
            ei = apq.y / g;
            const double z = (aqq - app) / (2.0 * g);
            const double t = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        cs[4 * i] = c;
        cs[4 * i + 1] = s;
        cs[4 * i + 2] = er;
        cs[4 * i + 3] = ei;
      }
      __syncthreads();
      // columns: A <- A V and E <- E V
      for (int e = tid; e < half * m; e += nth) {
        const int i = e / m, k = e - i * m;
        const int p = P[i], q = Qi[i];
        if (q >= m) continue;
        const double c = cs[4 * i], s = cs[4 * i + 1];
        const cplx ec = mkc(cs[4 * i + 2], -cs[4 * i + 3]);  // conj(e)
        {
          const cplx ap = A[k * m + p], aq = A[k * m + q];
          const cplx t = cmul(ec, aq);
          A[k * m + p] = csub(cscale(c, ap), cscale(s, t));
          A[k * m + q] = cadd(cscale(s, ap), cscale(c, t));
        }
        {
          const cplx ap = E[k * m + p], aq = E[k * m + q];
          const cplx t = cmul(ec, aq);
          E[k * m + p] = csub(cscale(c, ap), cscale(s, t));
          E[k * m + q] = cadd(cscale(s, ap), cscale(c, t));
        }
      }
      __syncthreads();
      // rows: A <- V^H A
      for (int e = tid; e < half * m; e += nth) {
        const int i = e / m, k = e - i * m;
        const int p = P[i], q = Qi[i];
        if (q >= m) continue;
        const double c = cs[4 * i], s = cs[4 * i + 1];
        const cplx ev = mkc(cs[4 * i + 2], cs[4 * i + 3]);
        const cplx ap = A[p * m + k], aq = A[q * m + k];
        const cplx t = cmul(ev, aq);
        A[p * m + k] = csub(cscale(c, ap), cscale(s, t));
        A[q * m + k] = cadd(cscale(s, ap), cscale(c, t));
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < m; i += nth) w[i] = A[i * m + i].x;
  if (tid == 0 && sweeps_out) *sweeps_out = sweep;
}

void jacobi_eigh(qd_ctx& ctx, int m, cplx* A, cplx* E, double* w, int* sweeps_dev) {
  QD_REQUIRE(m >= 1 && m <= 2048, "Jacobi eigensolver size out of range");
  const int threads = 1024;
  const int half = ((m + 1) & ~1) / 2;
  const size_t smem = (size_t)(2 * half + 2) * sizeof(int) + (size_t)4 * half * sizeof(double) +
                      2 * threads * sizeof(double) + 16;
  ensure_smem_limit(reinterpret_cast<const void*>(k_jacobi), smem);
  k_jacobi<<<1, threads, smem, ctx.stream>>>(m, A, E, w, 40, 1e-15, sweeps_dev);
  QD_LAUNCH_CHECK();
}

// Sort eigenpairs by |w| ascending (stable): perm[i] = old index of the i-th.
// Then Eout[:, i] = E[:, perm[i]], wout[i] = w[perm[i]].  One thread sorts.
__global__ void k_sort_abs(int m, const double* __restrict__ w, const cplx* __restrict__ E, double* __restrict__ wout,
                           cplx* __restrict__ Eout, int* __restrict__ perm) {
  if (threadIdx.x == 0) {
    for (int i = 0; i < m; ++i) perm[i] = i;
    for (int i = 1; i < m; ++i) {  // insertion sort, stable
      const int v = perm[i];
      int j = i - 1;
      while (j >= 0 && fabs(w[perm[j]]) > fabs(w[v])) {
        perm[j + 1] = perm[j];
        --j;
      }
      perm[j + 1] = v;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int r = e / m, c = e - r * m;
    Eout[e] = E[r * m + perm[c]];
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) wout[i] = w[perm[i]];
}

void sort_by_abs(qd_ctx& ctx, int m, const double* w, const cplx* E, double* wout, cplx* Eout, int* perm) {
  k_sort_abs<<<1, 1024, 0, ctx.stream>>>(m, w, E, wout, Eout, perm);
  QD_LAUNCH_CHECK();
}

// A <- (A + A^H) / 2 for an m x m matrix
__global__ void k_hermitize(int m, cplx* A) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    const int r = e / m, c = e - r * m;
    if (r > c) continue;
    const cplx a = A[r * m + c], b = A[c * m + r];
    const cplx h = mkc(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    A[r * m + c] = h;
    A[c * m + r] = cconj(h);
  }
}
void hermitize(qd_ctx& ctx, int m, cplx* A) {
  k_hermitize<<<div_up((int64_t)m * m, 256), 256, 0, ctx.stream>>>(m, A);
  QD_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// Cholesky G = R^H R (R upper triangular) and Rinv = R^{-1}, one CTA.
// G is overwritten by R.  flag = 1 if a pivot is not positive.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_cholinv(int m, cplx* __restrict__ G, cplx* __restrict__ Rinv,
                                                  int* __restrict__ flag) {
  __shared__ double s_d;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int k = 0; k < m; ++k) {
    if (tid == 0) {
      const double d = G[k * m + k].x;
      s_d = d;
      if (!(d > 0.0) && flag) *flag = 1;
    }
    __syncthreads();
    const double d = s_d > 0.0 ? sqrt(s_d) : 1.0;
    const double inv = 1.0 / d;
    for (int j = k + tid; j < m; j += nth) G[k * m + j] = (j == k) ? mkc(d, 0.0) : cscale(inv, G[k * m + j]);
    __syncthreads();
    // trailing update: G[i][j] -= conj(R[k][i]) R[k][j], k < i <= j
    const int rem = m - k - 1;
    for (int e = tid; e < rem * rem; e += nth) {
      const int i = k + 1 + e / rem, j = k + 1 + e % rem;
      if (j < i) continue;
      G[i * m + j] = csub(G[i * m + j], cmulc(G[k * m + i], G[k * m + j]));
    }
    __syncthreads();
  }
  // zero the strict lower triangle of R
  for (int e = tid; e < m * m; e += nth)
    if ((e / m) > (e % m)) G[e] = mkc(0, 0);
  __syncthreads();
  // Rinv by back substitution, one column per thread
  for (int j = tid; j < m; j += nth) {
    for (int i = 0; i < m; ++i) Rinv[i * m + j] = mkc(0, 0);
    const cplx rjj = G[j * m + j];
    Rinv[j * m + j] = mkc(1.0 / rjj.x, 0.0);
    for (int i = j - 1; i >= 0; --i) {
      cplx s = mkc(0, 0);
      for (int l = i + 1; l <= j; ++l) cfma(s, G[i * m + l], Rinv[l * m + j]);
      const double rii = G[i * m + i].x;
      Rinv[i * m + j] = cscale(-1.0 / rii, s);
    }
  }
}

void cholesky_inverse(qd_ctx& ctx, int m, cplx* G, cplx* Rinv, int* flag_dev) {
  k_cholinv<<<1, 1024, 0, ctx.stream>>>(m, G, Rinv, flag_dev);
  QD_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// Column helpers on n x m fields (RHS-innermost, ld = m)
// ---------------------------------------------------------------------------
// rows scaled: Y[i][b] *= 1 / lambda[i]  (for a k x s coefficient block)
__global__ void k_scale_rows(int k, int s, const double* __restrict__ lam, cplx* __restrict__ Y) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * s) return;
  Y[e] = cscale(1.0 / lam[e / s], Y[e]);
}
void scale_rows_inv(qd_ctx& ctx, int k, int s, const double* lam, cplx* Y) {
  k_scale_rows<<<div_up((int64_t)k * s, 256), 256, 0, ctx.stream>>>(k, s, lam, Y);
  QD_LAUNCH_CHECK();
}

// res[b] = || HX[:, b] - theta[b] X[:, b] ||^2 (two-pass deterministic)
__global__ void k_eig_resid(int64_t n, int m, const cplx* __restrict__ HX, const cplx* __restrict__ X,
                            const double* __restrict__ theta, cplx* __restrict__ partials) {
  const int b = blockIdx.y * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (b < m) {
    const double th = theta[b];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i < n; i += (int64_t)gridDim.x * blockDim.y) {
      const cplx h = HX[i * m + b], x = X[i * m + b];
      acc += cnorm2(mkc(h.x - th * x.x, h.y - th * x.y));
    }
  }
  __shared__ double sm[256];
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  sm[t] = acc;
  __syncthreads();
  for (int h = blockDim.y / 2; h > 0; h >>= 1) {
    if (threadIdx.y < h) sm[t] += sm[t + h * blockDim.x];
    __syncthreads();
  }
  if (threadIdx.y == 0 && b < m) partials[(int64_t)blockIdx.x * m + b] = mkc(sm[threadIdx.x], 0.0);
}

void eig_residuals(qd_ctx& ctx, int64_t n, int m, const cplx* HX, const cplx* X, const double* theta,
                   cplx* out) {
  int rt = 1;
  while (rt < m && rt < 32) rt <<= 1;
  const int ry = 256 / rt;
  const int gy = div_up(m, rt);
  int gx = div_up(n, ry);
  if (gx > 4 * kNumSMs / gy) gx = 4 * kNumSMs / gy;
  if (gx < 1) gx = 1;
  ctx.red_partials.resize((size_t)gx * m * sizeof(cplx));
  k_eig_resid<<<dim3(gx, gy), dim3(rt, ry), 0, ctx.stream>>>(n, m, HX, X, theta, ctx.red_partials.as<cplx>());
  QD_LAUNCH_CHECK();
  k_chunk_sum<<<div_up(m, 128), 128, 0, ctx.stream>>>(gx, m, ctx.red_partials.as<cplx>(), out);
  QD_LAUNCH_CHECK();
}

}  // namespace qd
