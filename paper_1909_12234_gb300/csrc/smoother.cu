// Learned gauge-covariant smoother of the fine level (an extension of the
// V-cycle's smoothing step; the paper has no counterpart).
//
//   (S r)(x)_{o,a} = sum_{d=0..8} sum_{i=0..3} w[d][o][i] (T_d r)(x)_{i,a}
//
// with T_0 the identity, T_{1+mu} r(x) = U_mu(x) r(x+mu) and
// T_{5+mu} r(x) = U_mu(x-mu)^H r(x-mu): one linear layer of link-transported
// one-hop terms, 144 complex weights.  Colour is moved only by links, so S
// is gauge covariant.  Training fits w to pairs (e, r) that the solver
// generates - r the residual left by the coarse-grid correction of a random
// vector, e = A^{-1} r its error - by linear least squares (normal
// equations of the 36 transported features per output spin, solved by a
// Cholesky factorisation on the host).  A held-out set judges the result
// against the plain minimal-residual smoother; the V-cycle uses S only when
// it wins.  The FP32 V-cycle applies the weights rounded to FP16.
#include <cuda_fp16.h>

#include <cmath>

#include "blas.cuh"
#include "dense.cuh"
#include "defl.cuh"
#include "mg.cuh"
#include "tune.cuh"

namespace qd {

// Transport of the 4 colour triplets of `in` at site y through link matrix
// L (ADJ: L^H), into t[4][3].
template <bool ADJ, class C>
__device__ __forceinline__ void transport4(const C* __restrict__ L, const C* __restrict__ p, int64_t rs, C t[12]) {
  typedef typename CTraits<C>::R R;
  C l[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) l[k] = L[k];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    C v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = p[(s * 3 + c) * rs];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      C acc = mk<C>((R)0, (R)0);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (ADJ)
          cfmac(acc, l[b * 3 + a], v[b]);
        else
          cfma(acc, l[a * 3 + b], v[b]);
      }
      t[s * 3 + a] = acc;
    }
  }
}

// out (+)= S in; one thread per (site, right-hand side); weights staged in
// shared memory.
template <class C, bool ACC>
__global__ void __launch_bounds__(128) k_smoother_apply(const C* __restrict__ U, const int* __restrict__ nbr,
                                                        int64_t V, int nrhs, const C* __restrict__ w,
                                                        const C* __restrict__ in, C* __restrict__ out) {
  typedef typename CTraits<C>::R R;
  __shared__ C sw[144];
  for (int k = threadIdx.x; k < 144; k += blockDim.x) sw[k] = w[k];
  __syncthreads();
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= V * nrhs) return;
  const int64_t site = g / nrhs;
  const int r = (int)(g - site * nrhs);
  const int64_t rs = nrhs;
  C acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = mk<C>((R)0, (R)0);
  for (int d = 0; d < 9; ++d) {
    C t[12];
    if (d == 0) {
      const C* p = in + site * 12 * rs + r;
#pragma unroll
      for (int k = 0; k < 12; ++k) t[k] = p[k * rs];
    } else if (d <= 4) {
      const int mu = d - 1;
      const int64_t y = nbr[site * 8 + mu];
      transport4<false>(U + ((int64_t)mu * V + site) * 9, in + y * 12 * rs + r, rs, t);
    } else {
      const int mu = d - 5;
      const int64_t y = nbr[site * 8 + 4 + mu];
      transport4<true>(U + ((int64_t)mu * V + y) * 9, in + y * 12 * rs + r, rs, t);
    }
    const C* wd = sw + d * 16;
#pragma unroll
    for (int o = 0; o < 4; ++o)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const C c = wd[o * 4 + i];
#pragma unroll
        for (int a = 0; a < 3; ++a) cfma(acc[o * 3 + a], c, t[i * 3 + a]);
      }
  }
  C* y = out + site * 12 * rs + r;
#pragma unroll
  for (int k = 0; k < 12; ++k) y[k * rs] = ACC ? cadd(y[k * rs], acc[k]) : acc[k];
}

// FP32, two right-hand sides per thread: each colour component of the two is
// one 16-byte load and each link is loaded once for both (even nrhs, 16-byte
// aligned fields; the launcher checks).
template <bool ADJ>
__device__ __forceinline__ void transport4x2(const float2* __restrict__ L, const float2* __restrict__ p, int64_t rs,
                                             float2 t[2][12]) {
  float2 l[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) l[k] = L[k];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    float4 v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = *reinterpret_cast<const float4*>(p + (s * 3 + c) * rs);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float2 x0 = make_float2(v[b].x, v[b].y), x1 = make_float2(v[b].z, v[b].w);
        if (ADJ) {
          cfmac(a0, l[b * 3 + a], x0);
          cfmac(a1, l[b * 3 + a], x1);
        } else {
          cfma(a0, l[a * 3 + b], x0);
          cfma(a1, l[a * 3 + b], x1);
        }
      }
      t[0][s * 3 + a] = a0;
      t[1][s * 3 + a] = a1;
    }
  }
}

// Sites are taken in the stencil visiting order (visit: 4^4 tiles, Morton
// inside; nullptr: index order) and the columns in chunks of 2 rc2,
// chunk-major, so that the neighbour fields a traversal keeps in flight fit
// in L2 (the same traversal as the Wilson stencil).
template <bool ACC>
__global__ void __launch_bounds__(128, 4) k_smoother_apply_x2(const float2* __restrict__ U, const int* __restrict__ nbr,
                                                              const int* __restrict__ visit, int64_t V, int nrhs,
                                                              int rc2, const float2* __restrict__ w,
                                                              const float2* __restrict__ in, float2* __restrict__ out) {
  __shared__ float2 sw[144];
  for (int k = threadIdx.x; k < 144; k += blockDim.x) sw[k] = w[k];
  __syncthreads();
  const int half = nrhs >> 1;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= V * half) return;
  const int64_t per_chunk = V * rc2;
  const int ch = (int)(g / per_chunk);
  const int64_t rem = g - ch * per_chunk;
  const int64_t slot = rem / rc2;
  const int r0 = 2 * (ch * rc2 + (int)(rem - slot * rc2));
  const int64_t site = visit ? visit[slot] : slot;
  const int64_t rs = nrhs;
  float2 acc[2][12];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[j][k] = make_float2(0.f, 0.f);
  for (int d = 0; d < 9; ++d) {
    float2 t[2][12];
    if (d == 0) {
      const float2* p = in + site * 12 * rs + r0;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const float4 q = *reinterpret_cast<const float4*>(p + k * rs);
        t[0][k] = make_float2(q.x, q.y);
        t[1][k] = make_float2(q.z, q.w);
      }
    } else if (d <= 4) {
      const int mu = d - 1;
      const int64_t y = nbr[site * 8 + mu];
      transport4x2<false>(U + ((int64_t)mu * V + site) * 9, in + y * 12 * rs + r0, rs, t);
    } else {
      const int mu = d - 5;
      const int64_t y = nbr[site * 8 + 4 + mu];
      transport4x2<true>(U + ((int64_t)mu * V + y) * 9, in + y * 12 * rs + r0, rs, t);
    }
    const float2* wd = sw + d * 16;
#pragma unroll
    for (int o = 0; o < 4; ++o)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 c = wd[o * 4 + i];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          cfma(acc[0][o * 3 + a], c, t[0][i * 3 + a]);
          cfma(acc[1][o * 3 + a], c, t[1][i * 3 + a]);
        }
      }
  }
  float2* y = out + site * 12 * rs + r0;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    float4 v = make_float4(acc[0][k].x, acc[0][k].y, acc[1][k].x, acc[1][k].y);
    if (ACC) {
      const float4 o = *reinterpret_cast<const float4*>(y + k * rs);
      v = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
    }
    *reinterpret_cast<float4*>(y + k * rs) = v;
  }
}

// Packed-FP32 form of k_smoother_apply_x2 (fma.rn.f32x2: one instruction
// for two FP32 multiply-adds).  A complex value is one 64-bit pair (re, im);
// acc += c t is fma2((c.x, c.x), (t.x, t.y), fma2((-c.y, c.y), (t.y, t.x),
// acc)) and acc += conj(l) x is fma2((l.x, l.x), (x.x, x.y), fma2((l.y,
// -l.y), (x.y, x.x), acc)): lane by lane the same multiply-adds in the same
// order as cfma / cfmac, so the results are bit-identical to the unpacked
// kernel.  The weights are staged in shared memory already packed.
typedef unsigned long long u64;
__device__ __forceinline__ u64 pk2(float lo, float hi) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 upk2(u64 v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ u64 swap2(u64 v) {
  const float2 f = upk2(v);
  return pk2(f.y, f.x);
}

template <bool ADJ>
__device__ __forceinline__ void transport4p(const float2* __restrict__ L, const float2* __restrict__ p, int64_t rs,
                                            u64 t[2][12]) {
  float2 l[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) l[k] = L[k];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    u64 x[2][3], xs[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float4 v = *reinterpret_cast<const float4*>(p + (s * 3 + c) * rs);
      x[0][c] = pk2(v.x, v.y);
      xs[0][c] = pk2(v.y, v.x);
      x[1][c] = pk2(v.z, v.w);
      xs[1][c] = pk2(v.w, v.z);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      u64 a0 = 0ull, a1 = 0ull;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float2 lv = ADJ ? l[b * 3 + a] : l[a * 3 + b];
        const u64 lxx = pk2(lv.x, lv.x);
        const u64 ly = ADJ ? pk2(lv.y, -lv.y) : pk2(-lv.y, lv.y);
        a0 = fma2(lxx, x[0][b], fma2(ly, xs[0][b], a0));
        a1 = fma2(lxx, x[1][b], fma2(ly, xs[1][b], a1));
      }
      t[0][s * 3 + a] = a0;
      t[1][s * 3 + a] = a1;
    }
  }
}

template <bool ACC>
__global__ void __launch_bounds__(128, 4) k_smoother_apply_p2(const float2* __restrict__ U, const int* __restrict__ nbr,
                                                              const int* __restrict__ visit, int64_t V, int nrhs,
                                                              int rc2, const float2* __restrict__ w,
                                                              const float2* __restrict__ in, float2* __restrict__ out) {
  __shared__ u64 sw[144][2];  // (c.x, c.x), (-c.y, c.y)
  for (int k = threadIdx.x; k < 144; k += blockDim.x) {
    const float2 c = w[k];
    sw[k][0] = pk2(c.x, c.x);
    sw[k][1] = pk2(-c.y, c.y);
  }
  __syncthreads();
  const int half = nrhs >> 1;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= V * half) return;
  const int64_t per_chunk = V * rc2;
  const int ch = (int)(g / per_chunk);
  const int64_t rem = g - ch * per_chunk;
  const int64_t slot = rem / rc2;
  const int r0 = 2 * (ch * rc2 + (int)(rem - slot * rc2));
  const int64_t site = visit ? visit[slot] : slot;
  const int64_t rs = nrhs;
  u64 acc[2][12];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[j][k] = 0ull;
  for (int d = 0; d < 9; ++d) {
    u64 t[2][12];
    if (d == 0) {
      const float2* p = in + site * 12 * rs + r0;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const float4 q = *reinterpret_cast<const float4*>(p + k * rs);
        t[0][k] = pk2(q.x, q.y);
        t[1][k] = pk2(q.z, q.w);
      }
    } else if (d <= 4) {
      const int mu = d - 1;
      const int64_t y = nbr[site * 8 + mu];
      transport4p<false>(U + ((int64_t)mu * V + site) * 9, in + y * 12 * rs + r0, rs, t);
    } else {
      const int mu = d - 5;
      const int64_t y = nbr[site * 8 + 4 + mu];
      transport4p<true>(U + ((int64_t)mu * V + y) * 9, in + y * 12 * rs + r0, rs, t);
    }
    // spin mixing, i outer: each accumulator still takes its i terms in order
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      u64 ts[2][3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        ts[0][a] = swap2(t[0][i * 3 + a]);
        ts[1][a] = swap2(t[1][i * 3 + a]);
      }
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const u64 cxx = sw[d * 16 + o * 4 + i][0], cny = sw[d * 16 + o * 4 + i][1];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          acc[0][o * 3 + a] = fma2(cxx, t[0][i * 3 + a], fma2(cny, ts[0][a], acc[0][o * 3 + a]));
          acc[1][o * 3 + a] = fma2(cxx, t[1][i * 3 + a], fma2(cny, ts[1][a], acc[1][o * 3 + a]));
        }
      }
    }
  }
  float2* y = out + site * 12 * rs + r0;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const float2 a0 = upk2(acc[0][k]), a1 = upk2(acc[1][k]);
    float4 v = make_float4(a0.x, a0.y, a1.x, a1.y);
    if (ACC) {
      const float4 o = *reinterpret_cast<const float4*>(y + k * rs);
      v = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
    }
    *reinterpret_cast<float4*>(y + k * rs) = v;
  }
}

// out (+)= S_l in for one layer with device weights w.
template <class C>
static void apply_layer(qd_ctx& ctx, const qd_mg& mg, int nrhs, const C* w, const C* in, C* out, bool accumulate) {
  const LevelGeom& geo = mg.gauge->geo;
  const int64_t tot = geo.nsites * nrhs;
  const C* links;
  if (sizeof(C) == 16)
    links = reinterpret_cast<const C*>(mg.gauge->links.as<cplx>());
  else
    links = reinterpret_cast<const C*>(const_cast<qd_gauge*>(mg.gauge)->links_f32());
  const double cb = (double)sizeof(C);
  ProfScope ps(ctx, sizeof(C) == 16 ? QD_PROF_SMOOTHER_F64 : QD_PROF_SMOOTHER_F32,
               (9.0 * 36 + 9.0 * 48) * 8.0 * (double)tot,
               (double)geo.nsites * ((accumulate ? 36.0 : 24.0) * cb * nrhs + 36.0 * cb));
  if (sizeof(C) == 8 && (nrhs % 2) == 0 &&
      ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0) {
    const int blocks2 = div_up(geo.nsites * (nrhs / 2), 128);
    const float2* L = reinterpret_cast<const float2*>(links);
    const float2* W2 = reinterpret_cast<const float2*>(w);
    const float2* xi = reinterpret_cast<const float2*>(in);
    float2* yo = reinterpret_cast<float2*>(out);
    // candidates: two right-hand sides per thread in index order (0), in the
    // stencil visiting order with the columns swept whole (1), in chunks of
    // 64 (2) or 32 (3), and the packed-FP32 form in the visiting order (4).
    // All bit-identical.  Accumulating launches are not timed by the tuner
    // (they change out): they take the choice timed on the plain form.
    const int* vis = geo.visit.as<int>();
    auto shape = [&](int c, int& rc, const int*& vv) -> bool {
      rc = c == 2 ? 64 : (c == 3 ? 32 : nrhs);
      vv = c == 0 ? nullptr : vis;
      if (rc > nrhs || nrhs % rc != 0 || rc % 2 != 0) return false;
      if ((c == 2 && nrhs <= 64) || (c == 3 && nrhs <= 32)) return false;
      return true;
    };
    auto launch_into = [&](int c, bool acc, float2* dst) -> bool {
      int rc;
      const int* vv;
      if (!shape(c, rc, vv)) return false;
      const int h = rc / 2;
      if (c == 4) {
        if (acc)
          k_smoother_apply_p2<true><<<blocks2, 128, 0, ctx.stream>>>(L, geo.nbr.as<int>(), vv, geo.nsites, nrhs, h, W2,
                                                                     xi, dst);
        else
          k_smoother_apply_p2<false><<<blocks2, 128, 0, ctx.stream>>>(L, geo.nbr.as<int>(), vv, geo.nsites, nrhs, h, W2,
                                                                      xi, dst);
      } else {
        if (acc)
          k_smoother_apply_x2<true><<<blocks2, 128, 0, ctx.stream>>>(L, geo.nbr.as<int>(), vv, geo.nsites, nrhs, h, W2,
                                                                     xi, dst);
        else
          k_smoother_apply_x2<false><<<blocks2, 128, 0, ctx.stream>>>(L, geo.nbr.as<int>(), vv, geo.nsites, nrhs, h, W2,
                                                                      xi, dst);
      }
      QD_LAUNCH_CHECK();
      return true;
    };
    auto launch = [&](int c) -> bool { return launch_into(c, accumulate, yo); };
    const std::string key = "smoother f32 sites" + std::to_string(geo.nsites) + " rhs" + std::to_string(nrhs);
    int c = tune_lookup(key);
    if (c < 0 && tune_can_time(ctx)) {
      // time the non-accumulating form into scratch (the candidates then
      // neither change out nor read it), released afterwards
      DevBuf& scr = mg.ls->tune_scratch;
      scr.resize((size_t)tot * 12 * sizeof(C));
      float2* so = scr.as<float2>();
      c = tune_pick(ctx, key, 5, [&](int cc) { return launch_into(cc, false, so); });
      QD_CUDA(cudaStreamSynchronize(ctx.stream));
      scr.release();
    }
    if (c < 0 || !launch(c)) launch(1);
    return;
  }
  const int blocks = div_up(tot, 128);
  if (accumulate)
    k_smoother_apply<C, true><<<blocks, 128, 0, ctx.stream>>>(links, geo.nbr.as<int>(), geo.nsites, nrhs, w, in, out);
  else
    k_smoother_apply<C, false><<<blocks, 128, 0, ctx.stream>>>(links, geo.nbr.as<int>(), geo.nsites, nrhs, w, in, out);
  QD_LAUNCH_CHECK();
}

template <class C>
void smoother_apply(qd_ctx& ctx, qd_mg& mg, int nrhs, const C* in, C* out, bool accumulate) {
  const LearnedSmoother& ls = *mg.ls;
  const LevelGeom& geo = mg.gauge->geo;
  const int64_t tot = geo.nsites * nrhs;
  if (tot == 0) return;
  const C* w = sizeof(C) == 16 ? ls.w64.as<C>() : ls.w32.as<C>();
  // S_L ... S_1 in: the intermediate fields alternate between two buffers
  const C* src = in;
  for (int l = 0; l < ls.layers; ++l) {
    const bool last = l == ls.layers - 1;
    C* dst = out;
    if (!last) {
      DevBuf& tb = ls.t[l & 1];
      tb.resize((size_t)tot * 12 * sizeof(C));
      dst = tb.as<C>();
    }
    apply_layer<C>(ctx, mg, nrhs, w + (size_t)144 * l, src, dst, last && accumulate);
    src = dst;
  }
}
template void smoother_apply<cplx>(qd_ctx&, qd_mg&, int, const cplx*, cplx*, bool);
template void smoother_apply<cplxf>(qd_ctx&, qd_mg&, int, const cplxf*, cplxf*, bool);

// ---------------------------------------------------------------------------
// Training
// ---------------------------------------------------------------------------

// F[((x * 3 + a) * s + j) * 36 + d * 4 + i] = (T_d r_j)(x)_{i,a} and
// E[((x * 3 + a) * s + j) * 4 + o] = e_j(x)_{o,a}; one thread per (x, j).
__global__ void k_smoother_features(const cplx* __restrict__ U, const int* __restrict__ nbr, int64_t V, int s,
                                    const cplx* __restrict__ r, const cplx* __restrict__ e, cplx* __restrict__ F,
                                    cplx* __restrict__ E) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= V * s) return;
  const int64_t x = g / s;
  const int j = (int)(g - x * s);
  const int64_t rs = s;
  for (int d = 0; d < 9; ++d) {
    cplx t[12];
    if (d == 0) {
      const cplx* p = r + x * 12 * rs + j;
      for (int k = 0; k < 12; ++k) t[k] = p[k * rs];
    } else if (d <= 4) {
      const int mu = d - 1;
      const int64_t y = nbr[x * 8 + mu];
      transport4<false>(U + ((int64_t)mu * V + x) * 9, r + y * 12 * rs + j, rs, t);
    } else {
      const int mu = d - 5;
      const int64_t y = nbr[x * 8 + 4 + mu];
      transport4<true>(U + ((int64_t)mu * V + y) * 9, r + y * 12 * rs + j, rs, t);
    }
    for (int a = 0; a < 3; ++a) {
      cplx* row = F + ((x * 3 + a) * s + j) * 36 + d * 4;
      for (int i = 0; i < 4; ++i) row[i] = t[i * 3 + a];
    }
  }
  for (int a = 0; a < 3; ++a)
    for (int o = 0; o < 4; ++o) E[((x * 3 + a) * s + j) * 4 + o] = e[x * 12 * rs + (o * 3 + a) * rs + j];
}

// Cholesky solve of the Hermitian positive definite G (n x n) for the
// columns of H (n x m), on the host in double precision.
static void chol_solve(int n, int m, std::vector<cplx>& G, std::vector<cplx>& H) {
  // small ridge relative to the mean diagonal keeps rank-deficient feature
  // sets (e.g. a field with a vanishing component) solvable
  double tr = 0.0;
  for (int i = 0; i < n; ++i) tr += G[(size_t)i * n + i].x;
  const double ridge = 1e-13 * tr / n;
  for (int i = 0; i < n; ++i) G[(size_t)i * n + i].x += ridge;
  // G = L L^H, L lower triangular stored in G
  for (int j = 0; j < n; ++j) {
    double djj = G[(size_t)j * n + j].x;
    for (int k = 0; k < j; ++k) djj -= cnorm2(G[(size_t)j * n + k]);
    QD_REQUIRE(djj > 0.0, "learned-smoother normal equations are not positive definite");
    const double ljj = std::sqrt(djj);
    G[(size_t)j * n + j] = mkc(ljj, 0.0);
    for (int i = j + 1; i < n; ++i) {
      cplx v = G[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) {
        const cplx a = G[(size_t)i * n + k], b = G[(size_t)j * n + k];
        // v -= a conj(b)
        v.x -= a.x * b.x + a.y * b.y;
        v.y -= a.y * b.x - a.x * b.y;
      }
      G[(size_t)i * n + j] = mkc(v.x / ljj, v.y / ljj);
    }
  }
  for (int c = 0; c < m; ++c) {
    // L y = h
    for (int i = 0; i < n; ++i) {
      cplx v = H[(size_t)i * m + c];
      for (int k = 0; k < i; ++k) {
        const cplx a = G[(size_t)i * n + k], b = H[(size_t)k * m + c];
        v.x -= a.x * b.x - a.y * b.y;
        v.y -= a.x * b.y + a.y * b.x;
      }
      const double l = G[(size_t)i * n + i].x;
      H[(size_t)i * m + c] = mkc(v.x / l, v.y / l);
    }
    // L^H w = y
    for (int i = n - 1; i >= 0; --i) {
      cplx v = H[(size_t)i * m + c];
      for (int k = i + 1; k < n; ++k) {
        const cplx a = G[(size_t)k * n + i], b = H[(size_t)k * m + c];  // conj(a) b
        v.x -= a.x * b.x + a.y * b.y;
        v.y -= a.x * b.y - a.y * b.x;
      }
      const double l = G[(size_t)i * n + i].x;
      H[(size_t)i * m + c] = mkc(v.x / l, v.y / l);
    }
  }
}

static void upload_weights(qd_ctx& ctx, LearnedSmoother& ls) {
  const size_t nw = (size_t)144 * ls.layers;
  ls.w64.resize(nw * sizeof(cplx));
  ls.w32.resize(nw * sizeof(cplxf));
  std::vector<cplxf> h(nw);
  for (size_t k = 0; k < nw; ++k)
    h[k] = make_float2(__half2float(__float2half_rn((float)ls.w[k].x)), __half2float(__float2half_rn((float)ls.w[k].y)));
  QD_CUDA(cudaMemcpyAsync(ls.w64.as<cplx>(), ls.w.data(), nw * sizeof(cplx), cudaMemcpyHostToDevice, ctx.stream));
  QD_CUDA(cudaMemcpyAsync(ls.w32.as<cplxf>(), h.data(), nw * sizeof(cplxf), cudaMemcpyHostToDevice, ctx.stream));
  QD_CUDA(cudaStreamSynchronize(ctx.stream));
}

void smoother_set_layers(qd_mg& mg, int layers, const cplx* w) {
  QD_REQUIRE(layers >= 1 && layers <= 4, "layers must be in [1, 4]");
  if (!mg.ls) mg.ls.reset(new LearnedSmoother());
  mg.ls->layers = layers;
  mg.ls->w.assign(w, w + (size_t)144 * layers);
  upload_weights(*mg.ctx, *mg.ls);
}

void smoother_set_weights(qd_mg& mg, const cplx* w) { smoother_set_layers(mg, 1, w); }

// Least-squares weights of one layer for s pairs (e, r) in fine qd layout
// (device): e ~ S r.
static std::vector<cplx> fit_layer(qd_mg& mg, int s, const cplx* e, const cplx* r) {
  qd_ctx& ctx = *mg.ctx;
  const LevelGeom& geo = mg.gauge->geo;
  const int64_t rows = geo.nsites * 3 * (int64_t)s;
  DevBuf F((size_t)rows * 36 * sizeof(cplx)), E((size_t)rows * 4 * sizeof(cplx)), G(36 * 36 * sizeof(cplx)),
      H(36 * 4 * sizeof(cplx));
  k_smoother_features<<<div_up(geo.nsites * s, 128), 128, 0, ctx.stream>>>(
      mg.gauge->links.as<cplx>(), geo.nbr.as<int>(), geo.nsites, s, r, e, F.as<cplx>(), E.as<cplx>());
  QD_LAUNCH_CHECK();
  blockdot(ctx, rows, F.as<cplx>(), 36, 36, F.as<cplx>(), 36, 36, G.as<cplx>());
  blockdot(ctx, rows, F.as<cplx>(), 36, 36, E.as<cplx>(), 4, 4, H.as<cplx>());
  std::vector<cplx> hG(36 * 36), hH(36 * 4);
  QD_CUDA(cudaMemcpyAsync(hG.data(), G.as<cplx>(), hG.size() * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaMemcpyAsync(hH.data(), H.as<cplx>(), hH.size() * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaStreamSynchronize(ctx.stream));
  chol_solve(36, 4, hG, hH);
  std::vector<cplx> w(144);
  for (int d = 0; d < 9; ++d)
    for (int o = 0; o < 4; ++o)
      for (int i = 0; i < 4; ++i) w[(d * 4 + o) * 4 + i] = hH[(size_t)(d * 4 + i) * 4 + o];
  return w;
}

void smoother_fit(qd_mg& mg, int s, const cplx* e, const cplx* r) {
  const std::vector<cplx> w = fit_layer(mg, s, e, r);
  smoother_set_weights(mg, w.data());
}

// Pairs the solver generates: r = residual of the coarse-grid correction of
// a random vector, e = A^{-1} r solved to solve_tol.
static void make_pairs(qd_mg& mg, int s, uint64_t key, double solve_tol, DevBuf& e, DevBuf& r) {
  qd_ctx& ctx = *mg.ctx;
  const LevelGeom& geo = mg.gauge->geo;
  const int64_t tot = geo.nsites * 12 * (int64_t)s;
  DevBuf v((size_t)tot * sizeof(cplx)), z((size_t)tot * sizeof(cplx));
  e.resize((size_t)tot * sizeof(cplx));
  r.resize((size_t)tot * sizeof(cplx));
  random_starts_fill(ctx, geo, 12, key, s, v.as<cplx>());
  mg.pre64->coarse_correction(ctx, v.as<cplx>(), z.as<cplx>(), s);
  auto A = mg.op<cplx>(0);
  A->residual(ctx, v.as<cplx>(), z.as<cplx>(), r.as<cplx>(), s);
  // e = A^{-1} r to solve_tol on the FP64 residual: FP32 GCR corrections with
  // the FP32 V-cycle inside FP64 refinement (the pairs need no more than the
  // tolerance, and the FP64 V-cycle's dense coarsest product is slow here)
  qd_solver_params sp{};
  sp.tol = solve_tol;
  sp.maxit = 2000;
  sp.restart = 16;
  sp.precision = QD_PREC_MIXED;
  sp.inner_tol = 1e-5;
  sp.max_refine = 20;
  SolveInfo info;
  solve(ctx, *mg.gauge, &mg, mg.m0, mg.tau, s, r.as<cplx>(), e.as<cplx>(), sp, info);
  QD_REQUIRE(info.converged == s, "learned-smoother training solves did not converge");
}

// Mean over columns of ||e - x|| / ||e||.
static double mean_rel_err(qd_ctx& ctx, int64_t n, int s, const cplx* e, const cplx* x) {
  DevBuf d((size_t)n * s * sizeof(cplx)), nn(2 * (size_t)s * sizeof(cplx));
  blas::sub(ctx, n * s, e, x, d.as<cplx>());
  blas::dots(ctx, 1, n, s, d.as<cplx>(), 0, d.as<cplx>(), 0, nn.as<cplx>());
  blas::dots(ctx, 1, n, s, e, 0, e, 0, nn.as<cplx>() + s);
  std::vector<cplx> h(2 * s);
  QD_CUDA(cudaMemcpyAsync(h.data(), nn.as<cplx>(), h.size() * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaStreamSynchronize(ctx.stream));
  double m = 0.0;
  for (int j = 0; j < s; ++j) m += std::sqrt(h[j].x / (h[s + j].x > 0.0 ? h[s + j].x : 1.0));
  return m / s;
}

void smoother_train(qd_mg& mg, int s, double solve_tol, uint64_t seed, int mr_steps, int layers, double* err_learned,
                    double* err_plain, int* enabled) {
  QD_REQUIRE(s >= 1 && s <= 1024, "nsamples must be in [1, 1024]");
  QD_REQUIRE(mr_steps >= 0 && mr_steps <= 64, "mr_steps must be in [0, 64]");
  QD_REQUIRE(layers >= 1 && layers <= 4, "layers must be in [1, 4]");
  qd_ctx& ctx = *mg.ctx;
  const LevelGeom& geo = mg.gauge->geo;
  const int64_t n = geo.nsites * 12;
  DevBuf e, r;
  make_pairs(mg, s, seed, solve_tol, e, r);
  // layer by layer: S_1 fits e ~ S_1 r, then S_l fits e ~ S_l (S_{l-1} ... S_1 r)
  // with the layers below fixed (each layer's family holds the identity, so
  // the training error cannot grow with depth)
  std::vector<cplx> all = fit_layer(mg, s, e.as<cplx>(), r.as<cplx>());
  smoother_set_layers(mg, 1, all.data());
  if (layers > 1) {
    DevBuf rl((size_t)n * s * sizeof(cplx));
    for (int l = 2; l <= layers; ++l) {
      smoother_apply<cplx>(ctx, mg, s, r.as<cplx>(), rl.as<cplx>(), false);
      const std::vector<cplx> wl = fit_layer(mg, s, e.as<cplx>(), rl.as<cplx>());
      all.insert(all.end(), wl.begin(), wl.end());
      smoother_set_layers(mg, l, all.data());
    }
  }
  LearnedSmoother& ls = *mg.ls;
  ls.mr_steps = mr_steps;
  // held-out pairs: the whole smoothing step of each kind, from x = 0
  DevBuf he, hr;
  make_pairs(mg, s, seed + 0x9e3779b97f4a7c15ull, solve_tol, he, hr);
  auto A = mg.op<cplx>(0);
  DevBuf x((size_t)n * s * sizeof(cplx)), res((size_t)n * s * sizeof(cplx)), q((size_t)n * s * sizeof(cplx)), scr;
  // plain: smoother_steps minimal-residual steps
  blas::zero(ctx, n * s, x.as<cplx>());
  blas::copy(ctx, n * s, hr.as<cplx>(), res.as<cplx>());
  mr_smooth<cplx>(ctx, *A, x.as<cplx>(), res.as<cplx>(), q.as<cplx>(), s, mg.p.smoother_steps, scr);
  ls.err_plain = mean_rel_err(ctx, n, s, he.as<cplx>(), x.as<cplx>());
  // learned: S r, then its minimal-residual steps
  smoother_apply<cplx>(ctx, mg, s, hr.as<cplx>(), x.as<cplx>(), false);
  A->residual(ctx, hr.as<cplx>(), x.as<cplx>(), res.as<cplx>(), s);
  mr_smooth<cplx>(ctx, *A, x.as<cplx>(), res.as<cplx>(), q.as<cplx>(), s, mr_steps, scr);
  ls.err_learned = mean_rel_err(ctx, n, s, he.as<cplx>(), x.as<cplx>());
  ls.enabled = ls.err_learned < ls.err_plain;
  *err_learned = ls.err_learned;
  *err_plain = ls.err_plain;
  *enabled = ls.enabled ? 1 : 0;
}

}  // namespace qd
