// Wilson-Dirac stencil (the operator A of the paper; Sec. 2 and Sec. 3.2's
// i tau gamma5 shift), multi-RHS, one thread per (site, right-hand side).
//
//   (A x)(n) = (4 + m0 + i tau gamma5) x(n)
//              - 1/2 sum_mu [(1 - s gamma_mu) U_mu(n) x(n+mu)
//                            + (1 + s gamma_mu) U_mu(n-mu)^H x(n-mu)]
// with s = +1 for A and s = -1 (and tau -> -tau) for A^H.
//
// Spin projection in the chiral basis: gamma_mu = [[0, B], [B^H, 0]] with
// B_k = -i sigma_k (k = x, y, z) and B_t = 1, all unitary.  For a spinor
// psi = (up, lo): (1 - s gamma) psi = (-s B h, h) with h = lo - s B^H up, and
// (1 + s gamma) psi = (s B h', h') with h' = lo + s B^H up.  So each hop moves
// one half spinor h (2 spins x 3 colours) through the link: 2 SU(3) matvecs
// instead of 4.
#include <string>

#include <type_traits>

#include "ptx.cuh"
#include "qd_internal.cuh"
#include "tune.cuh"

namespace qd {

// B_mu^H applied to (u0, u1), times `sg` (+1 or -1).
template <int MU, class C>
__device__ __forceinline__ void bdag(C u0, C u1, C& o0, C& o1) {
  if (MU == 0) {        // B^H = i sigma_1
    o0 = ctimesi(u1);
    o1 = ctimesi(u0);
  } else if (MU == 1) { // B^H = [[0, 1], [-1, 0]]
    o0 = u1;
    o1 = mk<C>(-u0.x, -u0.y);
  } else if (MU == 2) { // B^H = diag(i, -i)
    o0 = ctimesi(u0);
    o1 = mk<C>(u1.y, -u1.x);
  } else {              // B^H = 1
    o0 = u0;
    o1 = u1;
  }
}

// B_mu applied to (h0, h1).
template <int MU, class C>
__device__ __forceinline__ void bmul(C h0, C h1, C& o0, C& o1) {
  if (MU == 0) {        // B = -i sigma_1
    o0 = mk<C>(h1.y, -h1.x);
    o1 = mk<C>(h0.y, -h0.x);
  } else if (MU == 1) { // B = [[0, -1], [1, 0]]
    o0 = mk<C>(-h1.x, -h1.y);
    o1 = h0;
  } else if (MU == 2) { // B = diag(-i, i)
    o0 = mk<C>(h0.y, -h0.x);
    o1 = ctimesi(h1);
  } else {
    o0 = h0;
    o1 = h1;
  }
}

// y = L x (3x3 complex, row major) or y = L^H x.
template <bool ADJ, class C>
__device__ __forceinline__ void su3mul(const C* __restrict__ L, const C x[3], C y[3]) {
  typedef typename CTraits<C>::R R;
  C l[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) l[k] = L[k];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    C acc = mk<C>((R)0, (R)0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (ADJ)
        cfmac(acc, l[b * 3 + a], x[b]);
      else
        cfma(acc, l[a * 3 + b], x[b]);
    }
    y[a] = acc;
  }
}

// One direction's forward and backward hop into the accumulators.
template <int MU, bool DAG, class C>
__device__ __forceinline__ void hop_dir(const C* __restrict__ U, const int* __restrict__ nb8,
                                        int64_t V, int64_t site, int64_t rs, int r,
                                        const C* __restrict__ in, C hu[6], C hl[6], int64_t in_off = 0) {
  const double sg = DAG ? -1.0 : 1.0;
  // forward: (1 - s gamma) U_mu(n) x(n + mu)
  {
    const int64_t nf = nb8[MU];
    const C* p = in + (nf - in_off) * 12 * rs + r;
    C h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      C b0, b1;
      bdag<MU>(p[(0 * 3 + c) * rs], p[(1 * 3 + c) * rs], b0, b1);
      const C l0 = p[(2 * 3 + c) * rs], l1 = p[(3 * 3 + c) * rs];
      if (sg > 0) { h0[c] = csub(l0, b0); h1[c] = csub(l1, b1); }
      else        { h0[c] = cadd(l0, b0); h1[c] = cadd(l1, b1); }
    }
    C g0[3], g1[3];
    const C* L = U + ((int64_t)MU * V + site) * 9;
    su3mul<false>(L, h0, g0);
    su3mul<false>(L, h1, g1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      hl[c] = cadd(hl[c], g0[c]);
      hl[3 + c] = cadd(hl[3 + c], g1[c]);
      C b0, b1;
      bmul<MU>(g0[c], g1[c], b0, b1);
      if (sg > 0) { hu[c] = csub(hu[c], b0); hu[3 + c] = csub(hu[3 + c], b1); }
      else        { hu[c] = cadd(hu[c], b0); hu[3 + c] = cadd(hu[3 + c], b1); }
    }
  }
  // backward: (1 + s gamma) U_mu(n - mu)^H x(n - mu)
  {
    const int64_t nbk = nb8[4 + MU];
    const C* p = in + (nbk - in_off) * 12 * rs + r;
    C h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      C b0, b1;
      bdag<MU>(p[(0 * 3 + c) * rs], p[(1 * 3 + c) * rs], b0, b1);
      const C l0 = p[(2 * 3 + c) * rs], l1 = p[(3 * 3 + c) * rs];
      if (sg > 0) { h0[c] = cadd(l0, b0); h1[c] = cadd(l1, b1); }
      else        { h0[c] = csub(l0, b0); h1[c] = csub(l1, b1); }
    }
    C g0[3], g1[3];
    const C* L = U + ((int64_t)MU * V + nbk) * 9;
    su3mul<true>(L, h0, g0);
    su3mul<true>(L, h1, g1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      hl[c] = cadd(hl[c], g0[c]);
      hl[3 + c] = cadd(hl[3 + c], g1[c]);
      C b0, b1;
      bmul<MU>(g0[c], g1[c], b0, b1);
      if (sg > 0) { hu[c] = cadd(hu[c], b0); hu[3 + c] = cadd(hu[3 + c], b1); }
      else        { hu[c] = csub(hu[c], b0); hu[3 + c] = csub(hu[3 + c], b1); }
    }
  }
}

// RESID: out = b - A in (the residual of A x = b) instead of out = A in.
// FP32: at most 64 registers so 8 blocks (32 warps) fit on an SM; FP64 is
// ALU-bound and keeps its registers.
template <class C, bool DAG, bool RESID>
__global__ void __launch_bounds__(128, sizeof(C) == 8 ? 8 : 1)
k_wilson(const C* __restrict__ U, const int* __restrict__ nbr, const int* __restrict__ visit, int64_t V, int nrhs,
         double mass, double tau, const C* __restrict__ in, C* __restrict__ out, const C* __restrict__ b) {
  typedef typename CTraits<C>::R R;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= V * nrhs) return;
  const int64_t slot = g / nrhs;
  const int r = (int)(g - slot * nrhs);
  const int64_t site = visit[slot];
  const int64_t rs = nrhs;
  int nb8[8];
#pragma unroll
  for (int h = 0; h < 8; ++h) nb8[h] = nbr[site * 8 + h];
  C hu[6], hl[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) { hu[k] = mk<C>((R)0, (R)0); hl[k] = mk<C>((R)0, (R)0); }
  hop_dir<0, DAG>(U, nb8, V, site, rs, r, in, hu, hl);
  hop_dir<1, DAG>(U, nb8, V, site, rs, r, in, hu, hl);
  hop_dir<2, DAG>(U, nb8, V, site, rs, r, in, hu, hl);
  hop_dir<3, DAG>(U, nb8, V, site, rs, r, in, hu, hl);
  const R te = (R)(DAG ? -tau : tau);
  const C mup = mk<C>((R)mass, te);    // upper spins: gamma5 = +1
  const C mlo = mk<C>((R)mass, -te);   // lower spins: gamma5 = -1
  const R mhalf = (R)(-0.5);
  const C* x = in + site * 12 * rs + r;
  C* y = out + site * 12 * rs + r;
  const C* bb = RESID ? b + site * 12 * rs + r : nullptr;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const C h = k < 6 ? hu[k] : hl[k - 6];
    C v = cmul(k < 6 ? mup : mlo, x[k * rs]);
    v.x = fma(mhalf, h.x, v.x);
    v.y = fma(mhalf, h.y, v.y);
    if (RESID) {
      const C bv = bb[k * rs];
      v = csub(bv, v);
    }
    y[k * rs] = v;
  }
}

// ---------------------------------------------------------------------------
// FP32, two right-hand sides per thread: every spinor component of the two
// is one 16-byte load, and each link is loaded once for both, which halves
// the load instructions per right-hand side and doubles the bytes each one
// moves.  Needs an even nrhs and 16-byte aligned fields (checked by the
// launcher, which otherwise takes the one-per-thread kernel).
// ---------------------------------------------------------------------------
template <bool ADJ>
__device__ __forceinline__ void su3mul_r(const float2 l[9], const float2 x[3], float2 y[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (ADJ)
        cfmac(acc, l[b * 3 + a], x[b]);
      else
        cfma(acc, l[a * 3 + b], x[b]);
    }
    y[a] = acc;
  }
}

// One hop (forward: FWD, via U_mu(n); backward: via U_mu(n-mu)^H) for both
// right-hand sides.  With s = +1 (A) or -1 (A^H), the projector is
// (1 + sig gamma_mu), sig = -s forward and +s backward: h = lo + sig B^H up,
// then lower += U h and upper += sig B (U h).
template <int MU, bool FWD, bool DAG>
__device__ __forceinline__ void hop2l(const float2 l[9], const float4* __restrict__ q, float2 hu[2][6],
                                      float2 hl[2][6]) {
  constexpr bool plus = (FWD == DAG);  // sig = +1 forward with DAG, backward without
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    float2 h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float4 u0 = q[0 * 3 + c], u1 = q[1 * 3 + c], w0 = q[2 * 3 + c], w1 = q[3 * 3 + c];
      const float2 a0 = j ? make_float2(u0.z, u0.w) : make_float2(u0.x, u0.y);
      const float2 a1 = j ? make_float2(u1.z, u1.w) : make_float2(u1.x, u1.y);
      const float2 l0 = j ? make_float2(w0.z, w0.w) : make_float2(w0.x, w0.y);
      const float2 l1 = j ? make_float2(w1.z, w1.w) : make_float2(w1.x, w1.y);
      float2 b0, b1;
      bdag<MU>(a0, a1, b0, b1);
      if (plus) { h0[c] = cadd(l0, b0); h1[c] = cadd(l1, b1); }
      else      { h0[c] = csub(l0, b0); h1[c] = csub(l1, b1); }
    }
    float2 g0[3], g1[3];
    su3mul_r<!FWD>(l, h0, g0);
    su3mul_r<!FWD>(l, h1, g1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      hl[j][c] = cadd(hl[j][c], g0[c]);
      hl[j][3 + c] = cadd(hl[j][3 + c], g1[c]);
      float2 b0, b1;
      bmul<MU>(g0[c], g1[c], b0, b1);
      if (plus) { hu[j][c] = cadd(hu[j][c], b0); hu[j][3 + c] = cadd(hu[j][3 + c], b1); }
      else      { hu[j][c] = csub(hu[j][c], b0); hu[j][3 + c] = csub(hu[j][3 + c], b1); }
    }
  }
}

// The same with the link read from L (the link of the hop).
template <int MU, bool FWD, bool DAG>
__device__ __forceinline__ void hop2(const float2* __restrict__ L, const float4* __restrict__ q,
                                     float2 hu[2][6], float2 hl[2][6]) {
  float2 l[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) l[k] = L[k];
  hop2l<MU, FWD, DAG>(l, q, hu, hl);
}

// The same hop with the neighbour spinor projected as it is loaded: only
// the half spinor h (both right-hand sides, 6 x 16 bytes) stays live instead
// of the 12 loaded words, which leaves registers for the next hop's loads.
template <int MU, bool FWD, bool DAG>
__device__ __forceinline__ void hop2p(const float2* __restrict__ L, const float2* __restrict__ p, int64_t rs,
                                      float2 hu[2][6], float2 hl[2][6]) {
  constexpr bool plus = (FWD == DAG);
  float4 hq[6];  // hq[c]: h0[c] of rhs 0 (xy) and 1 (zw); hq[3 + c]: h1[c]
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float4 u0 = *reinterpret_cast<const float4*>(p + (0 * 3 + c) * rs);
    const float4 u1 = *reinterpret_cast<const float4*>(p + (1 * 3 + c) * rs);
    const float4 w0 = *reinterpret_cast<const float4*>(p + (2 * 3 + c) * rs);
    const float4 w1 = *reinterpret_cast<const float4*>(p + (3 * 3 + c) * rs);
    float2 h[2][2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const float2 a0 = j ? make_float2(u0.z, u0.w) : make_float2(u0.x, u0.y);
      const float2 a1 = j ? make_float2(u1.z, u1.w) : make_float2(u1.x, u1.y);
      const float2 l0 = j ? make_float2(w0.z, w0.w) : make_float2(w0.x, w0.y);
      const float2 l1 = j ? make_float2(w1.z, w1.w) : make_float2(w1.x, w1.y);
      float2 b0, b1;
      bdag<MU>(a0, a1, b0, b1);
      if (plus) { h[j][0] = cadd(l0, b0); h[j][1] = cadd(l1, b1); }
      else      { h[j][0] = csub(l0, b0); h[j][1] = csub(l1, b1); }
    }
    hq[c] = make_float4(h[0][0].x, h[0][0].y, h[1][0].x, h[1][0].y);
    hq[3 + c] = make_float4(h[0][1].x, h[0][1].y, h[1][1].x, h[1][1].y);
  }
  float2 l[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) l[k] = L[k];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    float2 h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      h0[c] = j ? make_float2(hq[c].z, hq[c].w) : make_float2(hq[c].x, hq[c].y);
      h1[c] = j ? make_float2(hq[3 + c].z, hq[3 + c].w) : make_float2(hq[3 + c].x, hq[3 + c].y);
    }
    float2 g0[3], g1[3];
    su3mul_r<!FWD>(l, h0, g0);
    su3mul_r<!FWD>(l, h1, g1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      hl[j][c] = cadd(hl[j][c], g0[c]);
      hl[j][3 + c] = cadd(hl[j][3 + c], g1[c]);
      float2 b0, b1;
      bmul<MU>(g0[c], g1[c], b0, b1);
      if (plus) { hu[j][c] = cadd(hu[j][c], b0); hu[j][3 + c] = cadd(hu[j][3 + c], b1); }
      else      { hu[j][c] = csub(hu[j][c], b0); hu[j][3 + c] = csub(hu[j][3 + c], b1); }
    }
  }
}

template <int MU, bool DAG, bool PROJ = false>
__device__ __forceinline__ void hop2_dir(const float2* __restrict__ U, const int nb8[8], int64_t V, int64_t site,
                                         int64_t rs, int r0, const float2* __restrict__ in, float2 hu[2][6],
                                         float2 hl[2][6], int64_t in_off = 0) {
  if (PROJ) {
    const int64_t nbk = nb8[4 + MU];
    hop2p<MU, true, DAG>(U + ((int64_t)MU * V + site) * 9, in + ((int64_t)nb8[MU] - in_off) * 12 * rs + r0, rs, hu,
                         hl);
    hop2p<MU, false, DAG>(U + ((int64_t)MU * V + nbk) * 9, in + (nbk - in_off) * 12 * rs + r0, rs, hu, hl);
    return;
  }
  float4 q[12];
  {
    const float2* p = in + ((int64_t)nb8[MU] - in_off) * 12 * rs + r0;
#pragma unroll
    for (int k = 0; k < 12; ++k) q[k] = *reinterpret_cast<const float4*>(p + k * rs);
    hop2<MU, true, DAG>(U + ((int64_t)MU * V + site) * 9, q, hu, hl);
  }
  {
    const int64_t nbk = nb8[4 + MU];
    const float2* p = in + (nbk - in_off) * 12 * rs + r0;
#pragma unroll
    for (int k = 0; k < 12; ++k) q[k] = *reinterpret_cast<const float4*>(p + k * rs);
    hop2<MU, false, DAG>(U + ((int64_t)MU * V + nbk) * 9, q, hu, hl);
  }
}

// (128, 4): at most 128 registers, four blocks per SM; the output is written
// with evict-first stores so that it does not push neighbour spinors out of L2.
// The right-hand sides are swept in chunks of 2 rc2 columns, chunk-major: the
// lattice is traversed once per chunk, so that the spinors a traversal keeps
// in flight between a site and its farthest neighbour in visiting order take
// less L2 (a chunk of 2 rc2 = nrhs is the plain order).
template <bool DAG, bool RESID, int NT, bool PROJ = false>
__global__ void __launch_bounds__(NT, 512 / NT) k_wilson_f32x2(const float2* __restrict__ U, const int* __restrict__ nbr,
                                                      const int* __restrict__ visit, int64_t V, int nrhs, int rc2,
                                                      float mass, float tau,
                                                      const float2* __restrict__ in, float2* __restrict__ out,
                                                      const float2* __restrict__ b) {
  const int half = nrhs >> 1;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= V * half) return;
  const int64_t per_chunk = V * rc2;
  const int ch = (int)(g / per_chunk);
  const int64_t rem = g - ch * per_chunk;
  const int64_t slot = rem / rc2;
  const int r0 = 2 * (ch * rc2 + (int)(rem - slot * rc2));
  const int64_t site = visit[slot];
  const int64_t rs = nrhs;
  int nb8[8];
#pragma unroll
  for (int h = 0; h < 8; ++h) nb8[h] = nbr[site * 8 + h];
  float2 hu[2][6], hl[2][6];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int k = 0; k < 6; ++k) { hu[j][k] = make_float2(0.f, 0.f); hl[j][k] = make_float2(0.f, 0.f); }
  hop2_dir<0, DAG, PROJ>(U, nb8, V, site, rs, r0, in, hu, hl);
  hop2_dir<1, DAG, PROJ>(U, nb8, V, site, rs, r0, in, hu, hl);
  hop2_dir<2, DAG, PROJ>(U, nb8, V, site, rs, r0, in, hu, hl);
  hop2_dir<3, DAG, PROJ>(U, nb8, V, site, rs, r0, in, hu, hl);
  const float te = DAG ? -tau : tau;
  const float2 mup = make_float2(mass, te);
  const float2 mlo = make_float2(mass, -te);
  const float2* x = in + site * 12 * rs + r0;
  float2* y = out + site * 12 * rs + r0;
  const float2* bb = RESID ? b + site * 12 * rs + r0 : nullptr;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const float4 xv = *reinterpret_cast<const float4*>(x + k * rs);
    const float2 m = k < 6 ? mup : mlo;
    float2 v0 = cmul(m, make_float2(xv.x, xv.y));
    float2 v1 = cmul(m, make_float2(xv.z, xv.w));
    const float2 h0 = k < 6 ? hu[0][k] : hl[0][k - 6];
    const float2 h1 = k < 6 ? hu[1][k] : hl[1][k - 6];
    v0.x = fmaf(-0.5f, h0.x, v0.x);
    v0.y = fmaf(-0.5f, h0.y, v0.y);
    v1.x = fmaf(-0.5f, h1.x, v1.x);
    v1.y = fmaf(-0.5f, h1.y, v1.y);
    if (RESID) {
      const float4 bv = *reinterpret_cast<const float4*>(bb + k * rs);
      v0 = make_float2(bv.x - v0.x, bv.y - v0.y);
      v1 = make_float2(bv.z - v1.x, bv.w - v1.y);
    }
    __stcs(reinterpret_cast<float4*>(y + k * rs), make_float4(v0.x, v0.y, v1.x, v1.y));
  }
}

// ---------------------------------------------------------------------------
// Parity-restricted hopping (even-odd solves).  With the sites of parity p
// in [p V/2, (p+1) V/2) and every hop joining sites of opposite parity,
//   y(n) = Q1 z(n) + Q2 (H x)(n)   for the sites n of parity p,
// H x = sum_mu [(1 - gamma_mu) U_mu(n) x(n+mu) + (1 + gamma_mu) U_mu(n-mu)^H
// x(n-mu)] (so A = M - H/2 with M = 4 + m0 + i tau gamma5), Q1 and Q2
// spin-diagonal: q[0] on the upper spins (gamma5 = +1), q[1] on the lower.
// x is a half field of parity 1 - p, z (nullable) and y half fields of
// parity p: element (site, a, r) of a half field of parity q sits at
// ((site - q V/2) 12 + a) nrhs + r.
// ---------------------------------------------------------------------------
struct EoCoef {
  cplx q1[2], q2[2];
};

template <class C>
__global__ void __launch_bounds__(128) k_wilson_eo(const C* __restrict__ U, const int* __restrict__ nbr,
                                                   const int* __restrict__ visit, int64_t V, int nrhs, int p,
                                                   EoCoef q, const C* __restrict__ in, const C* __restrict__ z,
                                                   C* __restrict__ out) {
  typedef typename CTraits<C>::R R;
  const int64_t Vh = V / 2;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= Vh * nrhs) return;
  const int64_t slot = g / nrhs;
  const int r = (int)(g - slot * nrhs);
  const int64_t site = visit[slot];
  const int64_t rs = nrhs;
  const int64_t in_off = (int64_t)(1 - p) * Vh, own = site - (int64_t)p * Vh;
  int nb8[8];
#pragma unroll
  for (int h = 0; h < 8; ++h) nb8[h] = nbr[site * 8 + h];
  C hu[6], hl[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) { hu[k] = mk<C>((R)0, (R)0); hl[k] = mk<C>((R)0, (R)0); }
  hop_dir<0, false>(U, nb8, V, site, rs, r, in, hu, hl, in_off);
  hop_dir<1, false>(U, nb8, V, site, rs, r, in, hu, hl, in_off);
  hop_dir<2, false>(U, nb8, V, site, rs, r, in, hu, hl, in_off);
  hop_dir<3, false>(U, nb8, V, site, rs, r, in, hu, hl, in_off);
  const C q1u = mk<C>((R)q.q1[0].x, (R)q.q1[0].y), q1l = mk<C>((R)q.q1[1].x, (R)q.q1[1].y);
  const C q2u = mk<C>((R)q.q2[0].x, (R)q.q2[0].y), q2l = mk<C>((R)q.q2[1].x, (R)q.q2[1].y);
  const C* zz = z ? z + own * 12 * rs + r : nullptr;
  C* y = out + own * 12 * rs + r;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    C v = cmul(k < 6 ? q2u : q2l, k < 6 ? hu[k] : hl[k - 6]);
    if (zz) v = cadd(v, cmul(k < 6 ? q1u : q1l, zz[k * rs]));
    y[k * rs] = v;
  }
}

// FP32, two right-hand sides per thread (even nrhs, 16-byte aligned fields),
// the columns swept in chunks of 2 rc2 as in k_wilson_f32x2; PROJ: the
// neighbours projected as they load.
template <bool PROJ>
__global__ void __launch_bounds__(128, 4) k_wilson_eo_f32x2(const float2* __restrict__ U, const int* __restrict__ nbr,
                                                         const int* __restrict__ visit, int64_t V, int nrhs, int rc2,
                                                         int p, EoCoef q, const float2* __restrict__ in,
                                                         const float2* __restrict__ z, float2* __restrict__ out) {
  const int half = nrhs >> 1;
  const int64_t Vh = V / 2;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= Vh * half) return;
  const int64_t per_chunk = Vh * rc2;
  const int ch = (int)(g / per_chunk);
  const int64_t rem = g - ch * per_chunk;
  const int64_t slot = rem / rc2;
  const int r0 = 2 * (ch * rc2 + (int)(rem - slot * rc2));
  const int64_t site = visit[slot];
  const int64_t rs = nrhs;
  const int64_t in_off = (int64_t)(1 - p) * Vh, own = site - (int64_t)p * Vh;
  int nb8[8];
#pragma unroll
  for (int h = 0; h < 8; ++h) nb8[h] = nbr[site * 8 + h];
  float2 hu[2][6], hl[2][6];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int k = 0; k < 6; ++k) { hu[j][k] = make_float2(0.f, 0.f); hl[j][k] = make_float2(0.f, 0.f); }
  hop2_dir<0, false, PROJ>(U, nb8, V, site, rs, r0, in, hu, hl, in_off);
  hop2_dir<1, false, PROJ>(U, nb8, V, site, rs, r0, in, hu, hl, in_off);
  hop2_dir<2, false, PROJ>(U, nb8, V, site, rs, r0, in, hu, hl, in_off);
  hop2_dir<3, false, PROJ>(U, nb8, V, site, rs, r0, in, hu, hl, in_off);
  const float2 q1u = make_float2((float)q.q1[0].x, (float)q.q1[0].y), q1l = make_float2((float)q.q1[1].x, (float)q.q1[1].y);
  const float2 q2u = make_float2((float)q.q2[0].x, (float)q.q2[0].y), q2l = make_float2((float)q.q2[1].x, (float)q.q2[1].y);
  const float2* zz = z ? z + own * 12 * rs + r0 : nullptr;
  float2* y = out + own * 12 * rs + r0;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const float2 qa = k < 6 ? q2u : q2l, qb = k < 6 ? q1u : q1l;
    float2 v0 = cmul(qa, k < 6 ? hu[0][k] : hl[0][k - 6]);
    float2 v1 = cmul(qa, k < 6 ? hu[1][k] : hl[1][k - 6]);
    if (zz) {
      const float4 zv = *reinterpret_cast<const float4*>(zz + k * rs);
      v0 = cadd(v0, cmul(qb, make_float2(zv.x, zv.y)));
      v1 = cadd(v1, cmul(qb, make_float2(zv.z, zv.w)));
    }
    *reinterpret_cast<float4*>(y + k * rs) = make_float4(v0.x, v0.y, v1.x, v1.y);
  }
}

// ---------------------------------------------------------------------------
// FP32, two right-hand sides per thread, with the next hop's neighbour
// spinor copied into shared memory (cp.async, 12 x 16 bytes per thread) while
// the current hop computes, and the next hop's link loaded into registers
// likewise: each thread keeps one hop's loads in flight behind its
// arithmetic instead of waiting for them at the start of every hop.  Two
// stages of 12 x 16 bytes per thread (48 KB per 128-thread block, four
// blocks per SM).  After the eight hops the stages take the site's own input
// (full lattice) or z, then b (residual form).  MODE as k_wilson_bulk; the
// thread-to-(site, column pair) map, the sums and the epilogue are those of
// k_wilson_f32x2 / k_wilson_eo_f32x2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cpa16(float4* dst, const float2* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(ptx::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

constexpr int kCpThreads = 128;
constexpr size_t kCpSmem = 2 * 12 * kCpThreads * sizeof(float4);  // 48 KB

template <bool DAG, int MODE>
__global__ void __launch_bounds__(kCpThreads, 4) k_wilson_cp(const float2* __restrict__ U, const int* __restrict__ nbr,
                                                        const int* __restrict__ visit, int64_t V, int nrhs, int rc2,
                                                        float mass, float tau, EoCoef q, int p,
                                                        const float2* __restrict__ in,
                                                        const float2* __restrict__ aux, float2* __restrict__ out) {
  constexpr bool eo = MODE >= 2;
  extern __shared__ float4 cp_stage[];  // [2][12][kCpThreads]
  const int half = nrhs >> 1;
  const int64_t nslots = eo ? V / 2 : V;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= nslots * half) return;
  const int64_t per_chunk = nslots * rc2;
  const int ch = (int)(g / per_chunk);
  const int64_t rem = g - ch * per_chunk;
  const int64_t slot = rem / rc2;
  const int r0 = 2 * (ch * rc2 + (int)(rem - slot * rc2));
  const int64_t site = visit[slot];
  const int64_t rs = nrhs;
  const int64_t in_off = eo ? (int64_t)(1 - p) * (V / 2) : 0, own = eo ? site - (int64_t)p * (V / 2) : site;
  int nb8[8];
#pragma unroll
  for (int h = 0; h < 8; ++h) nb8[h] = nbr[site * 8 + h];
  float4* st = cp_stage + threadIdx.x;
  // operand h: hop h (mu = h / 2, forward when h is even), 8: the site's own
  // input (full lattice) or z, 9: b
  auto src = [&](int h) -> const float2* {
    if (h < 8) return in + ((int64_t)nb8[(h & 1) ? 4 + (h >> 1) : (h >> 1)] - in_off) * 12 * rs + r0;
    if (h == 8) return (eo ? aux : in) + own * 12 * rs + r0;
    return aux + site * 12 * rs + r0;
  };
  auto issue = [&](int j, const float2* ptr) {
#pragma unroll
    for (int k = 0; k < 12; ++k) cpa16(st + (j * 12 + k) * kCpThreads, ptr + k * rs);
    cpa_commit();
  };
  auto load_link = [&](int h, float2 l[9]) {
    const int mu = h >> 1;
    const float2* L = U + ((int64_t)mu * V + ((h & 1) ? (int64_t)nb8[4 + mu] : site)) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) l[k] = L[k];
  };
  float2 hu[2][6], hl[2][6];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int k = 0; k < 6; ++k) { hu[j][k] = make_float2(0.f, 0.f); hl[j][k] = make_float2(0.f, 0.f); }
  issue(0, src(0));
  float2 lc[9];
  load_link(0, lc);
  auto step = [&](auto hc) {
    constexpr int H = decltype(hc)::value;
    constexpr bool more = H + 1 < 8 || MODE != 2;  // an operand follows hop H
    if constexpr (more) issue((H + 1) & 1, src(H + 1));
    float2 ln[9];
    if constexpr (H + 1 < 8) load_link(H + 1, ln);
    if constexpr (more) cpa_wait<1>();
    else cpa_wait<0>();
    float4 qv[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) qv[k] = st[((H & 1) * 12 + k) * kCpThreads];
    hop2l<H / 2, (H % 2) == 0, DAG>(lc, qv, hu, hl);
    if constexpr (H + 1 < 8) {
#pragma unroll
      for (int k = 0; k < 9; ++k) lc[k] = ln[k];
    }
  };
  step(std::integral_constant<int, 0>{});
  step(std::integral_constant<int, 1>{});
  step(std::integral_constant<int, 2>{});
  step(std::integral_constant<int, 3>{});
  step(std::integral_constant<int, 4>{});
  step(std::integral_constant<int, 5>{});
  step(std::integral_constant<int, 6>{});
  step(std::integral_constant<int, 7>{});
  float2* y = out + own * 12 * rs + r0;
  if constexpr (MODE == 1) issue(1, src(9));  // b, into the stage hop 7 used
  if constexpr (MODE != 2) cpa_wait<0>();
  const float4* xs = st;                  // own input or z: stage 0
  const float4* bs = st + 12 * kCpThreads;  // b: stage 1
  if constexpr (!eo) {
    const float te = DAG ? -tau : tau;
    const float2 mup = make_float2(mass, te);
    const float2 mlo = make_float2(mass, -te);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const float4 xv = xs[k * kCpThreads];
      const float2 m = k < 6 ? mup : mlo;
      float2 v0 = cmul(m, make_float2(xv.x, xv.y));
      float2 v1 = cmul(m, make_float2(xv.z, xv.w));
      const float2 h0 = k < 6 ? hu[0][k] : hl[0][k - 6];
      const float2 h1 = k < 6 ? hu[1][k] : hl[1][k - 6];
      v0.x = fmaf(-0.5f, h0.x, v0.x);
      v0.y = fmaf(-0.5f, h0.y, v0.y);
      v1.x = fmaf(-0.5f, h1.x, v1.x);
      v1.y = fmaf(-0.5f, h1.y, v1.y);
      if constexpr (MODE == 1) {
        const float4 bv = bs[k * kCpThreads];
        v0 = make_float2(bv.x - v0.x, bv.y - v0.y);
        v1 = make_float2(bv.z - v1.x, bv.w - v1.y);
      }
      __stcs(reinterpret_cast<float4*>(y + k * rs), make_float4(v0.x, v0.y, v1.x, v1.y));
    }
  } else {
    const float2 q1u = make_float2((float)q.q1[0].x, (float)q.q1[0].y), q1l = make_float2((float)q.q1[1].x, (float)q.q1[1].y);
    const float2 q2u = make_float2((float)q.q2[0].x, (float)q.q2[0].y), q2l = make_float2((float)q.q2[1].x, (float)q.q2[1].y);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const float2 qa = k < 6 ? q2u : q2l, qb = k < 6 ? q1u : q1l;
      float2 v0 = cmul(qa, k < 6 ? hu[0][k] : hl[0][k - 6]);
      float2 v1 = cmul(qa, k < 6 ? hu[1][k] : hl[1][k - 6]);
      if constexpr (MODE == 3) {
        const float4 zv = xs[k * kCpThreads];
        v0 = cadd(v0, cmul(qb, make_float2(zv.x, zv.y)));
        v1 = cadd(v1, cmul(qb, make_float2(zv.z, zv.w)));
      }
      *reinterpret_cast<float4*>(y + k * rs) = make_float4(v0.x, v0.y, v1.x, v1.y);
    }
  }
}

// Launch of k_wilson_cp over chunks of 2 rc2 columns; false when it does not
// apply (odd nrhs, fields not 16-byte aligned, rc2 not dividing nrhs / 2).
template <bool DAG, int MODE>
bool launch_cp(qd_ctx& ctx, const float2* U, const int* nbr, const int* visit, int64_t V, int nrhs, int rc2,
               float mass, float tau, const EoCoef& q, int p, const float2* in, const float2* aux, float2* out) {
  if (nrhs % 2 != 0 || rc2 <= 0 || (nrhs / 2) % rc2 != 0) return false;
  if (((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(aux) | reinterpret_cast<uintptr_t>(out)) & 15) !=
      0)
    return false;
  const int64_t nslots = MODE >= 2 ? V / 2 : V;
  const int64_t tot = nslots * (nrhs / 2);
  if (tot == 0) return true;
  auto kern = k_wilson_cp<DAG, MODE>;
  ensure_smem_limit(reinterpret_cast<const void*>(kern), kCpSmem);
  kern<<<(int)div_up(tot, kCpThreads), kCpThreads, kCpSmem, ctx.stream>>>(U, nbr, visit, V, nrhs, rc2, mass, tau, q, p,
                                                                          in, aux, out);
  QD_LAUNCH_CHECK();
  return true;
}

// ---------------------------------------------------------------------------
// FP32 stencil with its operands staged in shared memory by bulk copies
// (cp.async.bulk, completion counted on an mbarrier).  A warp computes one
// site for a chunk of 64 columns at a time, lane l owning columns 2l and
// 2l + 1 of the chunk.  The site's operand chunks -- the eight neighbour
// spinors in hop order (mu = 0..3, forward then backward), then its own
// input (full lattice) or z (parity-restricted form), then b (residual
// form), each 12 rows of 512 contiguous bytes -- stream through a ring of NS
// slots per warp: once a slot has been read into registers, the warp refills
// it with the chunk NS positions ahead, so that NS x 6 KB of loads per warp
// stay in flight without holding registers.  The links of the next site are
// copied into a double buffer with cp.async while the current site
// computes; the neighbour indices are looked up two sites ahead and the
// visiting order three.  The arithmetic per element is that of
// k_wilson_f32x2 and k_wilson_eo_f32x2 (the same hop2 and epilogue).  Every
// wait is bounded: on a timeout the warp records it in *err, waits (bounded)
// for its own copies in flight and returns.
// ---------------------------------------------------------------------------
constexpr int kBulkCols = 64;
constexpr uint32_t kBulkRow = kBulkCols * 8;    // one spin-colour row of a chunk: 512 B
constexpr uint32_t kBulkChunk = 12 * kBulkRow;  // 6144 B

struct BulkArgs {
  const float2* U;
  const int* nbr;
  const int* visit;
  int64_t V;        // sites of the full lattice (the link stride)
  int64_t nslots;   // sites in the visiting order (V, or V/2 for one parity)
  int nrhs;
  int64_t in_off;   // first site of the input field (0, or (1 - p) V/2)
  int64_t own_off;  // first site of z and out (0, or p V/2)
  float mass, tau;  // full lattice: 4 + m0, tau
  EoCoef q;         // parity-restricted: Q1, Q2
  const float2* in;
  const float2* aux;  // b (residual form) or z (parity-restricted; null: none)
  float2* out;
  int* err;
};

// MODE 0: out = A in (A^H with DAG); 1: out = b - A in; 2: out = Q2 (H in)
// on one parity; 3: out = Q1 z + Q2 (H in).
template <int MODE>
struct BulkMode {
  static constexpr bool eo = MODE >= 2;
  static constexpr bool own = MODE != 2;
  static constexpr bool resid = MODE == 1;
  static constexpr int cps = 8 + (own ? 1 : 0) + (resid ? 1 : 0);  // chunks per site
};

template <int NW, int NS>
constexpr size_t bulk_smem_bytes() {
  return (size_t)NW * NS * kBulkChunk + (size_t)NW * 144 * sizeof(float2) + (size_t)NW * NS * 8 + 16;
}

// Lane k < cps of a warp holds the source of chunk k of a site (and, for a
// hop, its link); dst is the site's output chunk (the same in every lane).
struct BulkAddr {
  const float2* src;
  const float2* lnk;
  float2* dst;
};

__device__ __forceinline__ int bulk_visit(const BulkArgs& a, bool valid, int64_t u) {
  if (!valid) return 0;
  const int64_t ch = u / a.nslots;
  return a.visit[u - ch * a.nslots];
}

// The lookups of a site: lane k < 8 loads the neighbour of hop k.  Its
// value is first used when the record is turned into addresses (bulk_cook),
// one site later, so the load does not stall the warp.
struct BulkRaw {
  int nb;
  int site;
  int64_t r0;
  bool valid;
};

__device__ __forceinline__ BulkRaw bulk_raw(const BulkArgs& a, bool valid, int64_t u, int site, int lane) {
  BulkRaw w{0, site, 0, valid};
  if (!valid) return w;
  w.r0 = (u / a.nslots) * kBulkCols;
  if (lane < 8) w.nb = a.nbr[(int64_t)site * 8 + ((lane & 1) ? 4 + (lane >> 1) : (lane >> 1))];
  return w;
}

template <int MODE>
__device__ __forceinline__ BulkAddr bulk_cook(const BulkArgs& a, const BulkRaw& w, int lane) {
  using M = BulkMode<MODE>;
  BulkAddr o{nullptr, nullptr, nullptr};
  if (!w.valid) return o;
  const int64_t rs = a.nrhs;
  o.dst = a.out + ((int64_t)w.site - a.own_off) * 12 * rs + w.r0;
  if (lane < 8) {
    const int mu = lane >> 1;
    const bool fwd = (lane & 1) == 0;
    o.src = a.in + ((int64_t)w.nb - a.in_off) * 12 * rs + w.r0;
    o.lnk = a.U + ((int64_t)mu * a.V + (fwd ? w.site : w.nb)) * 9;
  } else if (M::own && lane == 8) {
    o.src = (M::eo ? a.aux : a.in) + ((int64_t)w.site - a.own_off) * 12 * rs + w.r0;
  } else if (M::resid && lane == 9) {
    o.src = a.aux + (int64_t)w.site * 12 * rs + w.r0;
  }
  return o;
}

template <class P>
__device__ __forceinline__ P* shfl_ptr(P* p, int src_lane) {
  return reinterpret_cast<P*>(__shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(p), src_lane));
}

// The 12 rows of one chunk into a ring slot (all lanes of the warp call it).
__device__ __forceinline__ void bulk_issue(uint32_t slot, uint32_t bar, const float2* src, int64_t rs, int lane) {
  if (lane == 0) ptx::mbar_expect_tx(bar, kBulkChunk);
  __syncwarp();
  if (lane < 12) ptx::bulk_g2s(slot + lane * kBulkRow, src + lane * rs, kBulkRow, bar);
}

// The eight links of a site (72 float2, 8-byte aligned) into dst with
// cp.async; lane k < 8 holds the address of link k.  One commit group.
__device__ __forceinline__ void bulk_links(float2* dst, const float2* lnk, int lane) {
#pragma unroll
  for (int it = 0; it < 3; ++it) {
    const int e = lane + 32 * it;
    const int h = e < 72 ? e / 9 : 7;
    const float2* L = shfl_ptr(lnk, h);
    if (e < 72) {
      const uint32_t d = ptx::smem_u32(dst + e);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(L + (e - 9 * h)) : "memory");
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <bool DAG, int MODE, int NW, int NS>
__global__ void __launch_bounds__(NW * 32, 1) k_wilson_bulk(const BulkArgs a) {
  using M = BulkMode<MODE>;
  constexpr int CPS = M::cps;
  static_assert(NS >= 1 && NS <= 8, "a refill must land at most one site ahead");
  extern __shared__ __align__(128) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t ring_bytes = (size_t)NW * NS * kBulkChunk, link_bytes = (size_t)NW * 144 * sizeof(float2);
  unsigned char* ring = smem + (size_t)warp * NS * kBulkChunk;
  float2* lbuf = reinterpret_cast<float2*>(smem + ring_bytes) + warp * 144;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + ring_bytes + link_bytes) + warp * NS;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + ring_bytes + link_bytes + (size_t)NW * NS * 8);
  if (threadIdx.x == 0) *abort_flag = 0;
  if (lane == 0)
    for (int s = 0; s < NS; ++s) ptx::mbar_init(ptx::smem_u32(bars + s), 1);
  ptx::mbar_init_fence();
  __syncthreads();

  const int64_t rs = a.nrhs;
  const int64_t total = a.nslots * (a.nrhs / kBulkCols);
  const int64_t GW = (int64_t)gridDim.x * NW;
  const int64_t gw = (int64_t)blockIdx.x * NW + warp;
  const int64_t nw = gw < total ? (total - 1 - gw) / GW + 1 : 0;  // sites of this warp: units gw + i GW
  if (nw == 0) return;
  const uint32_t ring_a = ptx::smem_u32(ring), bar_a = ptx::smem_u32(bars);

  // cur: site i, na: site i + 1 (addresses); nb: site i + 2 (lookups); vs:
  // the visiting order of site i + 3
  BulkAddr cur = bulk_cook<MODE>(a, bulk_raw(a, true, gw, bulk_visit(a, true, gw), lane), lane);
  BulkAddr na = bulk_cook<MODE>(a, bulk_raw(a, 1 < nw, gw + GW, bulk_visit(a, 1 < nw, gw + GW), lane), lane);
  BulkRaw nb = bulk_raw(a, 2 < nw, gw + 2 * GW, bulk_visit(a, 2 < nw, gw + 2 * GW), lane);
  int vs = bulk_visit(a, 3 < nw, gw + 3 * GW);
  bulk_links(lbuf, cur.lnk, lane);
#pragma unroll
  for (int k = 0; k < NS; ++k) bulk_issue(ring_a + k * kBulkChunk, bar_a + 8 * k, shfl_ptr(cur.src, k), rs, lane);

  int slot = 0;
  uint32_t ph = 0;
  int64_t consumed = 0, issued = NS;  // positions in the warp's sequence of chunks
  bool ok = true;
  const float te = DAG ? -a.tau : a.tau;
  const float2 mup = make_float2(a.mass, te), mlo = make_float2(a.mass, -te);
  const float2 q1u = make_float2((float)a.q.q1[0].x, (float)a.q.q1[0].y);
  const float2 q1l = make_float2((float)a.q.q1[1].x, (float)a.q.q1[1].y);
  const float2 q2u = make_float2((float)a.q.q2[0].x, (float)a.q.q2[0].y);
  const float2 q2l = make_float2((float)a.q.q2[1].x, (float)a.q.q2[1].y);

  for (int64_t i = 0; i < nw && ok; ++i) {
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();  // the links of site i are in lbuf[i & 1] for the whole warp
    const float2* L = lbuf + (i & 1) * 72;
    if (i + 1 < nw) bulk_links(lbuf + ((i + 1) & 1) * 72, na.lnk, lane);
    float2 hu[2][6], hl[2][6];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int k = 0; k < 6; ++k) { hu[j][k] = make_float2(0.f, 0.f); hl[j][k] = make_float2(0.f, 0.f); }

    auto step = [&](auto kc) {
      constexpr int K = decltype(kc)::value;
      if constexpr (K < CPS) {
        if (!ok) return;
        const bool got = ptx::mbar_wait(bar_a + 8 * slot, ph, abort_flag);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          return;
        }
        ++consumed;
        const float4* S = reinterpret_cast<const float4*>(ring + (size_t)slot * kBulkChunk) + lane;
        float4 q[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) q[c] = S[c * 32];
        __syncwarp();
        // the slot takes the chunk NS positions ahead: this site's, or the next one's
        constexpr int KN = K + NS;
        const float2* nsrc;
        if constexpr (KN < CPS) nsrc = shfl_ptr(cur.src, KN);
        else nsrc = shfl_ptr(na.src, KN - CPS);
        if (KN < CPS || i + 1 < nw) {
          ptx::fence_proxy_async_smem();
          bulk_issue(ring_a + slot * kBulkChunk, bar_a + 8 * slot, nsrc, rs, lane);
          ++issued;
        }
        if (++slot == NS) {
          slot = 0;
          ph ^= 1u;
        }
        if constexpr (K < 8) hop2<K / 2, (K % 2) == 0, DAG>(L + K * 9, q, hu, hl);
        if constexpr (MODE == 2 && K == 7) {  // Q2 (H in)
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            const float2 qa = c < 6 ? q2u : q2l;
            const float2 v0 = cmul(qa, c < 6 ? hu[0][c] : hl[0][c - 6]);
            const float2 v1 = cmul(qa, c < 6 ? hu[1][c] : hl[1][c - 6]);
            reinterpret_cast<float4*>(cur.dst + c * rs)[lane] = make_float4(v0.x, v0.y, v1.x, v1.y);
          }
        }
        if constexpr (MODE == 3 && K == 8) {  // Q2 (H in) + Q1 z
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            const float2 qa = c < 6 ? q2u : q2l, qb = c < 6 ? q1u : q1l;
            float2 v0 = cmul(qa, c < 6 ? hu[0][c] : hl[0][c - 6]);
            float2 v1 = cmul(qa, c < 6 ? hu[1][c] : hl[1][c - 6]);
            v0 = cadd(v0, cmul(qb, make_float2(q[c].x, q[c].y)));
            v1 = cadd(v1, cmul(qb, make_float2(q[c].z, q[c].w)));
            reinterpret_cast<float4*>(cur.dst + c * rs)[lane] = make_float4(v0.x, v0.y, v1.x, v1.y);
          }
        }
        if constexpr (MODE <= 1 && K == 8) {  // (4 + m0 + i tau gamma5) in - H in / 2
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            const float2 m = c < 6 ? mup : mlo;
            float2 v0 = cmul(m, make_float2(q[c].x, q[c].y));
            float2 v1 = cmul(m, make_float2(q[c].z, q[c].w));
            float2& h0 = c < 6 ? hu[0][c] : hl[0][c - 6];
            float2& h1 = c < 6 ? hu[1][c] : hl[1][c - 6];
            v0.x = fmaf(-0.5f, h0.x, v0.x);
            v0.y = fmaf(-0.5f, h0.y, v0.y);
            v1.x = fmaf(-0.5f, h1.x, v1.x);
            v1.y = fmaf(-0.5f, h1.y, v1.y);
            if constexpr (MODE == 1) {
              h0 = v0;
              h1 = v1;
            } else {
              __stcs(reinterpret_cast<float4*>(cur.dst + c * rs) + lane, make_float4(v0.x, v0.y, v1.x, v1.y));
            }
          }
        }
        if constexpr (MODE == 1 && K == 9) {  // b - A in
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            const float2 v0 = c < 6 ? hu[0][c] : hl[0][c - 6];
            const float2 v1 = c < 6 ? hu[1][c] : hl[1][c - 6];
            __stcs(reinterpret_cast<float4*>(cur.dst + c * rs) + lane,
                   make_float4(q[c].x - v0.x, q[c].y - v0.y, q[c].z - v1.x, q[c].w - v1.y));
          }
        }
      }
    };
    step(std::integral_constant<int, 0>{});
    step(std::integral_constant<int, 1>{});
    step(std::integral_constant<int, 2>{});
    step(std::integral_constant<int, 3>{});
    step(std::integral_constant<int, 4>{});
    step(std::integral_constant<int, 5>{});
    step(std::integral_constant<int, 6>{});
    step(std::integral_constant<int, 7>{});
    step(std::integral_constant<int, 8>{});
    step(std::integral_constant<int, 9>{});
    cur = na;
    na = bulk_cook<MODE>(a, nb, lane);
    nb = bulk_raw(a, i + 3 < nw, gw + (i + 3) * GW, vs, lane);
    vs = bulk_visit(a, i + 4 < nw, gw + (i + 4) * GW);
  }
  if (!ok) {
    if (lane == 0) {
      atomicExch(a.err, 1);
      *abort_flag = 1;
    }
    // the copies this warp still has in flight land before it leaves
    int never = 0;
    for (int64_t j = consumed; j < issued; ++j)
      (void)ptx::mbar_wait(bar_a + 8 * (uint32_t)(j % NS), (uint32_t)((j / NS) & 1), &never);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Launch of k_wilson_bulk: NW warps per CTA, NS ring slots per warp, one
// CTA per SM (persistent).  false when the shape does not apply (nrhs not a
// multiple of 64, fields not 16-byte aligned).
template <bool DAG, int MODE, int NW, int NS>
bool launch_bulk(qd_ctx& ctx, const BulkArgs& a) {
  if (a.nrhs % kBulkCols != 0) return false;
  if (((reinterpret_cast<uintptr_t>(a.in) | reinterpret_cast<uintptr_t>(a.aux) | reinterpret_cast<uintptr_t>(a.out)) &
       15) != 0)
    return false;
  const int64_t total = a.nslots * (a.nrhs / kBulkCols);
  if (total == 0) return true;
  constexpr size_t smem = bulk_smem_bytes<NW, NS>();
  static_assert(smem <= 227 * 1024, "shared memory per CTA");
  auto kern = k_wilson_bulk<DAG, MODE, NW, NS>;
  ensure_smem_limit(reinterpret_cast<const void*>(kern), smem);
  const int blocks = (int)std::min<int64_t>(div_up(total, NW), kNumSMs);
  kern<<<blocks, NW * 32, smem, ctx.stream>>>(a);
  QD_LAUNCH_CHECK();
  return true;
}

// The ring shapes the tuner tries: (warps, slots) = (8, 4), (4, 8), (6, 5),
// 192 KB, 192 KB and 180 KB of loads in flight per SM.
template <bool DAG, int MODE>
bool launch_bulk_shape(qd_ctx& ctx, const BulkArgs& a, int shape) {
  switch (shape) {
    case 0: return launch_bulk<DAG, MODE, 8, 4>(ctx, a);
    case 1: return launch_bulk<DAG, MODE, 4, 8>(ctx, a);
    default: return launch_bulk<DAG, MODE, 6, 5>(ctx, a);
  }
}

int wilson_bulk_error(qd_ctx& ctx, const LevelGeom& geo) {
  if (geo.bulk_err.bytes() == 0) return 0;
  int h = 0;
  QD_CUDA(cudaMemcpyAsync(&h, geo.bulk_err.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaStreamSynchronize(ctx.stream));
  return h;
}

template <class C>
void wilson_eo(qd_ctx& ctx, const LevelGeom& geo, const C* links, int p, const cplx q1[2], const cplx q2[2],
               const C* in, const C* z, C* out, int nrhs) {
  QD_REQUIRE(geo.eo && geo.nsites % 2 == 0, "parity-restricted hopping needs an even-odd lattice");
  const int64_t Vh = geo.nsites / 2;
  const int64_t tot = Vh * nrhs;
  if (tot == 0) return;
  EoCoef q;
  for (int h = 0; h < 2; ++h) {
    q.q1[h] = q1[h];
    q.q2[h] = q2[h];
  }
  const double cb = (double)sizeof(C);
  ProfScope ps(ctx, sizeof(C) == 16 ? QD_PROF_WILSON_F64 : QD_PROF_WILSON_F32, 1368.0 * (double)tot,
               (double)Vh * ((z ? 36.0 : 24.0) * cb * nrhs + 72.0 * cb));
  const int* nb = geo.nbr.as<int>();
  const int* vis = geo.visit_par[p].as<int>();
  const bool x2 = sizeof(C) == 8 && nrhs % 2 == 0 &&
                  ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out) | reinterpret_cast<uintptr_t>(z)) &
                   15) == 0;
  if (x2) {
    // candidates: columns swept whole, in chunks of 64 or 32, and the whole
    // sweep with the neighbours projected as they load (same sums per
    // element in the first three: the same bits)
    auto launch = [&](int c) -> bool {
      const int rc = c == 1 ? 64 : (c == 2 ? 32 : nrhs);
      if (rc > nrhs || nrhs % rc != 0 || (c == 1 && nrhs <= 64) || (c == 2 && nrhs <= 32)) return false;
      auto kern = c == 3 ? k_wilson_eo_f32x2<true> : k_wilson_eo_f32x2<false>;
      kern<<<div_up(Vh * (nrhs / 2), 128), 128, 0, ctx.stream>>>(
          reinterpret_cast<const float2*>(links), nb, vis, geo.nsites, nrhs, rc / 2, p, q,
          reinterpret_cast<const float2*>(in), reinterpret_cast<const float2*>(z), reinterpret_cast<float2*>(out));
      QD_LAUNCH_CHECK();
      return true;
    };
    // candidates 4-6: operands staged by bulk copies (k_wilson_bulk), ring
    // shapes 0-2; nrhs a multiple of 64
    auto launch_any = [&](int c) -> bool {
      if (c < 4) return launch(c);
      if (c >= 7) {  // the next hop's operands in flight behind the current one (k_wilson_cp)
        const int rc = c == 8 ? 64 : nrhs;
        if (c == 8 && (nrhs <= 64 || nrhs % 64 != 0)) return false;
        const float2* Lf = reinterpret_cast<const float2*>(links);
        const float2* xin = reinterpret_cast<const float2*>(in);
        const float2* zz = reinterpret_cast<const float2*>(z);
        float2* yo = reinterpret_cast<float2*>(out);
        return z ? launch_cp<false, 3>(ctx, Lf, nb, vis, geo.nsites, nrhs, rc / 2, 0.f, 0.f, q, p, xin, zz, yo)
                 : launch_cp<false, 2>(ctx, Lf, nb, vis, geo.nsites, nrhs, rc / 2, 0.f, 0.f, q, p, xin, zz, yo);
      }
      BulkArgs a{};
      a.U = reinterpret_cast<const float2*>(links);
      a.nbr = nb;
      a.visit = vis;
      a.V = geo.nsites;
      a.nslots = Vh;
      a.nrhs = nrhs;
      a.in_off = (int64_t)(1 - p) * Vh;
      a.own_off = (int64_t)p * Vh;
      a.q = q;
      a.in = reinterpret_cast<const float2*>(in);
      a.aux = reinterpret_cast<const float2*>(z);
      a.out = reinterpret_cast<float2*>(out);
      a.err = geo.bulk_err.as<int>();
      return z ? launch_bulk_shape<false, 3>(ctx, a, c - 4) : launch_bulk_shape<false, 2>(ctx, a, c - 4);
    };
    // out-of-place (out differs from in and z): safe to time
    const std::string key = "wilson eo f32 sites" + std::to_string(geo.nsites) + " rhs" + std::to_string(nrhs) +
                            (z ? " z" : "");
    const int c = (out == in || out == z) ? -1 : tune_pick(ctx, key, 9, launch_any);
    if (c >= 4 && launch_any(c)) return;
    if (c < 0 || !launch(c)) launch(0);
    return;
  } else {
    k_wilson_eo<C><<<div_up(tot, 128), 128, 0, ctx.stream>>>(links, nb, vis, geo.nsites, nrhs, p, q, in, z, out);
  }
  QD_LAUNCH_CHECK();
}

template void wilson_eo<cplx>(qd_ctx&, const LevelGeom&, const cplx*, int, const cplx*, const cplx*, const cplx*,
                              const cplx*, cplx*, int);
template void wilson_eo<cplxf>(qd_ctx&, const LevelGeom&, const cplxf*, int, const cplx*, const cplx*, const cplxf*,
                               const cplxf*, cplxf*, int);

// out = Q in on a half field (Q spin-diagonal as above).
template <class C>
__global__ void k_spin_diag(int64_t nh, int nrhs, cplx qu, cplx ql, const C* __restrict__ in, C* __restrict__ out) {
  typedef typename CTraits<C>::R R;
  const int64_t tot = nh * 12 * nrhs;
  const C a = mk<C>((R)qu.x, (R)qu.y), b = mk<C>((R)ql.x, (R)ql.y);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)((e / nrhs) % 12);
    out[e] = cmul(k < 6 ? a : b, in[e]);
  }
}

template <class C>
void spin_diag(qd_ctx& ctx, int64_t nh, int nrhs, const cplx q[2], const C* in, C* out) {
  const int64_t tot = nh * 12 * nrhs;
  if (tot == 0) return;
  k_spin_diag<C><<<(int)std::min<int64_t>(div_up(tot, 256), 32 * kNumSMs), 256, 0, ctx.stream>>>(nh, nrhs, q[0], q[1],
                                                                                               in, out);
  QD_LAUNCH_CHECK();
}
template void spin_diag<cplx>(qd_ctx&, int64_t, int, const cplx*, const cplx*, cplx*);
template void spin_diag<cplxf>(qd_ctx&, int64_t, int, const cplx*, const cplxf*, cplxf*);

template <class C>
void wilson_apply(qd_ctx& ctx, const LevelGeom& geo, const C* links, double m0, double tau,
                  bool dagger, const C* in, C* out, int nrhs, const C* b) {
  const int64_t tot = geo.nsites * nrhs;
  if (tot == 0) return;
  const int threads = 128;
  const int blocks = div_up(tot, threads);
  const double cb = (double)sizeof(C);
  ProfScope ps(ctx, sizeof(C) == 16 ? QD_PROF_WILSON_F64 : QD_PROF_WILSON_F32, 1368.0 * (double)tot,
               (double)geo.nsites * ((b ? 36.0 : 24.0) * cb * nrhs + 36.0 * cb));
  const int* nb = geo.nbr.as<int>();
  const int* vis = geo.visit.as<int>();
  const double mass = 4.0 + m0;
  // candidates 0, 2-7: two right-hand sides per thread (FP32, even nrhs,
  // 16-byte aligned fields), the columns swept whole or in chunks, in blocks
  // of 128, 256 or 512 threads (a block of nt threads covers nt / (chunk / 2)
  // consecutive sites of the visiting order, whose shared neighbours then
  // hit in L1); 8-9: whole or chunks of 64 with the neighbours projected as
  // they load (hop2p); candidate 1: one per thread.  The FP32 choice is tuned.
  auto launch_x2 = [&](int rc, int nt, bool proj = false) -> bool {
    if (!(sizeof(C) == 8 && (nrhs % 2) == 0 &&
          ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out) | reinterpret_cast<uintptr_t>(b)) &
           15) == 0))
      return false;
    if (rc <= 0) rc = nrhs;
    if (rc > nrhs || nrhs % rc != 0 || rc % 2 != 0) return false;
    const int rc2 = rc / 2;
    const int64_t tot2 = geo.nsites * (nrhs / 2);
    const float2* L = reinterpret_cast<const float2*>(links);
    const float2* xin = reinterpret_cast<const float2*>(in);
    float2* yout = reinterpret_cast<float2*>(out);
    const float2* bb = reinterpret_cast<const float2*>(b);
    const float fm = (float)mass, ft = (float)tau;
    auto go = [&](auto kern) {
      kern<<<(int)div_up(tot2, nt), nt, 0, ctx.stream>>>(L, nb, vis, geo.nsites, nrhs, rc2, fm, ft, xin, yout, bb);
    };
    auto pick = [&](auto k128, auto k256, auto k512, auto k128p) {
      if (proj) go(k128p);
      else if (nt == 512) go(k512);
      else if (nt == 256) go(k256);
      else go(k128);
    };
    if (b) {
      if (dagger)
        pick(k_wilson_f32x2<true, true, 128>, k_wilson_f32x2<true, true, 256>, k_wilson_f32x2<true, true, 512>,
             k_wilson_f32x2<true, true, 128, true>);
      else
        pick(k_wilson_f32x2<false, true, 128>, k_wilson_f32x2<false, true, 256>, k_wilson_f32x2<false, true, 512>,
             k_wilson_f32x2<false, true, 128, true>);
    } else {
      if (dagger)
        pick(k_wilson_f32x2<true, false, 128>, k_wilson_f32x2<true, false, 256>, k_wilson_f32x2<true, false, 512>,
             k_wilson_f32x2<true, false, 128, true>);
      else
        pick(k_wilson_f32x2<false, false, 128>, k_wilson_f32x2<false, false, 256>, k_wilson_f32x2<false, false, 512>,
             k_wilson_f32x2<false, false, 128, true>);
    }
    QD_LAUNCH_CHECK();
    return true;
  };
  auto launch_x1 = [&]() -> bool {
    if (b) {
      if (dagger)
        k_wilson<C, true, true><<<blocks, threads, 0, ctx.stream>>>(links, nb, vis, geo.nsites, nrhs, mass, tau, in, out, b);
      else
        k_wilson<C, false, true><<<blocks, threads, 0, ctx.stream>>>(links, nb, vis, geo.nsites, nrhs, mass, tau, in, out, b);
    } else {
      if (dagger)
        k_wilson<C, true, false><<<blocks, threads, 0, ctx.stream>>>(links, nb, vis, geo.nsites, nrhs, mass, tau, in, out,
                                                                     nullptr);
      else
        k_wilson<C, false, false><<<blocks, threads, 0, ctx.stream>>>(links, nb, vis, geo.nsites, nrhs, mass, tau, in, out,
                                                                      nullptr);
    }
    QD_LAUNCH_CHECK();
    return true;
  };
  if (sizeof(C) == 16) {
    launch_x1();
    return;
  }
  // candidates 10-12: operands staged by bulk copies (k_wilson_bulk), ring
  // shapes 0-2; FP32, nrhs a multiple of 64, 16-byte aligned fields
  auto launch_bulk_c = [&](int shape) -> bool {
    if (sizeof(C) != 8) return false;
    BulkArgs a{};
    a.U = reinterpret_cast<const float2*>(links);
    a.nbr = nb;
    a.visit = vis;
    a.V = geo.nsites;
    a.nslots = geo.nsites;
    a.nrhs = nrhs;
    a.mass = (float)mass;
    a.tau = (float)tau;
    a.in = reinterpret_cast<const float2*>(in);
    a.aux = reinterpret_cast<const float2*>(b);
    a.out = reinterpret_cast<float2*>(out);
    a.err = geo.bulk_err.as<int>();
    if (b) return dagger ? launch_bulk_shape<true, 1>(ctx, a, shape) : launch_bulk_shape<false, 1>(ctx, a, shape);
    return dagger ? launch_bulk_shape<true, 0>(ctx, a, shape) : launch_bulk_shape<false, 0>(ctx, a, shape);
  };
  // candidates 13-14: the next hop's operands in flight behind the current
  // one (k_wilson_cp), columns swept whole or in chunks of 64
  auto launch_cp_c = [&](int rc) -> bool {
    if (sizeof(C) != 8) return false;
    if (rc <= 0) rc = nrhs;
    if (rc > nrhs || nrhs % rc != 0 || rc % 2 != 0) return false;
    const float2* Lf = reinterpret_cast<const float2*>(links);
    const float2* xin = reinterpret_cast<const float2*>(in);
    const float2* bb = reinterpret_cast<const float2*>(b);
    float2* yo = reinterpret_cast<float2*>(out);
    const float fm = (float)mass, ft = (float)tau;
    const EoCoef q0{};
    if (b)
      return dagger ? launch_cp<true, 1>(ctx, Lf, nb, vis, geo.nsites, nrhs, rc / 2, fm, ft, q0, 0, xin, bb, yo)
                    : launch_cp<false, 1>(ctx, Lf, nb, vis, geo.nsites, nrhs, rc / 2, fm, ft, q0, 0, xin, bb, yo);
    return dagger ? launch_cp<true, 0>(ctx, Lf, nb, vis, geo.nsites, nrhs, rc / 2, fm, ft, q0, 0, xin, bb, yo)
                  : launch_cp<false, 0>(ctx, Lf, nb, vis, geo.nsites, nrhs, rc / 2, fm, ft, q0, 0, xin, bb, yo);
  };
  auto launch = [&](int c) -> bool {
    switch (c) {
      case 13: return launch_cp_c(0);
      case 14: return nrhs > 64 && launch_cp_c(64);
      case 10: case 11: case 12: return launch_bulk_c(c - 10);
      case 0: return launch_x2(0, 128);
      case 1: return launch_x1();
      case 2: return nrhs > 64 && launch_x2(64, 128);
      case 3: return nrhs > 32 && launch_x2(32, 128);
      case 4: return nrhs > 32 && launch_x2(32, 256);
      case 5: return nrhs > 32 && launch_x2(32, 512);
      case 6: return nrhs > 16 && launch_x2(16, 512);
      case 7: return nrhs > 64 && launch_x2(64, 512);
      case 8: return launch_x2(0, 128, true);
      default: return nrhs > 64 && launch_x2(64, 128, true);
    }
  };
  // the residual form writes out = b - A in: out-of-place, safe to repeat
  const std::string key = std::string("wilson f32 sites") + std::to_string(geo.nsites) + " rhs" +
                          std::to_string(nrhs) + (b ? " resid" : "") + (dagger ? " dag" : "");
  const int c = (out == b || out == in) ? -1 : tune_pick(ctx, key, 15, launch);
  if (c >= 0 && launch(c)) return;
  if (!launch_x2(0, 128)) launch_x1();
}

template void wilson_apply<cplx>(qd_ctx&, const LevelGeom&, const cplx*, double, double, bool,
                                 const cplx*, cplx*, int, const cplx*);
template void wilson_apply<cplxf>(qd_ctx&, const LevelGeom&, const cplxf*, double, double, bool,
                                  const cplxf*, cplxf*, int, const cplxf*);

template <>
void WilsonOp<cplx>::apply(qd_ctx& ctx, const cplx* in, cplx* out, int nrhs) const {
  wilson_apply<cplx>(ctx, g->geo, links, m0, tau, dagger, in, out, nrhs, nullptr);
}
template <>
void WilsonOp<cplxf>::apply(qd_ctx& ctx, const cplxf* in, cplxf* out, int nrhs) const {
  wilson_apply<cplxf>(ctx, g->geo, links, m0, tau, dagger, in, out, nrhs, nullptr);
}
template <>
void WilsonOp<cplx>::residual(qd_ctx& ctx, const cplx* b, const cplx* x, cplx* r, int nrhs) const {
  wilson_apply<cplx>(ctx, g->geo, links, m0, tau, dagger, x, r, nrhs, b);
}
template <>
void WilsonOp<cplxf>::residual(qd_ctx& ctx, const cplxf* b, const cplxf* x, cplxf* r, int nrhs) const {
  wilson_apply<cplxf>(ctx, g->geo, links, m0, tau, dagger, x, r, nrhs, b);
}

}  // namespace qd
