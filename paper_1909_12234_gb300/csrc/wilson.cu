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
#include "qd_internal.cuh"

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
                                        const C* __restrict__ in, C hu[6], C hl[6]) {
  const double sg = DAG ? -1.0 : 1.0;
  // forward: (1 - s gamma) U_mu(n) x(n + mu)
  {
    const int64_t nf = nb8[MU];
    const C* p = in + nf * 12 * rs + r;
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
    const C* p = in + nbk * 12 * rs + r;
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
k_wilson(const C* __restrict__ U, const int* __restrict__ nbr, int64_t V, int nrhs, double mass,
         double tau, const C* __restrict__ in, C* __restrict__ out, const C* __restrict__ b) {
  typedef typename CTraits<C>::R R;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= V * nrhs) return;
  const int64_t site = g / nrhs;
  const int r = (int)(g - site * nrhs);
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
  const double mass = 4.0 + m0;
  if (b) {
    if (dagger)
      k_wilson<C, true, true><<<blocks, threads, 0, ctx.stream>>>(links, nb, geo.nsites, nrhs, mass, tau, in, out, b);
    else
      k_wilson<C, false, true><<<blocks, threads, 0, ctx.stream>>>(links, nb, geo.nsites, nrhs, mass, tau, in, out, b);
  } else {
    if (dagger)
      k_wilson<C, true, false><<<blocks, threads, 0, ctx.stream>>>(links, nb, geo.nsites, nrhs, mass, tau, in, out,
                                                                   nullptr);
    else
      k_wilson<C, false, false><<<blocks, threads, 0, ctx.stream>>>(links, nb, geo.nsites, nrhs, mass, tau, in, out,
                                                                    nullptr);
  }
  QD_LAUNCH_CHECK();
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
