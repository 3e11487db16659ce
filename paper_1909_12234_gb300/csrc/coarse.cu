// Multigrid transfer and coarse-level kernels (Sec. 2):
//   * blocking of the null vectors onto aggregates and a per-(aggregate,
//     chirality) orthonormal basis (CGS2), giving W with gamma5 W = W gamma5^W
//     (Algorithm 2, step 1);
//   * prolongation W c and restriction W^H x (two-grid step 1);
//   * the Galerkin coarse operator C = W^H A W as a 9-point block stencil,
//     and its application.
#include <string>
#include "coarse_tc.cuh"
#include "restrict_tc.cuh"
#include "qd_internal.cuh"
#include "tune.cuh"

namespace qd {

// ---------------------------------------------------------------------------
// Tables
// ---------------------------------------------------------------------------
void build_transfer_tables(Transfer& T, const LevelGeom& fine, const int block[4],
                           LevelGeom& coarse_geo) {
  int cd[4];
  T.bsites = 1;
  for (int m = 0; m < 4; ++m) {
    QD_REQUIRE(block[m] >= 1 && fine.dims[m] % block[m] == 0,
               "aggregate block must divide the lattice in every direction");
    T.block[m] = block[m];
    cd[m] = fine.dims[m] / block[m];
    T.bsites *= block[m];
  }
  coarse_geo.build(cd, false);
  T.nfine = fine.nsites;
  T.ncoarse = coarse_geo.nsites;
  std::vector<int> agg(T.nfine), members(T.ncoarse * T.bsites), fill(T.ncoarse, 0);
  std::vector<int8_t> hd(T.nfine * 8);
  for (int64_t s = 0; s < T.nfine; ++s) {
    int c[4], cc[4];
    fine.coords(fine.h_lex_of_site[s], c);
    for (int m = 0; m < 4; ++m) cc[m] = c[m] / block[m];
    const int a = (int)coarse_geo.lex(cc);
    agg[s] = a;
    members[(int64_t)a * T.bsites + fill[a]++] = (int)s;
    for (int mu = 0; mu < 4; ++mu) {
      const int rem = c[mu] % block[mu];
      hd[s * 8 + mu] = (rem == block[mu] - 1) ? (int8_t)(1 + mu) : (int8_t)0;
      hd[s * 8 + 4 + mu] = (rem == 0) ? (int8_t)(5 + mu) : (int8_t)0;
    }
  }
  T.agg_of.resize(T.nfine * sizeof(int));
  T.members.resize(members.size() * sizeof(int));
  T.hopdir.resize(hd.size());
  QD_CUDA(cudaMemcpy(T.agg_of.as<int>(), agg.data(), agg.size() * sizeof(int), cudaMemcpyHostToDevice));
  QD_CUDA(cudaMemcpy(T.members.as<int>(), members.data(), members.size() * sizeof(int),
                     cudaMemcpyHostToDevice));
  QD_CUDA(cudaMemcpy(T.hopdir.as<int8_t>(), hd.data(), hd.size(), cudaMemcpyHostToDevice));
}

// ---------------------------------------------------------------------------
// Prolongation: fine[s][a][r] = sum_j W[s][a][j] coarse[agg(s)][c(a) nv + j][r]
// ---------------------------------------------------------------------------
template <class C>
__global__ void k_prolong(int64_t nfine, int Df, int nv, int nrhs, const int* __restrict__ agg_of,
                          const C* __restrict__ W, const C* __restrict__ coarse, C* __restrict__ fine) {
  typedef typename CTraits<C>::R R;
  const int64_t tot = nfine * Df * nrhs;
  const int Dc = 2 * nv;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % nrhs);
    const int64_t sa = e / nrhs;
    const int a = (int)(sa % Df);
    const int64_t s = sa / Df;
    const int chir = (a >= Df / 2) ? 1 : 0;
    const C* w = W + sa * nv;
    const C* cv = coarse + ((int64_t)agg_of[s] * Dc + chir * nv) * nrhs + r;
    C acc = mk<C>((R)0, (R)0);
    for (int j = 0; j < nv; ++j) cfma(acc, w[j], cv[(int64_t)j * nrhs]);
    fine[e] = acc;
  }
}

// FP32 form.  Fine sites are taken aggregate by aggregate (through the
// member table), so that the 2 nv coarse values of an aggregate are read
// from memory once and then hit in cache for its other fine sites.  A block
// covers spb fine sites x tps threads: W[s][.][.] of its sites is staged in
// shared memory (broadcast reads), and thread (site, rp) holds
// coarse[agg][c nv + j][2rp, 2rp + 1] of one chirality c at a time in
// registers and forms fine[s][a][2rp, 2rp + 1] for the Df/2 components a of
// that chirality.  Same products in the same order as k_prolong, so the
// results are identical.
template <int NV>
__global__ void __launch_bounds__(256, NV <= 12 ? 3 : 2) k_prolong_f32x2(int nsites, int bsites, int Df, int nrhs2, int tps, int spb,
                                                      const int* __restrict__ members, const float4* __restrict__ W,
                                                      const float4* __restrict__ coarse, float4* __restrict__ fine) {
  extern __shared__ float4 wsm[];  // [spb][Df][NV / 2]
  const int half = Df / 2;
  const int wrow = Df * (NV / 2);  // float4 per site
  const int li = threadIdx.x / tps, lane = threadIdx.x - li * tps;
  for (int q0 = blockIdx.x * spb; q0 < nsites; q0 += gridDim.x * spb) {
    __syncthreads();  // the previous sites' W is no longer read
    for (int e = threadIdx.x; e < spb * wrow; e += blockDim.x) {
      const int i = e / wrow, k = e - i * wrow;
      if (q0 + i < nsites) wsm[e] = __ldg(W + (size_t)members[q0 + i] * wrow + k);
    }
    __syncthreads();
    const int q = q0 + li;
    if (li >= spb || q >= nsites) continue;
    const int s = members[q];
    const int x = q / bsites;
    const float4* ws = wsm + li * wrow;
    for (int rp = lane; rp < nrhs2; rp += tps) {
#pragma unroll 1
      for (int c = 0; c < 2; ++c) {
        float4 cv[NV];
        const float4* cb = coarse + ((size_t)x * 2 * NV + (size_t)c * NV) * nrhs2 + rp;
#pragma unroll
        for (int j = 0; j < NV; ++j) cv[j] = cb[(size_t)j * nrhs2];
        float4* fo = fine + ((size_t)s * Df + (size_t)c * half) * nrhs2 + rp;
#pragma unroll 2
        for (int a = 0; a < half; ++a) {
          const float4* w = ws + (c * half + a) * (NV / 2);
          float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int jj = 0; jj < NV / 2; ++jj) {
            const float4 wv = w[jj];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const float wr = h ? wv.z : wv.x, wi = h ? wv.w : wv.y;
              const float4 v = cv[2 * jj + h];
              acc.x = fmaf(wr, v.x, fmaf(-wi, v.y, acc.x));
              acc.y = fmaf(wr, v.y, fmaf(wi, v.x, acc.y));
              acc.z = fmaf(wr, v.z, fmaf(-wi, v.w, acc.z));
              acc.w = fmaf(wr, v.w, fmaf(wi, v.z, acc.w));
            }
          }
          fo[(size_t)a * nrhs2] = acc;
        }
      }
    }
  }
}

// Restriction: coarse[x][c nv + j][r] = sum_{s in x, a in c} conj(W[s][a][j]) fine[s][a][r]
template <class C>
__global__ void k_restrict(int64_t ncoarse, int bsites, int Df, int nv, int nrhs,
                           const int* __restrict__ members, const C* __restrict__ W,
                           const C* __restrict__ fine, C* __restrict__ coarse) {
  typedef typename CTraits<C>::R R;
  const int Dc = 2 * nv;
  const int64_t tot = ncoarse * Dc * nrhs;
  const int half = Df / 2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % nrhs);
    const int64_t xd = e / nrhs;
    const int d = (int)(xd % Dc);
    const int64_t x = xd / Dc;
    const int chir = d / nv, j = d - chir * nv;
    C acc = mk<C>((R)0, (R)0);
    for (int m = 0; m < bsites; ++m) {
      const int64_t s = members[x * bsites + m];
      const C* w = W + (s * Df + chir * half) * nv + j;
      const C* f = fine + (s * Df + chir * half) * nrhs + r;
      for (int a = 0; a < half; ++a) cfmac(acc, w[(int64_t)a * nv], f[(int64_t)a * nrhs]);
    }
    coarse[e] = acc;
  }
}

// Restriction with the aggregate staged in shared memory: one CTA per
// (aggregate, tile of RT right-hand sides).  The block's fine values
// F[m][a][rr] and its W[m][a][j] are read from global memory once; every
// output coarse[x][c nv + j][r] = sum_{m, a in c} conj(W[m][a][j]) F[m][a][rr]
// is then formed from shared memory.
template <class C>
__global__ void k_restrict_smem(int bsites, int Df, int nv, int nrhs, int RT, const int* __restrict__ members,
                                const C* __restrict__ W, const C* __restrict__ fine, C* __restrict__ coarse) {
  typedef typename CTraits<C>::R R;
  extern __shared__ unsigned char smr[];
  C* F = reinterpret_cast<C*>(smr);       // [rows][RT]
  const int rows = bsites * Df;
  C* Ws = F + (size_t)rows * RT;          // [rows][nv]
  const int x = blockIdx.x;
  const int r0 = blockIdx.y * RT;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int e = tid; e < rows * RT; e += nth) {
    const int row = e / RT, rr = e - row * RT;
    const int m = row / Df, a = row - m * Df;
    const int64_t s = members[(int64_t)x * bsites + m];
    F[e] = (r0 + rr < nrhs) ? fine[(s * Df + a) * nrhs + r0 + rr] : mk<C>((R)0, (R)0);
  }
  for (int e = tid; e < rows * nv; e += nth) {
    const int row = e / nv, j = e - row * nv;
    const int m = row / Df, a = row - m * Df;
    const int64_t s = members[(int64_t)x * bsites + m];
    Ws[e] = W[(s * Df + a) * nv + j];
  }
  __syncthreads();
  const int Dc = 2 * nv, half = Df / 2;
  for (int o = tid; o < Dc * RT; o += nth) {
    const int d = o / RT, rr = o - d * RT;
    if (r0 + rr >= nrhs) continue;
    const int chir = d / nv, j = d - chir * nv;
    C acc = mk<C>((R)0, (R)0);
    for (int m = 0; m < bsites; ++m) {
      const int rbase = m * Df + chir * half;
      for (int a = 0; a < half; ++a) cfmac(acc, Ws[(rbase + a) * nv + j], F[(rbase + a) * RT + rr]);
    }
    coarse[((int64_t)x * Dc + d) * nrhs + r0 + rr] = acc;
  }
}

template <class C>
void prolongate(qd_ctx& ctx, const Transfer& T, const C* W, const C* coarse, C* fine, int nrhs) {
  const int64_t tot = T.nfine * T.Df * nrhs;
  const double cb = (double)sizeof(C);
  ProfScope ps(ctx, sizeof(C) == 16 ? QD_PROF_PROLONG_F64 : QD_PROF_PROLONG_F32, 8.0 * T.nv * (double)tot,
               cb * ((double)T.nfine * T.Df * T.nv + (double)tot + (double)T.ncoarse * T.Dc * nrhs));
  const bool al16 = ((reinterpret_cast<uintptr_t>(W) | reinterpret_cast<uintptr_t>(coarse) |
                      reinterpret_cast<uintptr_t>(fine)) & 15) == 0;
  if (sizeof(C) == sizeof(cplxf) && nrhs % 2 == 0 && al16 && (T.nv == 8 || T.nv == 12 || T.nv == 16) &&
      T.nfine * T.Df * (int64_t)nrhs < ((int64_t)1 << 31)) {
    const int nr2 = nrhs / 2;
    const int tps = nr2 < 256 ? nr2 : 256;
    // sites per block: 256 threads at most, their W in at most 32 KB
    const int wsite = T.Df * (T.nv / 2) * (int)sizeof(float4);
    int spb = 256 / tps;
    if (spb * wsite > 32 * 1024) spb = 32 * 1024 / wsite;
    if (spb < 1) spb = 1;
    const int nsites = (int)T.nfine;
    const int blocks = (int)std::min<int64_t>(div_up(nsites, spb), 16 * kNumSMs);
    const size_t smem = (size_t)spb * T.Df * (T.nv / 2) * sizeof(float4);
    const int* mem = T.members.as<int>();
    const float4* w4 = reinterpret_cast<const float4*>(W);
    const float4* c4 = reinterpret_cast<const float4*>(coarse);
    float4* f4 = reinterpret_cast<float4*>(fine);
    switch (T.nv) {
      case 8:
        k_prolong_f32x2<8><<<blocks, spb * tps, smem, ctx.stream>>>(nsites, T.bsites, T.Df, nr2, tps, spb, mem, w4, c4, f4);
        break;
      case 12:
        k_prolong_f32x2<12><<<blocks, spb * tps, smem, ctx.stream>>>(nsites, T.bsites, T.Df, nr2, tps, spb, mem, w4, c4,
                                                                     f4);
        break;
      default:
        k_prolong_f32x2<16><<<blocks, spb * tps, smem, ctx.stream>>>(nsites, T.bsites, T.Df, nr2, tps, spb, mem, w4, c4,
                                                                     f4);
        break;
    }
    QD_LAUNCH_CHECK();
    return;
  }
  k_prolong<C><<<div_up(tot, 256) < 32 * kNumSMs ? div_up(tot, 256) : 32 * kNumSMs, 256, 0, ctx.stream>>>(
      T.nfine, T.Df, T.nv, nrhs, T.agg_of.as<int>(), W, coarse, fine);
  QD_LAUNCH_CHECK();
}

template <class C>
void restrict_(qd_ctx& ctx, const Transfer& T, const C* W, const C* fine, C* coarse, int nrhs) {
  if (sizeof(C) == sizeof(cplxf) && T.use_tc && W == T.Wf.as<C>() && restrict_tc_supported(T, fine, coarse, nrhs)) {
    restrict_tc(ctx, const_cast<Transfer&>(T), reinterpret_cast<const cplxf*>(fine), reinterpret_cast<cplxf*>(coarse),
                nrhs);
    return;
  }
  const int64_t tot = T.ncoarse * T.Dc * nrhs;
  const double cb = (double)sizeof(C);
  ProfScope ps(ctx, sizeof(C) == 16 ? QD_PROF_RESTRICT_F64 : QD_PROF_RESTRICT_F32,
               8.0 * T.nv * (double)T.nfine * T.Df * nrhs,
               cb * ((double)T.nfine * T.Df * T.nv + (double)T.nfine * T.Df * nrhs + (double)tot));
  // staged kernel when the aggregate tile fits in 96 KB of shared memory
  const int rows = T.bsites * T.Df;
  int RT = 1;
  while (RT < nrhs && RT < 32) RT <<= 1;
  const size_t cap = 96 * 1024;
  while (RT > 1 && (size_t)rows * (RT + T.nv) * sizeof(C) > cap) RT >>= 1;
  const size_t smem = (size_t)rows * (RT + T.nv) * sizeof(C);
  if (smem <= cap && (RT >= 8 || RT >= nrhs)) {
    ensure_smem_limit(reinterpret_cast<const void*>(k_restrict_smem<C>), smem);
    k_restrict_smem<C><<<dim3((unsigned)T.ncoarse, div_up(nrhs, RT)), 256, smem, ctx.stream>>>(
        T.bsites, T.Df, T.nv, nrhs, RT, T.members.as<int>(), W, fine, coarse);
  } else {
    k_restrict<C><<<div_up(tot, 128) < 32 * kNumSMs ? div_up(tot, 128) : 32 * kNumSMs, 128, 0, ctx.stream>>>(
        T.ncoarse, T.bsites, T.Df, T.nv, nrhs, T.members.as<int>(), W, fine, coarse);
  }
  QD_LAUNCH_CHECK();
}

template void prolongate<cplx>(qd_ctx&, const Transfer&, const cplx*, const cplx*, cplx*, int);
template void prolongate<cplxf>(qd_ctx&, const Transfer&, const cplxf*, const cplxf*, cplxf*, int);
template void restrict_<cplx>(qd_ctx&, const Transfer&, const cplx*, const cplx*, cplx*, int);
template void restrict_<cplxf>(qd_ctx&, const Transfer&, const cplxf*, const cplxf*, cplxf*, int);

// ---------------------------------------------------------------------------
// Coarse stencil: y[x][d][r] = sum_dir sum_e C[x][dir][d][e] in[nb(x,dir)][e][r]
// ---------------------------------------------------------------------------
template <class C>
__global__ void k_coarse_apply(int64_t nsites, int D, int nrhs, const int* __restrict__ nbr,
                               const C* __restrict__ mat, const C* __restrict__ in, C* __restrict__ out) {
  typedef typename CTraits<C>::R R;
  const int64_t tot = nsites * D * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % nrhs);
    const int64_t xd = e / nrhs;
    const int d = (int)(xd % D);
    const int64_t x = xd / D;
    C acc = mk<C>((R)0, (R)0);
    for (int dir = 0; dir < 9; ++dir) {
      const int64_t y = (dir == 0) ? x : (int64_t)nbr[x * 8 + (dir <= 4 ? dir - 1 : dir - 1)];
      const C* row = mat + ((x * 9 + dir) * D + d) * D;
      const C* v = in + y * D * nrhs + r;
      for (int k = 0; k < D; ++k) cfma(acc, row[k], v[(int64_t)k * nrhs]);
    }
    out[e] = acc;
  }
}

// Register-blocked coarse stencil: one CTA per (coarse site, chunk of
// right-hand sides).  The site's nine D x D blocks are staged in shared
// memory transposed, [dir][e][d] with leading dimension ld, so that the RB
// rows a thread owns are contiguous for every column e.  Each thread keeps
// RB rows x NR right-hand sides of accumulators: per (dir, e) it reads NR
// neighbour values from global memory once (coalesced over the chunk) and
// the RB matrix entries as broadcast vector loads, then does RB x NR complex
// FMAs - instead of two loads per FMA in the one-thread-per-output form.
template <class C, int RB, int NR>
__global__ void __launch_bounds__(256) k_coarse_apply_tiled(int D, int ld, int nrhs, int rhs_per_cta, int nchunks,
                                                            const int* __restrict__ nbr, const C* __restrict__ mat,
                                                            const C* __restrict__ in, C* __restrict__ out) {
  typedef typename CTraits<C>::R R;
  extern __shared__ __align__(16) unsigned char coarse_smem[];
  C* sm = reinterpret_cast<C*>(coarse_smem);
  const int64_t x = blockIdx.x / nchunks;
  const int chunk = (int)(blockIdx.x - x * nchunks);
  const int tid = threadIdx.x;
  const int tpg = rhs_per_cta / NR;  // threads per row group
  const int g = tid / tpg, t = tid - g * tpg;
  const int DD = D * D;
  // stage C[x][dir][d][e] -> sm[(dir * D + e) * ld + d]
  const C* src = mat + x * 9 * (int64_t)DD;
  for (int idx = tid; idx < 9 * DD; idx += blockDim.x) {
    const int dir = idx / DD, rem = idx - dir * DD;
    const int d = rem / D, e = rem - d * D;
    sm[(dir * D + e) * ld + d] = src[idx];
  }
  __syncthreads();
  const int r0 = chunk * rhs_per_cta + t * NR;
  if (r0 >= nrhs) return;
  const bool full = (r0 + NR <= nrhs);
  C acc[RB][NR];
#pragma unroll
  for (int i = 0; i < RB; ++i)
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[i][j] = mk<C>((R)0, (R)0);
  for (int dir = 0; dir < 9; ++dir) {
    const int64_t y = dir == 0 ? x : (int64_t)nbr[x * 8 + dir - 1];
    const C* v = in + y * D * (int64_t)nrhs + r0;
    const C* colbase = sm + dir * D * ld + g * RB;
#pragma unroll 2
    for (int e = 0; e < D; ++e) {
      C xv[NR];
      if (NR == 2 && sizeof(C) == 8 && full) {
        const float4 q = *reinterpret_cast<const float4*>(v + (int64_t)e * nrhs);
        xv[0] = mk<C>((R)q.x, (R)q.y);
        xv[NR - 1] = mk<C>((R)q.z, (R)q.w);
      } else {
#pragma unroll
        for (int j = 0; j < NR; ++j) xv[j] = (r0 + j < nrhs) ? v[(int64_t)e * nrhs + j] : mk<C>((R)0, (R)0);
      }
      const C* col = colbase + e * ld;
      C m[RB];
      if (sizeof(C) == 8) {
#pragma unroll
        for (int i = 0; i < RB / 2; ++i) {
          const float4 q = reinterpret_cast<const float4*>(col)[i];
          m[2 * i] = mk<C>((R)q.x, (R)q.y);
          m[2 * i + 1] = mk<C>((R)q.z, (R)q.w);
        }
      } else {
#pragma unroll
        for (int i = 0; i < RB; ++i) m[i] = col[i];
      }
#pragma unroll
      for (int i = 0; i < RB; ++i)
#pragma unroll
        for (int j = 0; j < NR; ++j) cfma(acc[i][j], m[i], xv[j]);
    }
  }
  C* o = out + x * D * (int64_t)nrhs + r0;
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    C* orow = o + (int64_t)(g * RB + i) * nrhs;
    if (NR == 2 && sizeof(C) == 8 && full) {
      *reinterpret_cast<float4*>(orow) = make_float4((float)acc[i][0].x, (float)acc[i][0].y,
                                                     (float)acc[i][NR - 1].x, (float)acc[i][NR - 1].y);
    } else {
#pragma unroll
      for (int j = 0; j < NR; ++j)
        if (r0 + j < nrhs) orow[j] = acc[i][j];
    }
  }
}

// Launch the tiled kernel for rows-per-thread RB when D is a multiple of it;
// returns false (nothing launched) when the staged blocks would not fit.
template <class C, int RB>
static bool coarse_tiled_launch(qd_ctx& ctx, const CoarseLevel& lv, const C* mat, const C* in, C* out, int nrhs,
                                int tpg_cap = 256) {
  const int D = lv.D;
  if (D % RB != 0) return false;
  const int ngroups = D / RB;
  if (ngroups > 8) return false;
  // float2: rows 16-byte aligned (ld even); double2: odd ld spreads banks
  const int ld = sizeof(C) == 8 ? D + 2 : D + 1;
  const size_t smem = (size_t)9 * D * ld * sizeof(C);
  if (smem > 200 * 1024) return false;
  constexpr int NR = sizeof(C) == 8 ? 2 : 1;
  // the vector loads of two float2 values need an even row length and
  // 16-byte aligned fields
  if (NR == 2 && ((nrhs & 1) || ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15)))
    return false;
  int cap = (256 / ngroups) / 32 * 32;
  if (cap > tpg_cap) cap = tpg_cap;
  if (cap < 32) return false;
  int tpg = div_up(div_up(nrhs, NR), 32) * 32;
  if (tpg > cap) tpg = cap;
  const int rhs_per_cta = tpg * NR;
  const int nchunks = div_up(nrhs, rhs_per_cta);
  // one limit per kernel and device, the largest any shape of it needs
  ensure_smem_limit(reinterpret_cast<const void*>(k_coarse_apply_tiled<C, RB, NR>), 200 * 1024);
  const int64_t blocks = lv.geo.nsites * (int64_t)nchunks;
  k_coarse_apply_tiled<C, RB, NR><<<(unsigned)blocks, ngroups * tpg, smem, ctx.stream>>>(
      D, ld, nrhs, rhs_per_cta, nchunks, lv.geo.nbr.as<int>(), mat, in, out);
  QD_LAUNCH_CHECK();
  return true;
}

template <class C>
void coarse_apply(qd_ctx& ctx, const CoarseLevel& lv, const C* mat, const C* in, C* out, int nrhs) {
  const int64_t tot = lv.geo.nsites * lv.D * nrhs;
  const double cb = (double)sizeof(C);
  ProfScope ps(ctx, sizeof(C) == 16 ? QD_PROF_COARSE_F64 : QD_PROF_COARSE_F32, 72.0 * lv.D * (double)tot,
               cb * (double)lv.geo.nsites * (9.0 * lv.D * lv.D + 2.0 * lv.D * nrhs));
  // candidates: rows per thread 12, 16, 8, 6, 4 with the widest block, then
  // the same with 32 threads per row group (more, smaller blocks), then the
  // one-thread-per-output kernel; all sum every output in the same order,
  // so the choice changes the time, never the result
  auto launch = [&](int c) -> bool {
    const int cap = c < 5 ? 256 : 32;
    switch (c % 5 + (c == 10 ? 5 : 0)) {
      case 0: return coarse_tiled_launch<C, 12>(ctx, lv, mat, in, out, nrhs, cap);
      case 1: return coarse_tiled_launch<C, 16>(ctx, lv, mat, in, out, nrhs, cap);
      case 2: return coarse_tiled_launch<C, 8>(ctx, lv, mat, in, out, nrhs, cap);
      case 3: return coarse_tiled_launch<C, 6>(ctx, lv, mat, in, out, nrhs, cap);
      case 4: return coarse_tiled_launch<C, 4>(ctx, lv, mat, in, out, nrhs, cap);
      default:
        k_coarse_apply<C><<<div_up(tot, 128) < 64 * kNumSMs ? div_up(tot, 128) : 64 * kNumSMs, 128, 0, ctx.stream>>>(
            lv.geo.nsites, lv.D, nrhs, lv.geo.nbr.as<int>(), mat, in, out);
        QD_LAUNCH_CHECK();
        return true;
    }
  };
  const std::string key = std::string("coarse_stencil f") + std::to_string(8 * sizeof(C) / 2) + " D" +
                          std::to_string(lv.D) + " sites" + std::to_string(lv.geo.nsites) + " rhs" +
                          std::to_string(nrhs);
  const int c = in == out ? -1 : tune_pick(ctx, key, 11, launch);
  if (c >= 0 && launch(c)) return;
  for (int d = 0; d < 11; ++d)
    if (launch(d)) return;
}
template void coarse_apply<cplx>(qd_ctx&, const CoarseLevel&, const cplx*, const cplx*, cplx*, int);
template void coarse_apply<cplxf>(qd_ctx&, const CoarseLevel&, const cplxf*, const cplxf*, cplxf*, int);

template <>
void CoarseOp<cplx>::apply(qd_ctx& ctx, const cplx* in, cplx* out, int nrhs) const {
  coarse_apply<cplx>(ctx, *lv, mat, in, out, nrhs);
}
template <>
void CoarseOp<cplxf>::apply(qd_ctx& ctx, const cplxf* in, cplxf* out, int nrhs) const {
  if (lv->use_tc && in != out && coarse_tc_supported(*lv, in, out, nrhs)) {
    coarse_apply_tc(ctx, const_cast<CoarseLevel&>(*lv), in, out, nrhs);
    return;
  }
  coarse_apply<cplxf>(ctx, *lv, mat, in, out, nrhs);
}
template <>
void CoarseOp<cplx>::residual(qd_ctx& ctx, const cplx* b, const cplx* x, cplx* r, int nrhs) const {
  Op<cplx>::residual(ctx, b, x, r, nrhs);
}
// r = b - C x: on the tensor cores the subtraction is part of the epilogue
template <>
void CoarseOp<cplxf>::residual(qd_ctx& ctx, const cplxf* b, const cplxf* x, cplxf* r, int nrhs) const {
  if (lv->use_tc && r != x && r != b && coarse_tc_supported(*lv, x, r, nrhs) &&
      (reinterpret_cast<uintptr_t>(b) & 15) == 0) {
    coarse_apply_tc(ctx, const_cast<CoarseLevel&>(*lv), x, r, nrhs, b);
    return;
  }
  Op<cplxf>::residual(ctx, b, x, r, nrhs);
}

// ---------------------------------------------------------------------------
// Block orthonormalisation: one CTA per (aggregate, chirality).  The block
// of the null vectors Y (layout [nfine][Df][nv]) restricted to the aggregate
// and chirality is orthonormalised by classical Gram-Schmidt applied twice,
// column by column in null-vector order; the result is W on those rows.
// ---------------------------------------------------------------------------
__global__ void k_block_cgs2(int bsites, int Df, int nv, const int* __restrict__ members,
                             const cplx* __restrict__ Y, cplx* __restrict__ W, int* __restrict__ err) {
  extern __shared__ cplx sm[];
  const int half = Df / 2;
  const int rows = bsites * half;
  cplx* G = sm;               // [rows][nv]
  cplx* coef = sm + rows * nv;  // [nv]
  double* red = reinterpret_cast<double*>(coef + nv);  // [blockDim.x]
  const int x = blockIdx.x >> 1, chir = blockIdx.x & 1;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int e = tid; e < rows * nv; e += nth) {
    const int row = e / nv, v = e - row * nv;
    const int m = row / half, a = chir * half + (row - m * half);
    const int64_t s = members[(int64_t)x * bsites + m];
    G[e] = Y[(s * Df + a) * nv + v];
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
  for (int v = 0; v < nv; ++v) {
    for (int pass = 0; pass < 2; ++pass) {
      for (int u = warp; u < v; u += nwarp) {
        cplx acc = mkc(0.0, 0.0);
        for (int row = lane; row < rows; row += 32) cfmac(acc, G[row * nv + u], G[row * nv + v]);
        for (int off = 16; off > 0; off >>= 1) {
          acc.x += __shfl_down_sync(0xffffffffu, acc.x, off);
          acc.y += __shfl_down_sync(0xffffffffu, acc.y, off);
        }
        if (lane == 0) coef[u] = acc;
      }
      __syncthreads();
      for (int row = tid; row < rows; row += nth) {
        cplx w = G[row * nv + v];
        for (int u = 0; u < v; ++u) {
          const cplx c = coef[u];
          cfma(w, mkc(-c.x, -c.y), G[row * nv + u]);
        }
        G[row * nv + v] = w;
      }
      __syncthreads();
    }
    double part = 0.0;
    for (int row = tid; row < rows; row += nth) part += cnorm2(G[row * nv + v]);
    red[tid] = part;
    __syncthreads();
    for (int h = nth / 2; h > 0; h >>= 1) {
      if (tid < h) red[tid] += red[tid + h];
      __syncthreads();
    }
    const double nrm = sqrt(red[0]);
    __syncthreads();
    if (!(nrm > 1e-300)) {
      if (tid == 0) atomicExch(err, 1);
    } else {
      const double inv = 1.0 / nrm;
      for (int row = tid; row < rows; row += nth) G[row * nv + v] = cscale(inv, G[row * nv + v]);
    }
    __syncthreads();
  }
  for (int e = tid; e < rows * nv; e += nth) {
    const int row = e / nv, v = e - row * nv;
    const int m = row / half, a = chir * half + (row - m * half);
    const int64_t s = members[(int64_t)x * bsites + m];
    W[(s * Df + a) * nv + v] = G[e];
  }
}

void block_orthonormalize(qd_ctx& ctx, Transfer& T, const cplx* Y) {
  const int rows = T.bsites * (T.Df / 2);
  QD_REQUIRE(T.nv <= rows, "more null vectors than rows of an aggregate block");
  const int threads = 256;
  const size_t smem = ((size_t)rows * T.nv + T.nv) * sizeof(cplx) + threads * sizeof(double);
  QD_REQUIRE(smem <= 220 * 1024, "aggregate block too large for the shared-memory CGS2 kernel");
  ensure_smem_limit(reinterpret_cast<const void*>(k_block_cgs2), smem);
  T.W.resize(T.nfine * T.Df * T.nv * sizeof(cplx));
  DevBuf err(sizeof(int));
  QD_CUDA(cudaMemsetAsync(err.as<int>(), 0, sizeof(int), ctx.stream));
  k_block_cgs2<<<(int)(2 * T.ncoarse), threads, smem, ctx.stream>>>(T.bsites, T.Df, T.nv,
                                                                    T.members.as<int>(), Y,
                                                                    T.W.as<cplx>(), err.as<int>());
  QD_LAUNCH_CHECK();
  int herr = 0;
  QD_CUDA(cudaMemcpyAsync(&herr, err.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaStreamSynchronize(ctx.stream));
  if (herr) fail(QD_ERR_NONFINITE, "null vectors are linearly dependent on an aggregate block");
}

// ---------------------------------------------------------------------------
// Galerkin coarse operator, one CTA per (coarse site x, coarse direction cd):
//   C[x][cd] = sum over fine sites s of x and fine hops h of s whose target
//   t lies across the block face cd (cd = 0: hops inside the block and the
//   site term) of  W[s]^H H_{s,h} W[t].
// Y = H_{s,h} W[t] is formed in shared memory, then contracted with W[s].
// ---------------------------------------------------------------------------

// Full 12-component Wilson hop, chirality-blocked input column w (12):
//   fwd: -1/2 (1 - gamma_mu) U w ; bwd: -1/2 (1 + gamma_mu) U^H w
template <int MU>
__device__ void wilson_hop_full(bool fwd, const cplx* __restrict__ L, const cplx w[12], cplx out[12]) {
  cplx h0[3], h1[3];
  for (int c = 0; c < 3; ++c) {
    cplx b0, b1;
    // B^H applied to (up0, up1)
    const cplx u0 = w[c], u1 = w[3 + c];
    if (MU == 0) { b0 = ctimesi(u1); b1 = ctimesi(u0); }
    else if (MU == 1) { b0 = u1; b1 = mkc(-u0.x, -u0.y); }
    else if (MU == 2) { b0 = ctimesi(u0); b1 = mkc(u1.y, -u1.x); }
    else { b0 = u0; b1 = u1; }
    if (fwd) { h0[c] = csub(w[6 + c], b0); h1[c] = csub(w[9 + c], b1); }
    else     { h0[c] = cadd(w[6 + c], b0); h1[c] = cadd(w[9 + c], b1); }
  }
  cplx g0[3], g1[3];
  for (int a = 0; a < 3; ++a) {
    cplx s0 = mkc(0, 0), s1 = mkc(0, 0);
    for (int b = 0; b < 3; ++b) {
      const cplx l = fwd ? L[a * 3 + b] : cconj(L[b * 3 + a]);
      cfma(s0, l, h0[b]);
      cfma(s1, l, h1[b]);
    }
    g0[a] = s0;
    g1[a] = s1;
  }
  for (int c = 0; c < 3; ++c) {
    cplx b0, b1;  // B applied to (g0, g1)
    if (MU == 0) { b0 = mkc(g1[c].y, -g1[c].x); b1 = mkc(g0[c].y, -g0[c].x); }
    else if (MU == 1) { b0 = mkc(-g1[c].x, -g1[c].y); b1 = g0[c]; }
    else if (MU == 2) { b0 = mkc(g0[c].y, -g0[c].x); b1 = ctimesi(g1[c]); }
    else { b0 = g0[c]; b1 = g1[c]; }
    // fwd: (upper, lower) = (-B g, g); bwd: (B g, g); times -1/2
    const double su = fwd ? 0.5 : -0.5;
    out[c] = cscale(su, b0);
    out[3 + c] = cscale(su, b1);
    out[6 + c] = cscale(-0.5, g0[c]);
    out[9 + c] = cscale(-0.5, g1[c]);
  }
}

__device__ void wilson_hop_any(int mu, bool fwd, const cplx* L, const cplx w[12], cplx out[12]) {
  switch (mu) {
    case 0: wilson_hop_full<0>(fwd, L, w, out); break;
    case 1: wilson_hop_full<1>(fwd, L, w, out); break;
    case 2: wilson_hop_full<2>(fwd, L, w, out); break;
    default: wilson_hop_full<3>(fwd, L, w, out); break;
  }
}

// fine level = Wilson operator (Df = 12)
__global__ void k_coarse_build_wilson(int bsites, int nv, int64_t V, const int* __restrict__ members,
                                      const int8_t* __restrict__ hopdir, const int* __restrict__ nbr,
                                      const cplx* __restrict__ U, const cplx* __restrict__ W,
                                      double mass, double tau, cplx* __restrict__ Cout) {
  extern __shared__ cplx sm[];
  const int Df = 12, Dc = 2 * nv;
  cplx* Y = sm;                 // [12][Dc]
  cplx* Ws = Y + Df * Dc;       // [12][nv]
  cplx* acc = Ws + Df * nv;     // [Dc][Dc]
  const int x = blockIdx.x / 9, cd = blockIdx.x % 9;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int e = tid; e < Dc * Dc; e += nth) acc[e] = mkc(0, 0);
  for (int m = 0; m < bsites; ++m) {
    const int64_t s = members[(int64_t)x * bsites + m];
    for (int h = 0; h <= 8; ++h) {
      if (h < 8 && hopdir[s * 8 + h] != cd) continue;
      if (h == 8 && cd != 0) continue;
      const int64_t t = (h < 8) ? nbr[s * 8 + h] : s;
      __syncthreads();
      for (int e = tid; e < Df * nv; e += nth) Ws[e] = W[s * Df * nv + e];
      for (int dp = tid; dp < Dc; dp += nth) {
        const int chir = dp / nv, j = dp - chir * nv;
        cplx w[12], o[12];
        for (int a = 0; a < 12; ++a)
          w[a] = ((a >= 6) == (chir == 1)) ? W[(t * Df + a) * nv + j] : mkc(0, 0);
        if (h == 8) {
          for (int a = 0; a < 12; ++a) {
            const double te = (a < 6) ? tau : -tau;
            o[a] = cmul(mkc(mass, te), w[a]);
          }
        } else {
          const int mu = h & 3;
          const bool fwd = h < 4;
          const cplx* L = U + ((int64_t)mu * V + (fwd ? s : t)) * 9;
          wilson_hop_any(mu, fwd, L, w, o);
        }
        for (int a = 0; a < 12; ++a) Y[a * Dc + dp] = o[a];
      }
      __syncthreads();
      for (int e = tid; e < Dc * Dc; e += nth) {
        const int d = e / Dc, dp = e - d * Dc;
        const int chir = d / nv, j = d - chir * nv;
        cplx sacc = acc[e];
        for (int a = chir * 6; a < chir * 6 + 6; ++a) cfmac(sacc, Ws[a * nv + j], Y[a * Dc + dp]);
        acc[e] = sacc;
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < Dc * Dc; e += nth) Cout[((int64_t)x * 9 + cd) * Dc * Dc + e] = acc[e];
}

// fine level = coarse stencil of the level above (Df = D of that level)
__global__ void k_coarse_build_coarse(int bsites, int nv, int Df, const int* __restrict__ members,
                                      const int8_t* __restrict__ hopdir, const int* __restrict__ nbr,
                                      const cplx* __restrict__ Cf, const cplx* __restrict__ W,
                                      cplx* __restrict__ Cout) {
  extern __shared__ cplx sm[];
  const int Dc = 2 * nv;
  cplx* Y = sm;               // [Df][Dc]
  cplx* Ws = Y + Df * Dc;     // [Df][nv]
  cplx* acc = Ws + Df * nv;   // [Dc][Dc]
  const int x = blockIdx.x / 9, cd = blockIdx.x % 9;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int half = Df / 2;
  for (int e = tid; e < Dc * Dc; e += nth) acc[e] = mkc(0, 0);
  for (int m = 0; m < bsites; ++m) {
    const int64_t s = members[(int64_t)x * bsites + m];
    for (int h = 0; h <= 8; ++h) {
      if (h < 8 && hopdir[s * 8 + h] != cd) continue;
      if (h == 8 && cd != 0) continue;
      const int64_t t = (h < 8) ? nbr[s * 8 + h] : s;
      const int fdir = (h == 8) ? 0 : (h < 4 ? 1 + h : 5 + (h - 4));
      const cplx* Hm = Cf + ((int64_t)s * 9 + fdir) * Df * Df;
      __syncthreads();
      for (int e = tid; e < Df * nv; e += nth) Ws[e] = W[s * Df * nv + e];
      for (int e = tid; e < Df * Dc; e += nth) {
        const int a = e / Dc, dp = e - a * Dc;
        const int chir = dp / nv, j = dp - chir * nv;
        cplx sacc = mkc(0, 0);
        for (int b = chir * half; b < chir * half + half; ++b)
          cfma(sacc, Hm[a * Df + b], W[(t * Df + b) * nv + j]);
        Y[e] = sacc;
      }
      __syncthreads();
      for (int e = tid; e < Dc * Dc; e += nth) {
        const int d = e / Dc, dp = e - d * Dc;
        const int chir = d / nv, j = d - chir * nv;
        cplx sacc = acc[e];
        for (int a = chir * half; a < chir * half + half; ++a) cfmac(sacc, Ws[a * nv + j], Y[a * Dc + dp]);
        acc[e] = sacc;
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < Dc * Dc; e += nth) Cout[((int64_t)x * 9 + cd) * Dc * Dc + e] = acc[e];
}

void coarse_build_from_wilson(qd_ctx& ctx, const Transfer& T, const qd_gauge& g, double m0,
                              double tau, CoarseLevel& out) {
  const int Dc = T.Dc;
  out.D = Dc;
  out.Cm.resize(out.geo.nsites * 9 * Dc * Dc * sizeof(cplx));
  const size_t smem = ((size_t)12 * Dc + 12 * T.nv + (size_t)Dc * Dc) * sizeof(cplx);
  QD_REQUIRE(smem <= 220 * 1024, "coarse dimension too large for the coarse-build kernel");
  ensure_smem_limit(reinterpret_cast<const void*>(k_coarse_build_wilson), smem);
  k_coarse_build_wilson<<<(int)(out.geo.nsites * 9), 256, smem, ctx.stream>>>(
      T.bsites, T.nv, g.geo.nsites, T.members.as<int>(), T.hopdir.as<int8_t>(), g.geo.nbr.as<int>(),
      g.links.as<cplx>(), T.W.as<cplx>(), 4.0 + m0, tau, out.Cm.as<cplx>());
  QD_LAUNCH_CHECK();
}

void coarse_build_from_coarse(qd_ctx& ctx, const Transfer& T, const CoarseLevel& fine,
                              CoarseLevel& out) {
  const int Dc = T.Dc, Df = T.Df;
  out.D = Dc;
  out.Cm.resize(out.geo.nsites * 9 * Dc * Dc * sizeof(cplx));
  const size_t smem = ((size_t)Df * Dc + (size_t)Df * T.nv + (size_t)Dc * Dc) * sizeof(cplx);
  QD_REQUIRE(smem <= 220 * 1024, "coarse dimension too large for the coarse-build kernel");
  ensure_smem_limit(reinterpret_cast<const void*>(k_coarse_build_coarse), smem);
  k_coarse_build_coarse<<<(int)(out.geo.nsites * 9), 256, smem, ctx.stream>>>(
      T.bsites, T.nv, Df, T.members.as<int>(), T.hopdir.as<int8_t>(), fine.geo.nbr.as<int>(),
      fine.Cm.as<cplx>(), T.W.as<cplx>(), out.Cm.as<cplx>());
  QD_LAUNCH_CHECK();
}

}  // namespace qd
