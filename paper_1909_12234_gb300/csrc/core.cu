// Geometry tables, gauge import, field reordering and the counter-based
// random fields: Rademacher noise (Sec. 1, the x_j of Eq. 1) and the random
// starts of the adaptive multigrid setup (Sec. 2).
#include <algorithm>
#include <utility>
#include <vector>

#include "qd_internal.cuh"

namespace qd {

// ---------------------------------------------------------------------------
// Geometry
// ---------------------------------------------------------------------------
void LevelGeom::build(const int d[4], bool even_odd) {
  nsites = 1;
  for (int m = 0; m < 4; ++m) {
    QD_REQUIRE(d[m] >= 1, "lattice extents must be >= 1");
    dims[m] = d[m];
    nsites *= d[m];
  }
  QD_REQUIRE(nsites < (1LL << 31) / 12, "lattice too large for 32-bit site tables");
  eo = even_odd;
  if (eo) QD_REQUIRE(dims[0] % 2 == 0, "even-odd ordering needs an even Lx");
  const int64_t V = nsites;
  h_lex_of_site.assign(V, 0);
  h_site_of_lex.assign(V, 0);
  for (int64_t l = 0; l < V; ++l) {
    int64_t s = l;
    if (eo) {
      int c[4];
      coords(l, c);
      const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
      s = par * (V / 2) + l / 2;
    }
    h_site_of_lex[l] = (int)s;
    h_lex_of_site[s] = (int)l;
  }
  h_nbr.assign(V * 8, 0);
  for (int64_t s = 0; s < V; ++s) {
    int c[4];
    coords(h_lex_of_site[s], c);
    for (int mu = 0; mu < 4; ++mu) {
      int cp[4] = {c[0], c[1], c[2], c[3]}, cm[4] = {c[0], c[1], c[2], c[3]};
      cp[mu] = (c[mu] + 1) % dims[mu];
      cm[mu] = (c[mu] - 1 + dims[mu]) % dims[mu];
      h_nbr[s * 8 + mu] = h_site_of_lex[lex(cp)];
      h_nbr[s * 8 + 4 + mu] = h_site_of_lex[lex(cm)];
    }
  }
  // 4^4 tiles in lexicographic tile order, Morton order (coordinate bits
  // interleaved) inside a tile; the key is injective, so no ties
  int tdim[4];
  for (int m = 0; m < 4; ++m) tdim[m] = (dims[m] + 3) / 4;
  std::vector<std::pair<uint64_t, int>> key(V);
  for (int64_t s = 0; s < V; ++s) {
    int c[4];
    coords(h_lex_of_site[s], c);
    const uint64_t tile = (uint64_t)(c[0] / 4) +
                          (uint64_t)tdim[0] * ((c[1] / 4) + (uint64_t)tdim[1] * ((c[2] / 4) + (uint64_t)tdim[2] * (c[3] / 4)));
    uint64_t in = 0;
    for (int b = 0; b < 2; ++b)
      for (int m = 0; m < 4; ++m) in |= (uint64_t)((c[m] >> b) & 1) << (4 * b + m);
    key[s] = {(tile << 8) | in, (int)s};
  }
  std::sort(key.begin(), key.end());
  h_visit.resize(V);
  for (int64_t k = 0; k < V; ++k) h_visit[k] = key[k].second;
  visit.resize(V * sizeof(int));
  QD_CUDA(cudaMemcpy(visit.as<int>(), h_visit.data(), V * sizeof(int), cudaMemcpyHostToDevice));
  if (eo) {
    for (int par = 0; par < 2; ++par) {
      std::vector<int> vp;
      vp.reserve(V / 2);
      for (int64_t k = 0; k < V; ++k)
        if ((h_visit[k] >= V / 2) == (par == 1)) vp.push_back(h_visit[k]);
      visit_par[par].resize(vp.size() * sizeof(int));
      QD_CUDA(cudaMemcpy(visit_par[par].as<int>(), vp.data(), vp.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
  }
  bulk_err.resize(sizeof(int));
  QD_CUDA(cudaMemset(bulk_err.as<int>(), 0, sizeof(int)));
  nbr.resize(V * 8 * sizeof(int));
  lex_of_site.resize(V * sizeof(int));
  site_of_lex.resize(V * sizeof(int));
  QD_CUDA(cudaMemcpy(nbr.as<int>(), h_nbr.data(), V * 8 * sizeof(int), cudaMemcpyHostToDevice));
  QD_CUDA(cudaMemcpy(lex_of_site.as<int>(), h_lex_of_site.data(), V * sizeof(int),
                     cudaMemcpyHostToDevice));
  QD_CUDA(cudaMemcpy(site_of_lex.as<int>(), h_site_of_lex.data(), V * sizeof(int),
                     cudaMemcpyHostToDevice));
}

// ---------------------------------------------------------------------------
// Gauge import: host [V lex][4][9] -> device [4][V eo][9]
// ---------------------------------------------------------------------------
__global__ void k_gauge_permute(int64_t V, const int* __restrict__ lex_of_site,
                                const cplx* __restrict__ src, cplx* __restrict__ dst) {
  const int64_t tot = 4 * V * 9;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % 9);
    const int64_t ms = e / 9;
    const int64_t s = ms % V;
    const int mu = (int)(ms / V);
    dst[e] = src[((int64_t)lex_of_site[s] * 4 + mu) * 9 + k];
  }
}

void gauge_import(qd_ctx& ctx, qd_gauge& g, const double* links_host) {
  const int64_t V = g.geo.nsites;
  const size_t bytes = (size_t)4 * V * 9 * sizeof(cplx);
  DevBuf staging(bytes);
  g.links.resize(bytes);
  QD_CUDA(cudaMemcpyAsync(staging.as<cplx>(), links_host, bytes, cudaMemcpyHostToDevice, ctx.stream));
  k_gauge_permute<<<div_up(4 * V * 9, 256), 256, 0, ctx.stream>>>(V, g.geo.lex_of_site.as<int>(),
                                                                 staging.as<cplx>(), g.links.as<cplx>());
  QD_LAUNCH_CHECK();
  QD_CUDA(cudaStreamSynchronize(ctx.stream));
}

// ---------------------------------------------------------------------------
// Field reorder: canonical [r][V lex][12] <-> qd [V eo][12][r]
// ---------------------------------------------------------------------------
__global__ void k_reorder(int64_t V, int nrhs, int to_qd, const int* __restrict__ lex_of_site,
                          const cplx* __restrict__ in, cplx* __restrict__ out) {
  const int64_t tot = V * 12 * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % nrhs);
    const int64_t sa = e / nrhs;
    const int a = (int)(sa % 12);
    const int64_t s = sa / 12;
    const int64_t c = ((int64_t)r * V + lex_of_site[s]) * 12 + a;
    if (to_qd)
      out[e] = in[c];
    else
      out[c] = in[e];
  }
}

void field_reorder(qd_ctx& ctx, const LevelGeom& geo, int nrhs, bool to_qd, const cplx* in,
                   cplx* out) {
  const int64_t tot = geo.nsites * 12 * nrhs;
  k_reorder<<<div_up(tot, 256), 256, 0, ctx.stream>>>(geo.nsites, nrhs, to_qd ? 1 : 0,
                                                     geo.lex_of_site.as<int>(), in, out);
  QD_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// Rademacher noise.  One thread per (site, column): the 12 dofs of lex site l
// are i = 12 l .. 12 l + 11, spread over at most two 128-bit Philox blocks.
// ---------------------------------------------------------------------------
__global__ void k_rademacher(int64_t V, int nrhs, const int* __restrict__ lex_of_site,
                             uint32_t k0, uint32_t k1, uint32_t sample0, cplx* __restrict__ out) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= V * nrhs) return;
  const int64_t s = g / nrhs;
  const int r = (int)(g - s * nrhs);
  const uint32_t sample = sample0 + (uint32_t)r;
  const int64_t i0 = 12LL * lex_of_site[s];
  const uint32_t blk0 = (uint32_t)(i0 >> 7);
  U4 c0 = {{blk0, sample, 0u, 0u}};
  U4 w0 = philox4x32_10(c0, k0, k1);
  U4 c1 = {{blk0 + 1u, sample, 0u, 0u}};
  const bool two = ((i0 + 11) >> 7) != (int64_t)blk0;
  U4 w1 = w0;
  if (two) w1 = philox4x32_10(c1, k0, k1);
#pragma unroll
  for (int a = 0; a < 12; ++a) {
    const int64_t i = i0 + a;
    const U4& w = ((uint32_t)(i >> 7) == blk0) ? w0 : w1;
    const int pos = (int)(i & 127);
    const uint32_t bit = (w.v[pos >> 5] >> (pos & 31)) & 1u;
    out[(s * 12 + a) * nrhs + r] = mkc(bit ? -1.0 : 1.0, 0.0);
  }
}

void rademacher_fill(qd_ctx& ctx, const LevelGeom& geo, uint64_t seed, int64_t sample_offset,
                     int nrhs, cplx* out) {
  QD_REQUIRE(sample_offset >= 0 && sample_offset + nrhs <= (1LL << 32),
             "sample indices must lie in [0, 2^32)");
  const int64_t tot = geo.nsites * nrhs;
  k_rademacher<<<div_up(tot, 128), 128, 0, ctx.stream>>>(
      geo.nsites, nrhs, geo.lex_of_site.as<int>(), (uint32_t)(seed & 0xffffffffu),
      (uint32_t)(seed >> 32), (uint32_t)sample_offset, out);
  QD_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// Random starts for the adaptive setup: dof i = lex_site * dof + d takes
// re from bit 2 (i mod 64) and im from the next bit of
// Philox(counter = (i / 64, v, 1, 0)); bit 0 -> +1, 1 -> -1.
// ---------------------------------------------------------------------------
__global__ void k_random_starts(int64_t nsites, int dof, int nvec, const int* __restrict__ lex_of_site,
                                uint32_t k0, uint32_t k1, cplx* __restrict__ out) {
  const int64_t tot = nsites * dof * nvec;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int v = (int)(e % nvec);
    const int64_t sd = e / nvec;
    const int d = (int)(sd % dof);
    const int64_t s = sd / dof;
    const int64_t i = (int64_t)lex_of_site[s] * dof + d;
    U4 c = {{(uint32_t)(i >> 6), (uint32_t)v, 1u, 0u}};
    U4 w = philox4x32_10(c, k0, k1);
    const int pos = 2 * (int)(i & 63);
    const uint32_t word = w.v[pos >> 5];
    const uint32_t bre = (word >> (pos & 31)) & 1u;
    const uint32_t bim = (word >> ((pos + 1) & 31)) & 1u;
    out[e] = mkc(bre ? -1.0 : 1.0, bim ? -1.0 : 1.0);
  }
}

void random_starts_fill(qd_ctx& ctx, const LevelGeom& geo, int dof, uint64_t key, int nvec,
                        cplx* out) {
  const int64_t tot = geo.nsites * dof * nvec;
  k_random_starts<<<div_up(tot, 256), 256, 0, ctx.stream>>>(
      geo.nsites, dof, nvec, geo.lex_of_site.as<int>(), (uint32_t)(key & 0xffffffffu),
      (uint32_t)(key >> 32), out);
  QD_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// Precision conversion.
// ---------------------------------------------------------------------------
__global__ void k_to_f32(int64_t n, const cplx* __restrict__ in, cplxf* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = make_float2((float)in[e].x, (float)in[e].y);
}
__global__ void k_to_f64(int64_t n, const cplxf* __restrict__ in, cplx* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = mkc((double)in[e].x, (double)in[e].y);
}
void to_f32(qd_ctx& ctx, const cplx* in, cplxf* out, int64_t n) {
  k_to_f32<<<div_up(n, 256) < 8192 ? div_up(n, 256) : 8192, 256, 0, ctx.stream>>>(n, in, out);
  QD_LAUNCH_CHECK();
}
void to_f64(qd_ctx& ctx, const cplxf* in, cplx* out, int64_t n) {
  k_to_f64<<<div_up(n, 256) < 8192 ? div_up(n, 256) : 8192, 256, 0, ctx.stream>>>(n, in, out);
  QD_LAUNCH_CHECK();
}
void links_to_f32(qd_ctx& ctx, const cplx* in, cplxf* out, int64_t n) { to_f32(ctx, in, out, n); }

}  // namespace qd

const qd::cplxf* qd_gauge::links_f32() {
  if (linksf.bytes() == 0) {
    const int64_t n = 4 * geo.nsites * 9;
    linksf.resize(n * sizeof(qd::cplxf));
    qd::links_to_f32(*ctx, links.as<qd::cplx>(), linksf.as<qd::cplxf>(), n);
  }
  return linksf.as<qd::cplxf>();
}
