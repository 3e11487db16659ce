// Drivers: multigrid-preconditioned solves (Sec. 1 inexact solve, Sec. 2)
// and one batch of the deflated Hutchinson estimator (Eq. 1; Algorithms 1
// and 2: t0 + (1/s) sum_j z_j^H A^{-1}_xi (I - P) z_j).
#include "blas.cuh"
#include "coarse_tc.cuh"
#include "restrict_tc.cuh"
#include "defl.cuh"
#include "tc_gemm.cuh"

namespace qd {

// Per-column scales for the refinement: active columns (||r||^2 > tol2
// ||b||^2) get sin = 1/||r||, sout = ||r||; the others 0 (their FP32 system
// has a zero right-hand side and is skipped by the inner solve).
__global__ void k_refine_scales(int s, const cplx* __restrict__ rn2, const cplx* __restrict__ bn2, double tol2,
                                double* __restrict__ sin_, double* __restrict__ sout, int* __restrict__ count) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= s) return;
  const double r = rn2[c].x;
  const bool act = r > tol2 * bn2[c].x;
  sin_[c] = act ? 1.0 / sqrt(r) : 0.0;
  sout[c] = act ? sqrt(r) : 0.0;
  if (act) atomicAdd(count, 1);
}

// out (FP32) = r * sin[c]
__global__ void k_scale_to_f32(int64_t n, int s, const cplx* __restrict__ r, const double* __restrict__ sc,
                               cplxf* __restrict__ out) {
  const int64_t tot = n * s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const double f = sc[e % s];
    out[e] = make_float2((float)(r[e].x * f), (float)(r[e].y * f));
  }
}

// x += e (FP32) * sout[c]
__global__ void k_axpy_from_f32(int64_t n, int s, const cplxf* __restrict__ ev, const double* __restrict__ sc,
                                cplx* __restrict__ x) {
  const int64_t tot = n * s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const double f = sc[e % s];
    if (f == 0.0) continue;
    x[e].x += f * (double)ev[e].x;
    x[e].y += f * (double)ev[e].y;
  }
}

// Mixed precision: FP64 true-residual refinement around FP32 solves.
static void solve_mixed(qd_ctx& ctx, const qd_gauge& g, qd_mg* mg, double m0, double tau, int s, const cplx* b,
                        cplx* x, const qd_solver_params& p, SolveInfo& info) {
  SolverCache& sc = cache(ctx);
  const int64_t n = g.geo.nsites * 12, tot = n * s;
  WilsonOp<cplx> A64(&g, g.links.as<cplx>(), m0, tau, false);
  WilsonOp<cplxf> A32(&g, const_cast<qd_gauge&>(g).links_f32(), m0, tau, false);
  sc.mr.resize(tot * sizeof(cplx));
  sc.mt.resize(tot * sizeof(cplx));
  sc.mrf.resize(tot * sizeof(cplxf));
  sc.mef.resize(tot * sizeof(cplxf));
  sc.mscal.resize((size_t)(4 * s) * sizeof(cplx) + 4 * sizeof(int));
  cplx* r = sc.mr.as<cplx>();
  cplx* t = sc.mt.as<cplx>();
  cplxf* rf = sc.mrf.as<cplxf>();
  cplxf* ef = sc.mef.as<cplxf>();
  cplx* bn2 = sc.mscal.as<cplx>();
  cplx* rn2 = bn2 + s;
  double* sin_ = reinterpret_cast<double*>(rn2 + s);
  double* sout = sin_ + s;
  int* count = reinterpret_cast<int*>(sout + s);
  blas::zero(ctx, tot, x);
  blas::copy(ctx, tot, b, r);
  blas::dots(ctx, 1, n, s, b, 0, b, 0, bn2);
  QD_CUDA(cudaMemcpyAsync(rn2, bn2, s * sizeof(cplx), cudaMemcpyDeviceToDevice, ctx.stream));
  const double tol2 = p.tol * p.tol;
  int inner_total = 0;
  std::vector<int> iters(s, 0);
  for (int step = 0;; ++step) {
    QD_CUDA(cudaMemsetAsync(count, 0, sizeof(int), ctx.stream));
    k_refine_scales<<<div_up(s, 128), 128, 0, ctx.stream>>>(s, rn2, bn2, tol2, sin_, sout, count);
    QD_LAUNCH_CHECK();
    int hc = 0;
    QD_CUDA(cudaMemcpyAsync(&hc, count, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
    QD_CUDA(cudaStreamSynchronize(ctx.stream));
    if (hc == 0 || step >= p.max_refine) break;
    k_scale_to_f32<<<blas::grid_1d(tot), 256, 0, ctx.stream>>>(n, s, r, sin_, rf);
    QD_LAUNCH_CHECK();
    // inner tolerance: inner_tol, relaxed once the residual is close to the
    // target (the FP32 solve need only reach tol ||b|| / ||r||, halved)
    std::vector<cplx> hr(s), hb(s);
    QD_CUDA(cudaMemcpyAsync(hr.data(), rn2, s * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
    QD_CUDA(cudaMemcpyAsync(hb.data(), bn2, s * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
    QD_CUDA(cudaStreamSynchronize(ctx.stream));
    double need = 1.0;
    for (int c = 0; c < s; ++c)
      if (hr[c].x > tol2 * hb[c].x) need = std::min(need, 0.5 * p.tol * std::sqrt(hb[c].x / hr[c].x));
    const double itol = std::min(0.5, std::max(p.inner_tol, need));
    SolveInfo in;
    if (p.schur) {
      // the correction through the odd-site Schur complement
      sc.gcr32s.orth_passes = 1;
      sc.gcr32s.stag_window = p.stag_window;
      sc.spre32.mg = mg ? mg->pre32.get() : nullptr;
      sc.spre32.geo = &g.geo;
      schur_solve<cplxf>(ctx, g, const_cast<qd_gauge&>(g).links_f32(), m0, tau, mg ? &sc.spre32 : nullptr,
                         sc.gcr32s, sc.sch32, rf, ef, s, itol, p.maxit, p.restart, &in);
    } else {
      sc.gcr32.orth_passes = 1;
      sc.gcr32.stag_window = p.stag_window;
      sc.gcr32.solve(ctx, A32, mg ? mg->pre32.get() : nullptr, rf, ef, s, itol, p.maxit, p.restart, &in);
    }
    if (in.stagnated) info.stagnated = true;
    inner_total += in.iterations;
    for (int c = 0; c < s; ++c) iters[c] += in.iters[c];
    k_axpy_from_f32<<<blas::grid_1d(tot), 256, 0, ctx.stream>>>(n, s, ef, sout, x);
    QD_LAUNCH_CHECK();
    A64.residual(ctx, b, x, r, s);
    blas::dots(ctx, 1, n, s, r, 0, r, 0, rn2);
    if (info.stagnated) break;
  }
  {
    const int e = wilson_bulk_error(ctx, g.geo);
    if (e) fail(QD_ERR_TIMEOUT, "FP32 Wilson stencil: bounded wait timed out (code " + std::to_string(e) + ")");
  }
  if (mg && mg->L.back()->tc) {
    const int e = tc_error(ctx, *mg->L.back());
    if (e) fail(QD_ERR_TIMEOUT, "tensor-core coarsest solve: bounded wait timed out (code " + std::to_string(e) + ")");
  }
  if (mg) {
    for (auto& lv : mg->L)
      if (lv->use_tc) {
        const int e = coarse_tc_error(ctx, *lv);
        if (e) fail(QD_ERR_TIMEOUT, "tensor-core coarse stencil: bounded wait timed out (code " + std::to_string(e) + ")");
      }
    for (auto& t : mg->T)
      if (t->use_tc) {
        const int e = restrict_tc_error(ctx, *t);
        if (e) fail(QD_ERR_TIMEOUT, "tensor-core restriction: bounded wait timed out (code " + std::to_string(e) + ")");
      }
  }
  std::vector<cplx> hb(s), hr(s);
  QD_CUDA(cudaMemcpyAsync(hb.data(), bn2, s * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaMemcpyAsync(hr.data(), rn2, s * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaStreamSynchronize(ctx.stream));
  info.iterations = inner_total;
  info.iters = iters;
  info.true_rel.assign(s, 0.0);
  info.converged = 0;
  info.max_rel = 0.0;
  for (int c = 0; c < s; ++c) {
    const double rel = hb[c].x > 0.0 ? std::sqrt(hr[c].x / hb[c].x) : 0.0;
    info.true_rel[c] = rel;
    if (rel <= p.tol) info.converged++;
    if (rel > info.max_rel || rel != rel) info.max_rel = rel;
  }
}

// FP64 even-odd solve: Schur-complement solves of the full residual's
// system until ||b - A x|| <= tol ||b|| per column (the Schur system's own
// residual norm differs from the full one by the even-site scaling).
static void solve_schur64(qd_ctx& ctx, const qd_gauge& g, qd_mg* mg, double m0, double tau, int s, const cplx* b,
                          cplx* x, const qd_solver_params& p, SolveInfo& info) {
  SolverCache& sc = cache(ctx);
  const int64_t n = g.geo.nsites * 12, tot = n * s;
  WilsonOp<cplx> A64(&g, g.links.as<cplx>(), m0, tau, false);
  sc.mr.resize(tot * sizeof(cplx));
  sc.mt.resize(tot * sizeof(cplx));
  sc.mscal.resize((size_t)(4 * s) * sizeof(cplx) + 4 * sizeof(int));
  cplx* r = sc.mr.as<cplx>();
  cplx* e = sc.mt.as<cplx>();
  cplx* bn2 = sc.mscal.as<cplx>();
  cplx* rn2 = bn2 + s;
  blas::zero(ctx, tot, x);
  blas::copy(ctx, tot, b, r);
  blas::dots(ctx, 1, n, s, b, 0, b, 0, bn2);
  QD_CUDA(cudaMemcpyAsync(rn2, bn2, s * sizeof(cplx), cudaMemcpyDeviceToDevice, ctx.stream));
  sc.gcr64s.stag_window = p.stag_window;
  sc.spre64.mg = mg ? mg->pre64.get() : nullptr;
  sc.spre64.geo = &g.geo;
  std::vector<cplx> hb(s), hr(s);
  std::vector<int> iters(s, 0);
  int total = 0;
  const int steps = p.max_refine > 0 ? p.max_refine : 1;
  for (int step = 0; step < steps; ++step) {
    QD_CUDA(cudaMemcpyAsync(hb.data(), bn2, s * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
    QD_CUDA(cudaMemcpyAsync(hr.data(), rn2, s * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
    QD_CUDA(cudaStreamSynchronize(ctx.stream));
    double need = 1.0;
    bool open = false;
    for (int c = 0; c < s; ++c)
      if (hr[c].x > p.tol * p.tol * hb[c].x) {
        open = true;
        need = std::min(need, 0.5 * p.tol * std::sqrt(hb[c].x / hr[c].x));
      }
    if (!open) break;
    SolveInfo in;
    schur_solve<cplx>(ctx, g, g.links.as<cplx>(), m0, tau, mg ? &sc.spre64 : nullptr, sc.gcr64s, sc.sch64, r, e, s,
                      need, p.maxit, p.restart, &in);
    total += in.iterations;
    for (int c = 0; c < s; ++c) iters[c] += in.iters[c];
    blas::add(ctx, tot, e, x);
    A64.residual(ctx, b, x, r, s);
    blas::dots(ctx, 1, n, s, r, 0, r, 0, rn2);
    if (in.stagnated) {
      info.stagnated = true;
      break;
    }
  }
  QD_CUDA(cudaMemcpyAsync(hb.data(), bn2, s * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaMemcpyAsync(hr.data(), rn2, s * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaStreamSynchronize(ctx.stream));
  info.iterations = total;
  info.iters = iters;
  info.true_rel.assign(s, 0.0);
  info.converged = 0;
  info.max_rel = 0.0;
  for (int c = 0; c < s; ++c) {
    const double rel = hb[c].x > 0.0 ? std::sqrt(hr[c].x / hb[c].x) : 0.0;
    info.true_rel[c] = rel;
    if (rel <= p.tol) info.converged++;
    if (rel > info.max_rel || rel != rel) info.max_rel = rel;
  }
}

// x = A^{-1} b for s columns (FP64 GCR + FP64 V-cycle, or mixed precision).
void solve(qd_ctx& ctx, const qd_gauge& g, qd_mg* mg, double m0, double tau, int s, const cplx* b, cplx* x,
           const qd_solver_params& p, SolveInfo& info) {
  if (mg) {
    QD_REQUIRE(mg->gauge == &g, "multigrid hierarchy was built for another gauge field");
    QD_REQUIRE(mg->m0 == m0 && mg->tau == tau, "multigrid hierarchy was built for another m0 / tau");
  }
  QD_REQUIRE(p.tol > 0.0 && p.maxit >= 1 && p.restart >= 1, "bad solver parameters");
  if (p.precision == QD_PREC_MIXED) {
    QD_REQUIRE(p.inner_tol > 0.0 && p.inner_tol < 1.0 && p.max_refine >= 1, "bad mixed-precision parameters");
    solve_mixed(ctx, g, mg, m0, tau, s, b, x, p, info);
    return;
  }
  QD_REQUIRE(p.precision == QD_PREC_F64, "unknown precision");
  WilsonOp<cplx> A(&g, g.links.as<cplx>(), m0, tau, false);
  SolverCache& sc = cache(ctx);
  if (p.schur) {
    solve_schur64(ctx, g, mg, m0, tau, s, b, x, p, info);
    return;
  }
  sc.gcr64.stag_window = p.stag_window;
  sc.gcr64.solve(ctx, A, mg ? mg->pre64.get() : nullptr, b, x, s, p.tol, p.maxit, p.restart, &info);
}

// Spin-colour dilution: column 12 j + h of Zd is column j of Z restricted to
// the components a = 3 spin + colour equal to h (layout (site, a, column)).
__global__ void k_dilute(int64_t nsites, int s, const cplx* __restrict__ Z, cplx* __restrict__ Zd) {
  const int64_t tot = nsites * 12 * (int64_t)s * 12;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(e % (12 * s));
    const int64_t sa = e / (12 * s);
    const int a = (int)(sa % 12);
    const int j = col / 12, h = col - 12 * j;
    Zd[e] = (a == h) ? Z[sa * s + j] : mkc(0.0, 0.0);
  }
}

// t[j] = sum_h td[12 j + h] in order h = 0..11
__global__ void k_sum_dilution(int s, const cplx* __restrict__ td, cplx* __restrict__ t) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s) return;
  cplx acc = mkc(0.0, 0.0);
  for (int h = 0; h < 12; ++h) acc = cadd(acc, td[12 * j + h]);
  t[j] = acc;
}

void hutchinson(qd_ctx& ctx, const qd_gauge& g, qd_mg* mg, qd_defl* d, double m0, double tau,
                const qd_trace_params& p, bool want_coeffs, TraceOut& out, std::vector<cplx>* M1,
                std::vector<cplx>* M2) {
  const int s = p.nsamples;
  QD_REQUIRE(s >= 1, "nsamples must be >= 1");
  if (d) QD_REQUIRE(d->gauge == &g && d->m0 == m0 && d->tau == tau, "deflation space built for another operator");
  const bool dil = p.dilution == 12;
  const int nc = dil ? 12 * s : s;  // right-hand sides solved
  const int64_t n = g.geo.nsites * 12;
  SolverCache& sc = cache(ctx);
  const size_t vb = (size_t)n * nc * sizeof(cplx);
  sc.Z.resize(vb);
  sc.B.resize(vb);
  sc.X.resize(vb);
  sc.tdev.resize((size_t)nc * sizeof(cplx));
  sc.stats.resize(8 * sizeof(double));
  sc.loo.resize((size_t)s * sizeof(double));
  cplx* Z = sc.Z.as<cplx>();
  cplx* B = sc.B.as<cplx>();
  cplx* X = sc.X.as<cplx>();
  // a1: noise (diluted: the s samples are made in B, then split into Z)
  if (dil) {
    rademacher_fill(ctx, g.geo, p.seed, p.sample_offset, s, B);
    k_dilute<<<blas::grid_1d(n * nc), 256, 0, ctx.stream>>>(g.geo.nsites, s, B, Z);
    QD_LAUNCH_CHECK();
  } else {
    rademacher_fill(ctx, g.geo, p.seed, p.sample_offset, s, Z);
  }
  // a8: deflated right-hand sides
  if (d)
    defl_project(ctx, *d, nc, Z, B);
  else
    blas::copy(ctx, n * nc, Z, B);
  // a5/a6: solves
  solve(ctx, g, mg, m0, tau, nc, B, X, p.solver, out.info);
  // a9: t_j = z_j^H x_j (summed over the diluted parts), statistics
  if (dil) {
    DevBuf td((size_t)nc * sizeof(cplx));
    blas::dots(ctx, 1, n, nc, Z, 0, X, 0, td.as<cplx>());
    k_sum_dilution<<<div_up(s, 128), 128, 0, ctx.stream>>>(s, td.as<cplx>(), sc.tdev.as<cplx>());
    QD_LAUNCH_CHECK();
    QD_CUDA(cudaStreamSynchronize(ctx.stream));  // td goes out of scope
  } else {
    blas::dots(ctx, 1, n, s, Z, 0, X, 0, sc.tdev.as<cplx>());
  }
  trace_stats(ctx, s, sc.tdev.as<cplx>(), sc.stats.as<double>(), sc.loo.as<double>());
  out.t.resize(s);
  QD_CUDA(cudaMemcpyAsync(out.stats, sc.stats.as<double>(), 6 * sizeof(double), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaMemcpyAsync(out.t.data(), sc.tdev.as<cplx>(), s * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
  if (want_coeffs && d && !dil) {
    const int k = d->p.k;
    DevBuf m1((size_t)k * s * sizeof(cplx)), m2((size_t)k * s * sizeof(cplx));
    defl_coeffs(ctx, *d, s, Z, m1.as<cplx>(), m2.as<cplx>());
    M1->resize((size_t)k * s);
    M2->resize((size_t)k * s);
    QD_CUDA(cudaMemcpyAsync(M1->data(), m1.as<cplx>(), (size_t)k * s * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
    QD_CUDA(cudaMemcpyAsync(M2->data(), m2.as<cplx>(), (size_t)k * s * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
  }
  QD_CUDA(cudaStreamSynchronize(ctx.stream));
}

}  // namespace qd
