// Drivers: multigrid-preconditioned solves (Sec. 1 inexact solve, Sec. 2)
// and one batch of the deflated Hutchinson estimator (Eq. 1; Algorithms 1
// and 2: t0 + (1/s) sum_j z_j^H A^{-1}_xi (I - P) z_j).
#include "blas.cuh"
#include "defl.cuh"

namespace qd {

// x = A^{-1} b for s columns, FP64 flexible GCR right-preconditioned by the
// FP64 V-cycle (mg) or unpreconditioned.
void solve(qd_ctx& ctx, const qd_gauge& g, qd_mg* mg, double m0, double tau, int s, const cplx* b, cplx* x,
           double tol, int maxit, int restart, SolveInfo& info) {
  if (mg) {
    QD_REQUIRE(mg->gauge == &g, "multigrid hierarchy was built for another gauge field");
    QD_REQUIRE(mg->m0 == m0 && mg->tau == tau, "multigrid hierarchy was built for another m0 / tau");
  }
  WilsonOp<cplx> A(&g, g.links.as<cplx>(), m0, tau, false);
  SolverCache& sc = cache(ctx);
  sc.gcr64.solve(ctx, A, mg ? mg->pre64.get() : nullptr, b, x, s, tol, maxit, restart, &info);
}


void hutchinson(qd_ctx& ctx, const qd_gauge& g, qd_mg* mg, qd_defl* d, double m0, double tau,
                const qd_trace_params& p, bool want_coeffs, TraceOut& out, std::vector<cplx>* M1,
                std::vector<cplx>* M2) {
  const int s = p.nsamples;
  QD_REQUIRE(s >= 1, "nsamples must be >= 1");
  if (d) QD_REQUIRE(d->gauge == &g && d->m0 == m0 && d->tau == tau, "deflation space built for another operator");
  const int64_t n = g.geo.nsites * 12;
  SolverCache& sc = cache(ctx);
  const size_t vb = (size_t)n * s * sizeof(cplx);
  sc.Z.resize(vb);
  sc.B.resize(vb);
  sc.X.resize(vb);
  sc.tdev.resize((size_t)s * sizeof(cplx));
  sc.stats.resize(8 * sizeof(double));
  sc.loo.resize((size_t)s * sizeof(double));
  cplx* Z = sc.Z.as<cplx>();
  cplx* B = sc.B.as<cplx>();
  cplx* X = sc.X.as<cplx>();
  // a1: noise
  rademacher_fill(ctx, g.geo, p.seed, p.sample_offset, s, Z);
  // a8: deflated right-hand sides
  if (d)
    defl_project(*d, s, Z, B);
  else
    blas::copy(ctx, n * s, Z, B);
  // a5/a6: solves
  solve(ctx, g, mg, m0, tau, s, B, X, p.tol, p.maxit, p.restart, out.info);
  // a9: t_j = z_j^H x_j, statistics
  blas::dots(ctx, 1, n, s, Z, 0, X, 0, sc.tdev.as<cplx>());
  trace_stats(ctx, s, sc.tdev.as<cplx>(), sc.stats.as<double>(), sc.loo.as<double>());
  out.t.resize(s);
  QD_CUDA(cudaMemcpyAsync(out.stats, sc.stats.as<double>(), 6 * sizeof(double), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaMemcpyAsync(out.t.data(), sc.tdev.as<cplx>(), s * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
  if (want_coeffs && d && d->kind == QD_DEFL_MG_OBLIQUE) {
    const int k = d->p.k;
    DevBuf m1((size_t)k * s * sizeof(cplx)), m2((size_t)k * s * sizeof(cplx));
    defl_coeffs(*d, s, Z, m1.as<cplx>(), m2.as<cplx>());
    M1->resize((size_t)k * s);
    M2->resize((size_t)k * s);
    QD_CUDA(cudaMemcpyAsync(M1->data(), m1.as<cplx>(), (size_t)k * s * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
    QD_CUDA(cudaMemcpyAsync(M2->data(), m2.as<cplx>(), (size_t)k * s * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
  }
  QD_CUDA(cudaStreamSynchronize(ctx.stream));
}

}  // namespace qd
