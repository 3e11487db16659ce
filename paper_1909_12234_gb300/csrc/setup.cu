// Adaptive multigrid setup (Sec. 2; Algorithm 2 step 1): per level, null
// vectors from minimal-residual iterations on A y = 0 started at Philox
// random vectors (stop at relative residual null_tol or null_maxit steps,
// Sec. 4), chirality split + blocking + per-block CGS2 -> W, then the
// Galerkin coarse operator W^H A W.
#include "blas.cuh"
#include "coarse_tc.cuh"
#include "restrict_tc.cuh"
#include "direct.cuh"
#include "mg.cuh"
#include "tc_gemm.cuh"

namespace qd {

void mg_build(qd_mg& mg, const double* injected_null) {
  qd_ctx& ctx = *mg.ctx;
  const qd_mg_params& p = mg.p;
  QD_REQUIRE(p.nlevels >= 1 && p.nlevels < QD_MAX_LEVELS, "nlevels must be in [1, QD_MAX_LEVELS-1]");
  mg.nlevels = p.nlevels;
  for (int l = 0; l < p.nlevels; ++l) {
    QD_REQUIRE(p.nv[l] >= 1 && p.nv[l] <= 64, "nv must be in [1, 64]");
    const LevelGeom& fg = mg.geom(l);
    const int Df = mg.dof(l);
    std::unique_ptr<Transfer> T(new Transfer());
    std::unique_ptr<CoarseLevel> CL(new CoarseLevel());
    T->nv = p.nv[l];
    T->Df = Df;
    T->Dc = 2 * p.nv[l];
    build_transfer_tables(*T, fg, p.block[l], CL->geo);
    const int nv = T->nv;
    const int64_t n = fg.nsites * (int64_t)Df;
    DevBuf Y(n * nv * sizeof(cplx)), Y0(n * nv * sizeof(cplx)), R(n * nv * sizeof(cplx)),
        Qb(n * nv * sizeof(cplx)), steps(nv * sizeof(int)), scratch;
    T->null_steps.assign(nv, 0);
    if (l == 0 && injected_null) {
      QD_CUDA(cudaMemcpyAsync(Y.as<cplx>(), injected_null, n * nv * sizeof(cplx), cudaMemcpyDeviceToDevice,
                              ctx.stream));
    } else {
      random_starts_fill(ctx, fg, Df, p.seed + (uint64_t)l, nv, Y0.as<cplx>());
      QD_CUDA(cudaMemsetAsync(steps.as<int>(), 0, nv * sizeof(int), ctx.stream));
      QD_CUDA(cudaMemcpyAsync(Y.as<cplx>(), Y0.as<cplx>(), n * nv * sizeof(cplx), cudaMemcpyDeviceToDevice,
                              ctx.stream));
      DevBuf zero(n * nv * sizeof(cplx));
      QD_CUDA(cudaMemsetAsync(zero.as<cplx>(), 0, n * nv * sizeof(cplx), ctx.stream));
      if (p.null_f32) {
        // the same iteration with FP32 operators and vectors
        DevBuf Yf(n * nv * sizeof(cplxf)), Rf(n * nv * sizeof(cplxf)), Qf(n * nv * sizeof(cplxf)),
            zf(n * nv * sizeof(cplxf));
        to_f32(ctx, Y.as<cplx>(), Yf.as<cplxf>(), n * nv);
        QD_CUDA(cudaMemsetAsync(zf.as<cplxf>(), 0, n * nv * sizeof(cplxf), ctx.stream));
        auto A = mg.op<cplxf>(l);
        mr_steps<cplxf>(ctx, *A, zf.as<cplxf>(), Yf.as<cplxf>(), false, nv, p.null_maxit, p.null_tol,
                        Rf.as<cplxf>(), Qf.as<cplxf>(), steps.as<int>(), scratch);
        to_f64(ctx, Yf.as<cplxf>(), Y.as<cplx>(), n * nv);
      } else {
        auto A = mg.op<cplx>(l);
        mr_steps<cplx>(ctx, *A, zero.as<cplx>(), Y.as<cplx>(), false, nv, p.null_maxit, p.null_tol,
                       R.as<cplx>(), Qb.as<cplx>(), steps.as<int>(), scratch);
      }
      QD_CUDA(cudaMemcpyAsync(T->null_steps.data(), steps.as<int>(), nv * sizeof(int), cudaMemcpyDeviceToHost,
                              ctx.stream));
    }
    block_orthonormalize(ctx, *T, Y.as<cplx>());
    mg.T.push_back(std::move(T));
    if (l == 0)
      coarse_build_from_wilson(ctx, *mg.T[0], *mg.gauge, mg.m0, mg.tau, *CL);
    else
      coarse_build_from_coarse(ctx, *mg.T[l], *mg.L[l - 1], *CL);
    mg.L.push_back(std::move(CL));
    QD_CUDA(cudaStreamSynchronize(ctx.stream));
  }
  // coarsest level: dense FP64 inverse when small enough
  CoarseLevel& last = *mg.L.back();
  const int64_t nlast = last.geo.nsites * (int64_t)last.D;
  if (p.coarsest_direct > 0 && nlast <= p.coarsest_direct && nlast <= 16384) {
    coarse_dense_inverse(ctx, last);
    if (p.coarsest_bf16) {
      tc_prepare(ctx, last);
      last.tc = true;
    }
  }
  // tensor-core coarse stencils for the FP32 V-cycle where the shape allows
  for (auto& lv : mg.L) {
    lv->use_tc = p.coarse_tc != 0 && (lv->D == 8 || lv->D == 16 || lv->D == 24 || lv->D == 32);
    if (lv->use_tc) coarse_tc_prepare(ctx, *lv);
  }
  for (auto& t : mg.T) {
    t->use_tc = p.coarse_tc != 0 && (t->Df == 12 || t->Df == 16 || t->Df == 24 || t->Df == 32) &&
                (t->Dc == 16 || t->Dc == 24 || t->Dc == 32);
    if (t->use_tc) restrict_tc_prepare(ctx, *t);
  }
  mg.pre64.reset(new MGPrecond<cplx>(&mg, 0));
  mg.pre32.reset(new MGPrecond<cplxf>(&mg, 0));
}

}  // namespace qd
