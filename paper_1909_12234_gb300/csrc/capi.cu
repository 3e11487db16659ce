// extern "C" entry points of libqdtrace (declared in include/qdtrace.h).
// Every function catches internal errors and returns a qd_status code; the
// message is kept per host thread for qd_last_error().
#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>

#include "blas.cuh"
#include "coarse_tc.cuh"
#include "restrict_tc.cuh"
#include "defl.cuh"
#include "direct.cuh"
#include "tc_gemm.cuh"
#include "tune.cuh"


static thread_local std::string g_last_error;

template <class F> static int guarded(F&& f) {
  try {
    g_last_error.clear();
    f();
    return QD_OK;
  } catch (const qd::Error& e) {
    g_last_error = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return QD_ERR_OOM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return QD_ERR_INTERNAL;
  } catch (...) {
    g_last_error = "unknown error";
    return QD_ERR_INTERNAL;
  }
}

#define NONNULL(p) QD_REQUIRE((p) != nullptr, #p " must not be NULL")

static void set_device(const qd_ctx* c) { QD_CUDA(cudaSetDevice(c->device)); }

// Whether two byte ranges [a, a + bytes) and [b, b + bytes) share a byte.
static bool overlaps(const void* a, const void* b, size_t bytes) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + bytes && y < x + bytes;
}

extern "C" {

int qd_abi_version(void) { return QD_ABI_VERSION; }

const char* qd_last_error(void) { return g_last_error.c_str(); }

int qd_ctx_create(qd_ctx** ctx, int device, void* stream) {
  return guarded([&] {
    NONNULL(ctx);
    int ndev = 0;
    QD_CUDA(cudaGetDeviceCount(&ndev));
    QD_REQUIRE(device >= 0 && device < ndev, "no such CUDA device");
    QD_CUDA(cudaSetDevice(device));
    std::unique_ptr<qd_ctx> c(new qd_ctx());
    c->device = device;
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    QD_CUDA(cudaMallocHost(&c->host_pinned, 64 * sizeof(int)));
    // qd_deflate_project_static's array: loaded and looked up now, per
    // context (a device reset between contexts moves it)
    c->static_scratch = qd::static_scratch_resolve();
    *ctx = c.release();
  });
}

int qd_ctx_destroy(qd_ctx* ctx) {
  return guarded([&] {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
    for (auto& p : ctx->prof_pending) {
      cudaEventDestroy(p.e0);
      cudaEventDestroy(p.e1);
    }
    for (auto e : ctx->prof_pool) cudaEventDestroy(e);
    delete ctx;
  });
}

int qd_eo_index(const int dims[4], int64_t* eo_of_lex) {
  return guarded([&] {
    NONNULL(dims);
    NONNULL(eo_of_lex);
    int64_t V = 1;
    for (int m = 0; m < 4; ++m) {
      QD_REQUIRE(dims[m] >= 1, "lattice extents must be >= 1");
      V *= dims[m];
    }
    QD_REQUIRE(dims[0] % 2 == 0, "even-odd ordering needs an even Lx");
    for (int64_t l = 0; l < V; ++l) {
      const int64_t x = l % dims[0], y = (l / dims[0]) % dims[1];
      const int64_t z = (l / ((int64_t)dims[0] * dims[1])) % dims[2];
      const int64_t t = l / ((int64_t)dims[0] * dims[1] * dims[2]);
      eo_of_lex[l] = ((x + y + z + t) & 1) * (V / 2) + l / 2;
    }
  });
}

int qd_gauge_create(qd_ctx* ctx, const int dims[4], const double* links_host, qd_gauge** gauge) {
  return guarded([&] {
    NONNULL(ctx);
    NONNULL(dims);
    NONNULL(links_host);
    NONNULL(gauge);
    set_device(ctx);
    std::unique_ptr<qd_gauge> g(new qd_gauge());
    g->ctx = ctx;
    g->geo.build(dims, true);
    qd::gauge_import(*ctx, *g, links_host);
    *gauge = g.release();
  });
}

int qd_gauge_destroy(qd_gauge* gauge) {
  return guarded([&] {
    if (!gauge) return;
    cudaStreamSynchronize(gauge->ctx->stream);
    delete gauge;
  });
}

int qd_field_reorder(qd_ctx* ctx, const qd_gauge* gauge, int nrhs, int to_qd, const double* in, double* out) {
  return guarded([&] {
    NONNULL(ctx);
    NONNULL(gauge);
    NONNULL(in);
    NONNULL(out);
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    QD_REQUIRE(in != out, "in and out must not overlap");
    set_device(ctx);
    qd::field_reorder(*ctx, gauge->geo, nrhs, to_qd != 0, reinterpret_cast<const qd::cplx*>(in),
                      reinterpret_cast<qd::cplx*>(out));
  });
}

int qd_rademacher(qd_ctx* ctx, const qd_gauge* gauge, uint64_t seed, int64_t sample_offset, int nrhs, double* out) {
  return guarded([&] {
    NONNULL(ctx);
    NONNULL(gauge);
    NONNULL(out);
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    set_device(ctx);
    qd::rademacher_fill(*ctx, gauge->geo, seed, sample_offset, nrhs, reinterpret_cast<qd::cplx*>(out));
  });
}

int qd_dirac_apply(qd_ctx* ctx, const qd_gauge* gauge, double m0, double tau, int dagger, int nrhs,
                   const double* in, double* out) {
  return guarded([&] {
    NONNULL(ctx);
    NONNULL(gauge);
    NONNULL(in);
    NONNULL(out);
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    QD_REQUIRE(in != out, "in and out must not overlap");
    QD_REQUIRE(std::isfinite(m0) && std::isfinite(tau), "m0 and tau must be finite");
    set_device(ctx);
    qd::wilson_apply<qd::cplx>(*ctx, gauge->geo, gauge->links.as<qd::cplx>(), m0, tau, dagger != 0,
                               reinterpret_cast<const qd::cplx*>(in), reinterpret_cast<qd::cplx*>(out), nrhs);
  });
}

int qd_dirac_apply_f32(qd_ctx* ctx, qd_gauge* gauge, double m0, double tau, int dagger, int nrhs, const float* in,
                       float* out) {
  return guarded([&] {
    NONNULL(ctx);
    NONNULL(gauge);
    NONNULL(in);
    NONNULL(out);
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    QD_REQUIRE(in != out, "in and out must not overlap");
    QD_REQUIRE(std::isfinite(m0) && std::isfinite(tau), "m0 and tau must be finite");
    set_device(ctx);
    qd::wilson_apply<qd::cplxf>(*ctx, gauge->geo, gauge->links_f32(), m0, tau, dagger != 0,
                                reinterpret_cast<const qd::cplxf*>(in), reinterpret_cast<qd::cplxf*>(out), nrhs);
  });
}

int qd_dirac_residual_f32(qd_ctx* ctx, qd_gauge* gauge, double m0, double tau, int dagger, int nrhs, const float* b,
                          const float* x, float* r) {
  return guarded([&] {
    NONNULL(ctx);
    NONNULL(gauge);
    NONNULL(b);
    NONNULL(x);
    NONNULL(r);
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    const size_t bytes = (size_t)gauge->geo.nsites * 12 * nrhs * sizeof(qd::cplxf);
    QD_REQUIRE(!overlaps(r, x, bytes) && !overlaps(r, b, bytes), "r must not overlap b or x");
    QD_REQUIRE(std::isfinite(m0) && std::isfinite(tau), "m0 and tau must be finite");
    set_device(ctx);
    qd::wilson_apply<qd::cplxf>(*ctx, gauge->geo, gauge->links_f32(), m0, tau, dagger != 0,
                                reinterpret_cast<const qd::cplxf*>(x), reinterpret_cast<qd::cplxf*>(r), nrhs,
                                reinterpret_cast<const qd::cplxf*>(b));
  });
}

int qd_dirac_schur_apply(qd_ctx* ctx, const qd_gauge* gauge, double m0, double tau, int nrhs, const double* in,
                         double* out) {
  return guarded([&] {
    NONNULL(ctx);
    NONNULL(gauge);
    NONNULL(in);
    NONNULL(out);
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    QD_REQUIRE(in != out, "in and out must not overlap");
    QD_REQUIRE(std::isfinite(m0) && std::isfinite(tau), "m0 and tau must be finite");
    set_device(ctx);
    qd::SchurOp<qd::cplx> S(gauge, gauge->links.as<qd::cplx>(), m0, tau);
    S.apply(*ctx, reinterpret_cast<const qd::cplx*>(in), reinterpret_cast<qd::cplx*>(out), nrhs);
    QD_CUDA(cudaStreamSynchronize(ctx->stream));  // S's scratch is released on return
  });
}

int qd_dirac_schur_apply_f32(qd_ctx* ctx, qd_gauge* gauge, double m0, double tau, int nrhs, const float* in,
                             float* out) {
  return guarded([&] {
    NONNULL(ctx);
    NONNULL(gauge);
    NONNULL(in);
    NONNULL(out);
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    QD_REQUIRE(in != out, "in and out must not overlap");
    QD_REQUIRE(std::isfinite(m0) && std::isfinite(tau), "m0 and tau must be finite");
    set_device(ctx);
    qd::SchurOp<qd::cplxf> S(gauge, gauge->links_f32(), m0, tau);
    S.apply(*ctx, reinterpret_cast<const qd::cplxf*>(in), reinterpret_cast<qd::cplxf*>(out), nrhs);
    QD_CUDA(cudaStreamSynchronize(ctx->stream));  // S's scratch is released on return
    const int e = qd::wilson_bulk_error(*ctx, gauge->geo);
    if (e) qd::fail(QD_ERR_TIMEOUT, "FP32 Wilson stencil: bounded wait timed out (code " + std::to_string(e) + ")");
  });
}

void qd_mg_params_default(qd_mg_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->nlevels = 1;
  for (int l = 0; l < QD_MAX_LEVELS; ++l) {
    for (int m = 0; m < 4; ++m) p->block[l][m] = 2;
    p->nv[l] = 12;
  }
  p->null_tol = 1e-2;
  p->null_maxit = 200;
  p->seed = 7;
  p->smoother_steps = 4;
  p->coarse_tol = 0.1;
  p->coarse_maxit = 256;
  p->coarse_restart = 16;
  p->coarsest_direct = 16384;
  p->coarsest_bf16 = 1;
  p->use_graphs = 1;
  p->coarse_tc = 1;
  p->coarse_smoother_steps = -1;
  p->null_f32 = 0;
}

void qd_solver_params_default(qd_solver_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->tol = 1e-8;
  p->maxit = 500;
  p->restart = 16;
  p->precision = QD_PREC_F64;
  p->inner_tol = 1e-5;
  p->max_refine = 10;
  p->schur = 0;
}

int qd_mg_setup(qd_ctx* ctx, const qd_gauge* gauge, double m0, double tau, const qd_mg_params* params,
                const double* injected_null, qd_mg** mg) {
  return guarded([&] {
    NONNULL(ctx);
    NONNULL(gauge);
    NONNULL(params);
    NONNULL(mg);
    set_device(ctx);
    std::unique_ptr<qd_mg> h(new qd_mg());
    h->ctx = ctx;
    h->gauge = gauge;
    h->m0 = m0;
    h->tau = tau;
    h->p = *params;
    QD_REQUIRE(params->coarse_restart >= 1 && params->coarse_maxit >= 1, "coarse GCR parameters must be >= 1");
    QD_REQUIRE(params->smoother_steps >= 0 && params->null_maxit >= 0, "step counts must be >= 0");
    qd::mg_build(*h, injected_null);
    *mg = h.release();
  });
}

int qd_mg_destroy(qd_mg* mg) {
  return guarded([&] {
    if (!mg) return;
    cudaStreamSynchronize(mg->ctx->stream);
    delete mg;
  });
}

int qd_mg_level_info(const qd_mg* mg, int level, int dims[4], int* dof, int64_t* nsites, int* null_steps) {
  return guarded([&] {
    NONNULL(mg);
    QD_REQUIRE(level >= 0 && level <= mg->nlevels, "level out of range");
    const qd::LevelGeom& g = mg->geom(level);
    if (dims)
      for (int m = 0; m < 4; ++m) dims[m] = g.dims[m];
    if (dof) *dof = mg->dof(level);
    if (nsites) *nsites = g.nsites;
    if (null_steps && level < mg->nlevels)
      for (int v = 0; v < mg->T[level]->nv; ++v) null_steps[v] = mg->T[level]->null_steps[v];
  });
}

int qd_prolongate(qd_mg* mg, int level, int nrhs, const double* coarse, double* fine) {
  return guarded([&] {
    NONNULL(mg);
    NONNULL(coarse);
    NONNULL(fine);
    QD_REQUIRE(level >= 0 && level < mg->nlevels, "level out of range");
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    set_device(mg->ctx);
    const qd::Transfer& T = *mg->T[level];
    qd::prolongate<qd::cplx>(*mg->ctx, T, T.W.as<qd::cplx>(), reinterpret_cast<const qd::cplx*>(coarse),
                             reinterpret_cast<qd::cplx*>(fine), nrhs);
  });
}

int qd_prolongate_f32(qd_mg* mg, int level, int nrhs, const float* coarse, float* fine) {
  return guarded([&] {
    NONNULL(mg);
    NONNULL(coarse);
    NONNULL(fine);
    QD_REQUIRE(level >= 0 && level < mg->nlevels, "level out of range");
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    set_device(mg->ctx);
    const qd::cplxf* W = mg->W<qd::cplxf>(level);
    qd::prolongate<qd::cplxf>(*mg->ctx, *mg->T[level], W, reinterpret_cast<const qd::cplxf*>(coarse),
                              reinterpret_cast<qd::cplxf*>(fine), nrhs);
  });
}

int qd_restrict(qd_mg* mg, int level, int nrhs, const double* fine, double* coarse) {
  return guarded([&] {
    NONNULL(mg);
    NONNULL(coarse);
    NONNULL(fine);
    QD_REQUIRE(level >= 0 && level < mg->nlevels, "level out of range");
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    set_device(mg->ctx);
    const qd::Transfer& T = *mg->T[level];
    qd::restrict_<qd::cplx>(*mg->ctx, T, T.W.as<qd::cplx>(), reinterpret_cast<const qd::cplx*>(fine),
                            reinterpret_cast<qd::cplx*>(coarse), nrhs);
  });
}

int qd_restrict_tc(qd_mg* mg, int level, int nrhs, const float* fine, float* coarse) {
  return guarded([&] {
    NONNULL(mg);
    NONNULL(fine);
    NONNULL(coarse);
    QD_REQUIRE(level >= 0 && level < mg->nlevels, "level out of range");
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    set_device(mg->ctx);
    qd::Transfer& T = *mg->T[level];
    QD_REQUIRE(qd::restrict_tc_supported(T, fine, coarse, nrhs),
               "tensor-core restriction needs fine dof 12, 16, 24 or 32, coarse dof 16, 24 or 32, 16-byte aligned "
               "fields and an even nrhs above 128");
    qd::restrict_tc(*mg->ctx, T, reinterpret_cast<const qd::cplxf*>(fine), reinterpret_cast<qd::cplxf*>(coarse), nrhs);
  });
}

int qd_coarse_apply(qd_mg* mg, int level, int nrhs, const double* in, double* out) {
  return guarded([&] {
    NONNULL(mg);
    NONNULL(in);
    NONNULL(out);
    QD_REQUIRE(level >= 1 && level <= mg->nlevels, "coarse level out of range");
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    QD_REQUIRE(in != out, "in and out must not overlap");
    set_device(mg->ctx);
    const qd::CoarseLevel& lv = *mg->L[level - 1];
    qd::coarse_apply<qd::cplx>(*mg->ctx, lv, lv.Cm.as<qd::cplx>(), reinterpret_cast<const qd::cplx*>(in),
                               reinterpret_cast<qd::cplx*>(out), nrhs);
  });
}

int qd_coarse_apply_f32(qd_mg* mg, int level, int nrhs, const float* in, float* out) {
  return guarded([&] {
    NONNULL(mg);
    NONNULL(in);
    NONNULL(out);
    QD_REQUIRE(level >= 1 && level <= mg->nlevels, "coarse level out of range");
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    QD_REQUIRE(in != out, "in and out must not overlap");
    set_device(mg->ctx);
    mg->op<qd::cplxf>(level);  // makes the FP32 copy of the stencil
    const qd::CoarseLevel& lv = *mg->L[level - 1];
    qd::coarse_apply<qd::cplxf>(*mg->ctx, lv, lv.Cmf.as<qd::cplxf>(), reinterpret_cast<const qd::cplxf*>(in),
                                reinterpret_cast<qd::cplxf*>(out), nrhs);
  });
}

int qd_coarse_residual_tc(qd_mg* mg, int level, int nrhs, const float* b, const float* x, float* r) {
  return guarded([&] {
    NONNULL(mg);
    NONNULL(b);
    NONNULL(x);
    NONNULL(r);
    QD_REQUIRE(level >= 1 && level <= mg->nlevels, "coarse level out of range");
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    QD_REQUIRE((const void*)x != (void*)r && (const void*)b != (void*)r && b != x, "b, x and r must be distinct");
    set_device(mg->ctx);
    qd::CoarseLevel& lv = *mg->L[level - 1];
    QD_REQUIRE(qd::coarse_tc_supported(lv, x, r, nrhs) && (reinterpret_cast<uintptr_t>(b) & 15) == 0,
               "tensor-core coarse stencil needs dof 8, 16, 24 or 32, 16-byte aligned fields and an even nrhs "
               "above 128");
    qd::coarse_apply_tc(*mg->ctx, lv, reinterpret_cast<const qd::cplxf*>(x), reinterpret_cast<qd::cplxf*>(r), nrhs,
                        reinterpret_cast<const qd::cplxf*>(b));
  });
}

int qd_coarse_apply_tc(qd_mg* mg, int level, int nrhs, const float* in, float* out) {
  return guarded([&] {
    NONNULL(mg);
    NONNULL(in);
    NONNULL(out);
    QD_REQUIRE(level >= 1 && level <= mg->nlevels, "coarse level out of range");
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    QD_REQUIRE((const void*)in != (void*)out, "in and out must not overlap");
    set_device(mg->ctx);
    qd::CoarseLevel& lv = *mg->L[level - 1];
    QD_REQUIRE(qd::coarse_tc_supported(lv, in, out, nrhs),
               "tensor-core coarse stencil needs dof 8, 16, 24 or 32, 16-byte aligned fields and an even nrhs "
               "above 128");
    qd::coarse_apply_tc(*mg->ctx, lv, reinterpret_cast<const qd::cplxf*>(in), reinterpret_cast<qd::cplxf*>(out),
                        nrhs);
  });
}

int qd_coarse_solve(qd_mg* mg, int level, int nrhs, const double* in, double* out) {
  return guarded([&] {
    NONNULL(mg);
    NONNULL(in);
    NONNULL(out);
    QD_REQUIRE(level >= 1 && level <= mg->nlevels, "coarse level out of range");
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    QD_REQUIRE(in != out, "in and out must not overlap");
    set_device(mg->ctx);
    qd_ctx& ctx = *mg->ctx;
    const qd::cplx* x = reinterpret_cast<const qd::cplx*>(in);
    qd::cplx* y = reinterpret_cast<qd::cplx*>(out);
    const qd::cplx* inv = mg->Cinv<qd::cplx>(level);
    if (inv) {
      qd::coarsest_solve_refined(ctx, *mg->L[level - 1], nrhs, x, y, 3);
    } else {
      auto A = mg->op<qd::cplx>(level);
      std::unique_ptr<qd::MGPrecond<qd::cplx>> pre;
      if (level < mg->nlevels) pre.reset(new qd::MGPrecond<qd::cplx>(mg, level));
      qd::GCR<qd::cplx> gcr;
      gcr.solve(ctx, *A, pre.get(), x, y, nrhs, mg->p.coarse_tol, mg->p.coarse_maxit, mg->p.coarse_restart,
                nullptr);
    }
    QD_CUDA(cudaStreamSynchronize(ctx.stream));
  });
}

int qd_coarse_solve_f32(qd_mg* mg, int level, int nrhs, const float* in, float* out) {
  return guarded([&] {
    NONNULL(mg);
    NONNULL(in);
    NONNULL(out);
    QD_REQUIRE(level >= 1 && level <= mg->nlevels, "coarse level out of range");
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    QD_REQUIRE((const void*)in != (void*)out, "in and out must not overlap");
    set_device(mg->ctx);
    qd_ctx& ctx = *mg->ctx;
    qd::CoarseLevel& lv = *mg->L[level - 1];
    const qd::cplxf* inv = mg->Cinv<qd::cplxf>(level);
    QD_REQUIRE(inv != nullptr, "level has no dense inverse");
    const qd::cplxf* x = reinterpret_cast<const qd::cplxf*>(in);
    qd::cplxf* y = reinterpret_cast<qd::cplxf*>(out);
    if (lv.tc) {
      qd::tc_dense_apply(ctx, lv, x, y, nrhs);
      const int e = qd::tc_error(ctx, lv);
      if (e) qd::fail(QD_ERR_TIMEOUT, "tensor-core coarsest solve: bounded wait timed out (code " + std::to_string(e) + ")");
    } else {
      qd::dense_apply<qd::cplxf>(ctx, lv.ndense, nrhs, inv, x, y);
    }
    QD_CUDA(cudaStreamSynchronize(ctx.stream));
  });
}

int qd_solve(qd_ctx* ctx, const qd_gauge* gauge, qd_mg* mg, double m0, double tau, int nrhs, const double* b,
             double* x, const qd_solver_params* params, qd_solve_stats* stats) {
  int not_conv = 0;
  int rc = guarded([&] {
    NONNULL(ctx);
    NONNULL(gauge);
    NONNULL(b);
    NONNULL(x);
    NONNULL(params);
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    set_device(ctx);
    qd::SolveInfo info;
    qd::solve(*ctx, *gauge, mg, m0, tau, nrhs, reinterpret_cast<const qd::cplx*>(b), reinterpret_cast<qd::cplx*>(x),
              *params, info);
    if (stats) {
      stats->iterations = info.iterations;
      stats->converged = info.converged;
      stats->max_true_rel_residual = info.max_rel;
      if (stats->iters_per_rhs)
        for (int c = 0; c < nrhs; ++c) stats->iters_per_rhs[c] = info.iters[c];
      if (stats->true_rel_residual)
        for (int c = 0; c < nrhs; ++c) stats->true_rel_residual[c] = info.true_rel[c];
      stats->stagnated = info.stagnated ? 1 : 0;
    }
    not_conv = info.converged < nrhs;
  });
  if (rc == QD_OK && not_conv) {
    g_last_error = "solve did not reach the tolerance within maxit";
    return QD_ERR_NOT_CONVERGED;
  }
  return rc;
}

void qd_defl_params_default(qd_defl_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->kind = QD_DEFL_MG_OBLIQUE;
  p->k = 24;
  p->guard = 16;
  p->eig_tol = 1e-6;
  p->solve_tol = 1e-10;
  p->maxit = 50;
  p->seed = 12345;
  p->tau_restart = 0.1;
  p->max_restarts = 3;
  p->stag_window = 100;
  p->solve_restart = 32;
  p->fail_first = 0;
}

int qd_defl_create(qd_ctx* ctx, const qd_gauge* gauge, qd_mg* mg, double m0, double tau, const qd_defl_params* params,
                   const double* injected_basis, qd_defl** defl) {
  return guarded([&] {
    NONNULL(ctx);
    NONNULL(gauge);
    NONNULL(params);
    NONNULL(defl);
    set_device(ctx);
    if (mg) QD_REQUIRE(mg->gauge == gauge && mg->m0 == m0 && mg->tau == tau, "mg built for another operator");
    std::unique_ptr<qd_defl> d(new qd_defl());
    d->ctx = ctx;
    d->gauge = gauge;
    d->mg = mg;
    d->m0 = m0;
    d->tau = tau;
    d->p = *params;
    d->kind = params->kind;
    qd::defl_build(*d, injected_basis);
    *defl = d.release();
  });
}

int qd_defl_destroy(qd_defl* defl) {
  return guarded([&] {
    if (!defl) return;
    cudaStreamSynchronize(defl->ctx->stream);
    delete defl;
  });
}

int qd_defl_set_rank(qd_defl* defl, int rank, double* t0) {
  return guarded([&] {
    NONNULL(defl);
    set_device(defl->ctx);
    qd::defl_set_rank(*defl, rank);
    if (t0) {
      t0[0] = defl->t0[0];
      t0[1] = defl->t0[1];
    }
  });
}

int qd_defl_info(const qd_defl* defl, double* mu, double* lambda, int* iterations) {
  return guarded([&] {
    NONNULL(defl);
    if (mu)
      for (int i = 0; i < defl->p.k; ++i) mu[i] = defl->mu[i];
    if (lambda && defl->kind == QD_DEFL_MG_OBLIQUE) {
      QD_CUDA(cudaMemcpy(lambda, defl->lam.as<double>(), defl->rank * sizeof(double), cudaMemcpyDeviceToHost));
    }
    if (iterations) *iterations = defl->iterations;
  });
}

int qd_defl_shift_info(const qd_defl* defl, double* tau_eig, int* restarts) {
  return guarded([&] {
    NONNULL(defl);
    if (tau_eig) *tau_eig = defl->tau_eig;
    if (restarts) *restarts = defl->restarts;
  });
}

int qd_defl_gram(const qd_defl* defl, double* G) {
  return guarded([&] {
    NONNULL(defl);
    NONNULL(G);
    QD_REQUIRE(defl->kind == QD_DEFL_MG_OBLIQUE, "the Gram matrix G is defined for Algorithm 2 (Algorithm 1: G = I)");
    set_device(defl->ctx);
    const int k = defl->p.k;
    QD_CUDA(cudaMemcpy(G, defl->G.as<qd::cplx>(), (size_t)k * k * sizeof(qd::cplx), cudaMemcpyDeviceToHost));
  });
}

int qd_defl_basis(const qd_defl* defl, double* out) {
  return guarded([&] {
    NONNULL(defl);
    NONNULL(out);
    set_device(defl->ctx);
    QD_CUDA(cudaMemcpyAsync(out, defl->Ubar.as<qd::cplx>(), (size_t)defl->nb * defl->p.k * sizeof(qd::cplx),
                            cudaMemcpyDeviceToDevice, defl->ctx->stream));
  });
}

int qd_deflate_project(qd_defl* defl, int nrhs, const double* z, double* out) {
  return guarded([&] {
    NONNULL(defl);
    NONNULL(z);
    NONNULL(out);
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    QD_REQUIRE(!overlaps(z, out, (size_t)defl->gauge->geo.nsites * 12 * nrhs * sizeof(qd::cplx)),
               "z and out must not overlap");
    set_device(defl->ctx);
    qd::defl_project(*defl->ctx, *defl, nrhs, reinterpret_cast<const qd::cplx*>(z), reinterpret_cast<qd::cplx*>(out));
  });
}

int qd_deflate_project_static(qd_defl* defl, int nrhs, const double* z, double* out) {
  return guarded([&] {
    NONNULL(defl);
    NONNULL(z);
    NONNULL(out);
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    QD_REQUIRE(!overlaps(z, out, (size_t)defl->gauge->geo.nsites * 12 * nrhs * sizeof(qd::cplx)),
               "z and out must not overlap");
    set_device(defl->ctx);
    qd::defl_project_static(*defl, nrhs, reinterpret_cast<const qd::cplx*>(z), reinterpret_cast<qd::cplx*>(out));
  });
}

int qd_deflate_coeffs(qd_defl* defl, int nrhs, const double* z, double* ZhV, double* UhKZ) {
  return guarded([&] {
    NONNULL(defl);
    NONNULL(z);
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    set_device(defl->ctx);
    const int k = defl->p.k;
    qd::DevBuf m1((size_t)k * nrhs * sizeof(qd::cplx)), m2((size_t)k * nrhs * sizeof(qd::cplx));
    qd::defl_coeffs(*defl->ctx, *defl, nrhs, reinterpret_cast<const qd::cplx*>(z), m1.as<qd::cplx>(), m2.as<qd::cplx>());
    std::vector<qd::cplx> h1((size_t)k * nrhs), h2((size_t)k * nrhs);
    QD_CUDA(cudaMemcpyAsync(h1.data(), m1.as<qd::cplx>(), h1.size() * sizeof(qd::cplx), cudaMemcpyDeviceToHost,
                            defl->ctx->stream));
    QD_CUDA(cudaMemcpyAsync(h2.data(), m2.as<qd::cplx>(), h2.size() * sizeof(qd::cplx), cudaMemcpyDeviceToHost,
                            defl->ctx->stream));
    QD_CUDA(cudaStreamSynchronize(defl->ctx->stream));
    // ZhV[j][i] = conj((U_bar^H W^H Z)[i][j]); UhKZ[i][j] as computed
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < nrhs; ++j) {
        const qd::cplx a = h1[(size_t)i * nrhs + j], b = h2[(size_t)i * nrhs + j];
        if (ZhV) {
          ZhV[2 * ((size_t)j * k + i)] = a.x;
          ZhV[2 * ((size_t)j * k + i) + 1] = -a.y;
        }
        if (UhKZ) {
          UhKZ[2 * ((size_t)i * nrhs + j)] = b.x;
          UhKZ[2 * ((size_t)i * nrhs + j) + 1] = b.y;
        }
      }
  });
}

int qd_mg_subspace_sines(qd_mg* mg, int depth, int k, const double* V, double* sin_out) {
  return guarded([&] {
    NONNULL(mg);
    NONNULL(V);
    NONNULL(sin_out);
    QD_REQUIRE(depth >= 1 && depth <= mg->nlevels, "depth must be in [1, nlevels]");
    QD_REQUIRE(k >= 1, "k must be >= 1");
    set_device(mg->ctx);
    qd::mg_subspace_sines(*mg->ctx, *mg, depth, k, reinterpret_cast<const qd::cplx*>(V), sin_out);
  });
}

// Host outputs of one estimator call (shared by the single and batched forms).
static void fill_trace_result(qd_trace_result* result, const qd_defl* defl, const qd::TraceOut& out,
                              const std::vector<qd::cplx>& M1, const std::vector<qd::cplx>& M2, int s, bool coeffs) {
  result->t0[0] = defl ? defl->t0[0] : 0.0;
  result->t0[1] = defl ? defl->t0[1] : 0.0;
  result->mean[0] = out.stats[0];
  result->mean[1] = out.stats[1];
  result->estimate[0] = result->t0[0] + out.stats[0];
  result->estimate[1] = result->t0[1] + out.stats[1];
  result->var = out.stats[2];
  result->var_re = out.stats[3];
  result->stderr_mean = out.stats[4];
  result->var_jackknife_err = out.stats[5];
  result->nsamples = s;
  result->iterations = out.info.iterations;
  result->max_true_rel_residual = out.info.max_rel;
  if (result->t_samples)
    for (int j = 0; j < s; ++j) {
      result->t_samples[2 * j] = out.t[j].x;
      result->t_samples[2 * j + 1] = out.t[j].y;
    }
  if (coeffs) {
    const int k = defl->p.k;
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < s; ++j) {
        const qd::cplx a = M1[(size_t)i * s + j], b = M2[(size_t)i * s + j];
        if (result->ZhV) {
          result->ZhV[2 * ((size_t)j * k + i)] = a.x;
          result->ZhV[2 * ((size_t)j * k + i) + 1] = -a.y;
        }
        if (result->UhKZ) {
          result->UhKZ[2 * ((size_t)i * s + j)] = b.x;
          result->UhKZ[2 * ((size_t)i * s + j) + 1] = b.y;
        }
      }
  }
}

// One estimator call on ctx; returns whether every sample converged.
static bool run_trace(qd_ctx& ctx, const qd_gauge& gauge, qd_mg* mg, qd_defl* defl, double m0, double tau,
                      const qd_trace_params& params, qd_trace_result* result) {
  QD_REQUIRE(params.nsamples >= 1, "nsamples must be >= 1");
  qd::TraceOut out;
  std::vector<qd::cplx> M1, M2;
  const bool coeffs = defl && (result->ZhV || result->UhKZ);
  QD_REQUIRE(!(coeffs && params.dilution), "a-posteriori coefficients are not available with dilution");
  QD_REQUIRE(params.dilution == 0 || params.dilution == 12, "dilution must be 0 or 12");
  qd::hutchinson(ctx, gauge, mg, defl, m0, tau, params, coeffs, out, &M1, &M2);
  fill_trace_result(result, defl, out, M1, M2, params.nsamples, coeffs);
  return out.info.converged >= (params.dilution == 12 ? 12 : 1) * params.nsamples;
}

int qd_hutchinson_trace(qd_ctx* ctx, const qd_gauge* gauge, qd_mg* mg, qd_defl* defl, double m0, double tau,
                        const qd_trace_params* params, qd_trace_result* result) {
  int not_conv = 0;
  int rc = guarded([&] {
    NONNULL(ctx);
    NONNULL(gauge);
    NONNULL(params);
    NONNULL(result);
    set_device(ctx);
    not_conv = !run_trace(*ctx, *gauge, mg, defl, m0, tau, *params, result);
  });
  if (rc == QD_OK && not_conv) {
    g_last_error = "a solve did not reach the tolerance within maxit";
    return QD_ERR_NOT_CONVERGED;
  }
  return rc;
}

// Lazily made FP32 copies (links, W, coarse operators, coarsest inverse)
// are created on the object's own context; make them all before worker
// threads read them from other streams.
static void prewarm_fp32(qd_batch_item& it) {
  const_cast<qd_gauge*>(it.gauge)->links_f32();
  if (!it.mg) return;
  for (int l = 0; l < it.mg->nlevels; ++l) it.mg->W<qd::cplxf>(l);
  for (int l = 1; l <= it.mg->nlevels; ++l) it.mg->op<qd::cplxf>(l);
  it.mg->Cinv<qd::cplxf>(it.mg->nlevels);
}

int qd_hutchinson_batch(qd_ctx* ctx, int nitems, qd_batch_item* items, int nstreams) {
  std::vector<std::string> msgs;
  int first_bad = -1;
  int rc = guarded([&] {
    NONNULL(ctx);
    QD_REQUIRE(nitems >= 0, "nitems must be >= 0");
    QD_REQUIRE(nitems == 0 || items != nullptr, "items must not be NULL");
    QD_REQUIRE(nstreams >= 1 && nstreams <= 64, "nstreams must be in [1, 64]");
    set_device(ctx);
    for (int i = 0; i < nitems; ++i) {
      NONNULL(items[i].gauge);
      NONNULL(items[i].result);
      QD_REQUIRE(items[i].params.nsamples >= 1, "nsamples must be >= 1");
      for (int j = 0; j < i; ++j) {
        QD_REQUIRE(!items[i].mg || items[i].mg != items[j].mg, "an mg handle appears in two batch items");
        QD_REQUIRE(!items[i].defl || items[i].defl != items[j].defl, "a defl handle appears in two batch items");
      }
      items[i].status = QD_OK;
    }
    if (nitems == 0) return;
    for (int i = 0; i < nitems; ++i) prewarm_fp32(items[i]);
    QD_CUDA(cudaDeviceSynchronize());
    // largest first (longest-processing-time order), dynamic hand-out
    std::vector<int> order(nitems);
    for (int i = 0; i < nitems; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return items[a].gauge->geo.nsites * (double)items[a].params.nsamples >
             items[b].gauge->geo.nsites * (double)items[b].params.nsamples;
    });
    const int nw = std::min(nstreams, nitems);
    std::vector<std::unique_ptr<qd_ctx>> workers(nw);
    for (int w = 0; w < nw; ++w) {
      workers[w].reset(new qd_ctx());
      workers[w]->device = ctx->device;
      QD_CUDA(cudaStreamCreateWithFlags(&workers[w]->stream, cudaStreamNonBlocking));
      QD_CUDA(cudaMallocHost(&workers[w]->host_pinned, 64 * sizeof(int)));
    }
    msgs.assign(nitems, std::string());
    std::atomic<int> next{0};
    auto work = [&](qd_ctx* wc) {
      cudaSetDevice(wc->device);
      for (int k = next.fetch_add(1); k < nitems; k = next.fetch_add(1)) {
        qd_batch_item& it = items[order[k]];
        try {
          const bool ok = run_trace(*wc, *it.gauge, it.mg, it.defl, it.m0, it.tau, it.params, it.result);
          it.status = ok ? QD_OK : QD_ERR_NOT_CONVERGED;
          if (!ok) msgs[order[k]] = "a solve did not reach the tolerance within maxit";
        } catch (const qd::Error& e) {
          it.status = e.code;
          msgs[order[k]] = e.what();
        } catch (const std::exception& e) {
          it.status = QD_ERR_INTERNAL;
          msgs[order[k]] = e.what();
        }
      }
    };
    std::vector<std::thread> threads;
    for (int w = 1; w < nw; ++w) threads.emplace_back(work, workers[w].get());
    work(workers[0].get());
    for (std::thread& t : threads) t.join();
    for (auto& wc : workers) {
      cudaStreamSynchronize(wc->stream);
      cudaFreeHost(wc->host_pinned);
      wc->host_pinned = nullptr;
      cudaStreamDestroy(wc->stream);
      wc->stream = nullptr;
    }
    // first hard error, else first non-convergence
    for (int pass = 0; pass < 2 && first_bad < 0; ++pass)
      for (int i = 0; i < nitems; ++i)
        if (items[i].status != QD_OK && (pass == 1 || items[i].status != QD_ERR_NOT_CONVERGED)) {
          first_bad = i;
          break;
        }
  });
  if (rc == QD_OK && first_bad >= 0) {
    g_last_error = msgs[first_bad];
    return items[first_bad].status;
  }
  return rc;
}

int qd_trace_stats(qd_ctx* ctx, int s, const double* t, const double t0[2], qd_trace_result* result) {
  return guarded([&] {
    NONNULL(ctx);
    NONNULL(t);
    NONNULL(t0);
    NONNULL(result);
    QD_REQUIRE(s >= 1, "s must be >= 1");
    set_device(ctx);
    qd::DevBuf st(8 * sizeof(double)), loo((size_t)s * sizeof(double));
    qd::trace_stats(*ctx, s, reinterpret_cast<const qd::cplx*>(t), st.as<double>(), loo.as<double>());
    double h[6];
    QD_CUDA(cudaMemcpyAsync(h, st.as<double>(), 6 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    QD_CUDA(cudaStreamSynchronize(ctx->stream));
    result->t0[0] = t0[0];
    result->t0[1] = t0[1];
    result->mean[0] = h[0];
    result->mean[1] = h[1];
    result->estimate[0] = t0[0] + h[0];
    result->estimate[1] = t0[1] + h[1];
    result->var = h[2];
    result->var_re = h[3];
    result->stderr_mean = h[4];
    result->var_jackknife_err = h[5];
    result->nsamples = s;
  });
}

void qd_smoother_params_default(qd_smoother_params* p) {
  if (!p) return;
  p->nsamples = 8;
  p->solve_tol = 1e-6;
  p->seed = 4242;
  p->mr_steps = 2;
  p->layers = 1;
}

int qd_smoother_train(qd_mg* mg, const qd_smoother_params* p, qd_smoother_info* info) {
  return guarded([&] {
    NONNULL(mg);
    NONNULL(p);
    QD_REQUIRE(p->solve_tol > 0.0 && p->solve_tol < 1.0, "solve_tol must be in (0, 1)");
    set_device(mg->ctx);
    double el = 0.0, ep = 0.0;
    int en = 0;
    qd::smoother_train(*mg, p->nsamples, p->solve_tol, p->seed, p->mr_steps, p->layers, &el, &ep, &en);
    if (info) {
      info->err_learned = el;
      info->err_plain = ep;
      info->enabled = en;
    }
  });
}

int qd_smoother_fit(qd_mg* mg, int nrhs, const double* e, const double* r) {
  return guarded([&] {
    NONNULL(mg);
    NONNULL(e);
    NONNULL(r);
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    set_device(mg->ctx);
    qd::smoother_fit(*mg, nrhs, reinterpret_cast<const qd::cplx*>(e), reinterpret_cast<const qd::cplx*>(r));
  });
}

int qd_smoother_set_weights(qd_mg* mg, const double* w) {
  return guarded([&] {
    NONNULL(mg);
    NONNULL(w);
    set_device(mg->ctx);
    qd::smoother_set_weights(*mg, reinterpret_cast<const qd::cplx*>(w));
  });
}

int qd_smoother_get_weights(const qd_mg* mg, double* w) {
  return guarded([&] {
    NONNULL(mg);
    NONNULL(w);
    QD_REQUIRE(mg->ls != nullptr, "no learned-smoother weights set");
    std::memcpy(w, mg->ls->w.data(), 144 * sizeof(qd::cplx));
  });
}

int qd_smoother_set_layer_weights(qd_mg* mg, int layers, const double* w) {
  return guarded([&] {
    NONNULL(mg);
    NONNULL(w);
    QD_REQUIRE(layers >= 1 && layers <= 4, "layers must be in [1, 4]");
    set_device(mg->ctx);
    qd::smoother_set_layers(*mg, layers, reinterpret_cast<const qd::cplx*>(w));
  });
}

int qd_smoother_layers(const qd_mg* mg) { return (mg && mg->ls) ? mg->ls->layers : 0; }

int qd_smoother_get_layer_weights(const qd_mg* mg, double* w) {
  return guarded([&] {
    NONNULL(mg);
    NONNULL(w);
    QD_REQUIRE(mg->ls != nullptr, "no learned-smoother weights set");
    std::memcpy(w, mg->ls->w.data(), mg->ls->w.size() * sizeof(qd::cplx));
  });
}

int qd_smoother_enable(qd_mg* mg, int enabled, int mr_steps) {
  return guarded([&] {
    NONNULL(mg);
    QD_REQUIRE(mr_steps >= 0 && mr_steps <= 64, "mr_steps must be in [0, 64]");
    QD_REQUIRE(!enabled || mg->ls != nullptr, "no learned-smoother weights set");
    if (mg->ls) {
      mg->ls->enabled = enabled != 0;
      mg->ls->mr_steps = mr_steps;
    }
  });
}

int qd_smoother_apply(qd_mg* mg, int nrhs, const double* in, double* out) {
  return guarded([&] {
    NONNULL(mg);
    NONNULL(in);
    NONNULL(out);
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    QD_REQUIRE(in != out, "in and out must not overlap");
    QD_REQUIRE(mg->ls != nullptr, "no learned-smoother weights set");
    set_device(mg->ctx);
    qd::smoother_apply<qd::cplx>(*mg->ctx, *mg, nrhs, reinterpret_cast<const qd::cplx*>(in),
                                 reinterpret_cast<qd::cplx*>(out), false);
  });
}

int qd_smoother_apply_f32(qd_mg* mg, int nrhs, const float* in, float* out) {
  return guarded([&] {
    NONNULL(mg);
    NONNULL(in);
    NONNULL(out);
    QD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    QD_REQUIRE(in != out, "in and out must not overlap");
    QD_REQUIRE(mg->ls != nullptr, "no learned-smoother weights set");
    set_device(mg->ctx);
    qd::smoother_apply<qd::cplxf>(*mg->ctx, *mg, nrhs, reinterpret_cast<const qd::cplxf*>(in),
                                  reinterpret_cast<qd::cplxf*>(out), false);
  });
}

void qd_autotune_set(int mode) { qd::tune_set_mode(mode); }
void qd_autotune_clear(void) { qd::tune_clear(); }
void qd_autotune_force(int candidate) { qd::tune_force(candidate); }
int qd_autotune_report(char* buf, int len) {
  const std::string r = qd::tune_report();
  if (buf && len > 0) {
    const size_t n = std::min((size_t)(len - 1), r.size());
    std::memcpy(buf, r.data(), n);
    buf[n] = '\0';
  }
  return (int)r.size() + 1;
}

long long qd_launch_count(void) { return qd::launch_counter().load(); }

long long qd_alloc_count(void) { return qd::alloc_counter().load(); }

int qd_prof_enable(qd_ctx* ctx, int enable) {
  return guarded([&] {
    NONNULL(ctx);
    if (!enable && ctx->prof) qd::prof_flush(*ctx);
    ctx->prof = enable != 0;
  });
}

int qd_prof_read(qd_ctx* ctx, int kind, int64_t* launches, double* ms, double* flops, double* bytes, int reset) {
  return guarded([&] {
    NONNULL(ctx);
    QD_REQUIRE(kind >= 0 && kind < QD_PROF_NKINDS, "unknown kernel kind");
    set_device(ctx);
    qd::prof_flush(*ctx);
    const qd::ProfTotals& t = ctx->prof_tot[kind];
    if (launches) *launches = t.launches;
    if (ms) *ms = t.ms;
    if (flops) *flops = t.flops;
    if (bytes) *bytes = t.bytes;
    if (reset) ctx->prof_tot[kind] = qd::ProfTotals();
  });
}

}  // extern "C"
