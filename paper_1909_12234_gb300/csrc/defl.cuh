// Deflation object and estimator helpers (see deflate.cu, trace.cu).
#pragma once

#include "mg.cuh"

namespace qd {

// Work spaces kept by a context between estimator / solve calls.
struct SolverCache {
  GCR<cplx> gcr64;
  GCR<cplxf> gcr32;
  // even-odd (Schur complement) fine solves
  GCR<cplx> gcr64s;
  GCR<cplxf> gcr32s;
  SchurPrecond<cplx> spre64;
  SchurPrecond<cplxf> spre32;
  DevBuf sch64, sch32;
  DevBuf Z, B, X, tdev, stats, loo;
  DevBuf mr, mt, mrf, mef, mscal;  // mixed-precision refinement
};
SolverCache& cache(qd_ctx& ctx);

}  // namespace qd

struct qd_defl {
  qd_ctx* ctx = nullptr;
  const qd_gauge* gauge = nullptr;
  qd_mg* mg = nullptr;
  double m0 = 0.0, tau = 0.0;
  qd_defl_params p{};
  int kind = 0;
  int level = 0;         // level of the basis vectors (1: Algorithm 2, 0: Algorithm 1)
  int64_t nb = 0;        // rows of the basis
  qd::DevBuf Ubar;       // nb x k (ld k): eigensolver output (or injected)
  qd::DevBuf G;          // k x k: U_bar^H gamma5^W C U_bar (Algorithm 2)
  qd::DevBuf AinvU;      // nb x k: A^{-1}_xi U (Algorithm 1)
  std::vector<double> mu;  // eigenvalues of H from the eigensolver
  int iterations = 0;
  int rank = 0;
  qd::DevBuf U;          // nb x rank (ld rank): U_bar U_hat (Alg 2) or U (Alg 1)
  qd::DevBuf pj[4];      // work spaces of the projection (grow-only)
  qd::DevBuf chain[2];   // intermediate levels of the composite W, W^H (grow-only)
  qd::DevBuf lam;        // rank doubles (Algorithm 2)
  qd::DevBuf t0buf;      // one complex on device
  double t0[2] = {0.0, 0.0};
  double tau_eig = 0.0;  // eigensolver shift after restarts (Sec. 3.2)
  int restarts = 0;
  std::unique_ptr<qd_mg> mg_shift;  // multigrid inverter of A + i tau_eig gamma5
  qd::cplx* t0_dev() {
    t0buf.resize(sizeof(qd::cplx));
    return t0buf.as<qd::cplx>();
  }
};

namespace qd {

void defl_build(qd_defl& d, const double* injected);
void defl_set_rank(qd_defl& d, int r);
// Launches go to ctx (the caller's stream), not to the context d was built on.
void defl_project(qd_ctx& ctx, qd_defl& d, int s, const cplx* z, cplx* out);
void defl_coeffs(qd_ctx& ctx, qd_defl& d, int s, const cplx* z, cplx* M1, cplx* M2);
// (I - U U^H) z with scratch in a fixed device array (noalloc.cu), and the
// address of that array on the current device (resolved at context creation).
void defl_project_static(qd_defl& d, int s, const cplx* z, cplx* out);
void* static_scratch_resolve();
void blockmul_identity_cols(qd_ctx& ctx, int64_t n, const cplx* X, int ldx, int r, cplx* Y);
void copy_leading_block(qd_ctx& ctx, int k, int r, const cplx* G, cplx* Gr);
void sum_over_lambda(qd_ctx& ctx, int r, const cplx* dv, const double* lam, cplx* out);
void trace_stats(qd_ctx& ctx, int s, const cplx* t, double* out_dev, double* loo_dev);
void mg_build(qd_mg& mg, const double* injected_null);
// sin of the angle between each of the k columns of V and range(W_0 ... W_{L-1})
void mg_subspace_sines(qd_ctx& ctx, qd_mg& mg, int L, int k, const cplx* V, double* out);

// Drivers (trace.cu).
void solve(qd_ctx& ctx, const qd_gauge& g, qd_mg* mg, double m0, double tau, int s, const cplx* b, cplx* x,
           const qd_solver_params& p, SolveInfo& info);
struct TraceOut {
  double stats[6];
  std::vector<cplx> t;
  SolveInfo info;
};
void hutchinson(qd_ctx& ctx, const qd_gauge& g, qd_mg* mg, qd_defl* d, double m0, double tau,
                const qd_trace_params& p, bool want_coeffs, TraceOut& out, std::vector<cplx>* M1,
                std::vector<cplx>* M2);

}  // namespace qd
