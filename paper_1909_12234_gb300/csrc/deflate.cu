// Deflation spaces, projection and the Hutchinson estimator.
//
// Algorithm 1: U = k eigenvectors of gamma5 (A + i tau gamma5)^{-1} of
//   largest magnitude (= eigenvectors of the Hermitian A gamma5 with smallest
//   |eigenvalue| at tau = 0); t0 = sum_i u_i^H A^{-1}_xi u_i; P = U U^H.
// Algorithm 2: U_bar = k eigenvectors of gamma5^W C^{-1} of largest
//   magnitude (= of the Hermitian C gamma5^W with smallest |mu|);
//   U_hat Lambda U_hat^H = U_bar^H gamma5^W C U_bar; U = U_bar U_hat;
//   t0 = sum_i u_i^H gamma5^W u_i / lambda_i;
//   P = A W U Lambda^{-1} U^H gamma5^W W^H (the K = gamma5 projector of
//   Sec. 2.1 with V = W U).
// Both eigenproblems are solved by block inverse subspace iteration with
// Rayleigh-Ritz on the inverse ("eigs" on the inverse with largest
// magnitude, Algorithm 1 step 1, Algorithm 2 step 2, Sec. 3.1):
//   Y = H^{-1} X (inexact GCR solves to solve_tol), T = X^H Y = S N S^H,
//   X <- orth(Y S) by Cholesky QR applied twice.
// Sec. 2.2: the a-posteriori matrices Z^H W U_bar and U_bar^H gamma5^W W^H Z.
#include <functional>

#include "blas.cuh"
#include "defl.cuh"
#include "dense.cuh"
#include "direct.cuh"

namespace qd {

SolverCache& cache(qd_ctx& ctx) {
  if (!ctx.cache) ctx.cache = std::make_shared<SolverCache>();
  return *static_cast<SolverCache*>(ctx.cache.get());
}

// Q <- Y R^{-1} with Y = Q R, twice (Cholesky QR 2).  Y: n x m (ld m).
static void cholqr2(qd_ctx& ctx, int64_t n, int m, cplx* Y, cplx* tmp, DevBuf& small) {
  small.resize((size_t)(2 * m * m) * sizeof(cplx) + 16);
  cplx* G = small.as<cplx>();
  cplx* Ri = G + (size_t)m * m;
  DevBuf flag(sizeof(int));
  QD_CUDA(cudaMemsetAsync(flag.as<int>(), 0, sizeof(int), ctx.stream));
  for (int pass = 0; pass < 2; ++pass) {
    blockdot(ctx, n, Y, m, m, Y, m, m, G);
    hermitize(ctx, m, G);
    cholesky_inverse(ctx, m, G, Ri, flag.as<int>());
    blockmul(ctx, n, Y, m, m, Ri, m, m, tmp, m, 1.0, 0.0);
    blas::copy(ctx, n * m, tmp, Y);
  }
  int h = 0;
  QD_CUDA(cudaMemcpyAsync(&h, flag.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaStreamSynchronize(ctx.stream));
  if (h) fail(QD_ERR_NONFINITE, "Cholesky QR: block is numerically rank deficient");
}

__global__ void k_reciprocal(int m, const double* __restrict__ in, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = 1.0 / in[i];
}

// Block inverse subspace iteration for the m eigenpairs of the Hermitian
// H = Op gamma5 closest to 0.  Rayleigh-Ritz is done on H^{-1} (whose wanted
// eigenvalues are the largest in magnitude, so spurious Ritz values of an
// indefinite H cannot displace them), using T = X^H (H^{-1} X) without an
// extra solve:
//   Y = H^{-1} X;  T = X^H Y = S diag(nu) S^H;  order by |1/nu| ascending;
//   residual_i = ||Y s_i - nu_i X s_i|| / |nu_i|;  X <- orth(Y S).
// With a shift (Op = A + i tau gamma5, tau = tau_s != 0) H is the normal
// A gamma5 + i tau; then T = Y^H Y = X^H (H_h^2 + tau^2)^{-1} X is the
// Hermitian matrix used (H_h = A gamma5, same eigenvectors, eigenvalues
// 1/(lambda^2 + tau^2) largest for the smallest |lambda|), mu_i = x_i^H Y s_i
// is the complex Rayleigh quotient, residual_i = ||Y s_i - mu_i x_i|| / |mu_i|
// and lambda_i = Re 1/mu_i.
// X (n x m, ld m) out: Ritz vectors; theta (host, m) out: eigenvalues of H_h.
// `solve(X, W, m)` must return W ~= Op^{-1} X for m columns.
typedef std::function<void(const cplx*, cplx*, int)> SolveFn;

static void subspace_eig(qd_ctx& ctx, const Op<cplx>& A, const SolveFn& solve, const LevelGeom& geo, int m, int k,
                         double eig_tol, int maxit, uint64_t seed, cplx* X, std::vector<double>& theta,
                         int& iters_out, double tau_s = 0.0) {
  const int64_t n = A.n();
  const int dof = A.dof();
  const size_t blk = (size_t)n * m * sizeof(cplx);
  DevBuf Yb(blk), Zb(blk), Tb(blk), small, eig((size_t)(3 * m * m + 4) * sizeof(cplx) + 6 * m * sizeof(double)),
      resid(m * sizeof(cplx)), iv((m + 8) * sizeof(int));
  DevBuf Rb(tau_s != 0.0 ? blk : 0), cm(tau_s != 0.0 ? (size_t)3 * m * sizeof(cplx) : 0);
  cplx* Y = Yb.as<cplx>();
  cplx* Z = Zb.as<cplx>();
  cplx* Tm = Tb.as<cplx>();
  cplx* Tmat = eig.as<cplx>();
  cplx* S = Tmat + (size_t)m * m;
  cplx* Ss = S + (size_t)m * m;
  double* nu = reinterpret_cast<double*>(Ss + (size_t)m * m);
  double* mu = nu + m;
  double* mus = mu + m;
  double* nus = mus + m;
  random_starts_fill(ctx, geo, dof, seed, m, X);
  cholqr2(ctx, n, m, X, Tm, small);
  theta.assign(m, 0.0);
  int it = 0;
  for (; it < maxit; ++it) {
    // Y = H^{-1} X = gamma5 Op^{-1} X
    solve(X, Tm, m);
    blas::gamma5(ctx, geo.nsites, dof, m, Tm, Y);
    if (tau_s != 0.0)
      blockdot(ctx, n, Y, m, m, Y, m, m, Tmat);  // Y^H Y
    else
      blockdot(ctx, n, X, m, m, Y, m, m, Tmat);  // X^H Y
    hermitize(ctx, m, Tmat);
    jacobi_eigh(ctx, m, Tmat, S, nu, nullptr);
    k_reciprocal<<<div_up(m, 128), 128, 0, ctx.stream>>>(m, nu, mu);
    QD_LAUNCH_CHECK();
    sort_by_abs(ctx, m, mu, S, mus, Ss, iv.as<int>());
    k_reciprocal<<<div_up(m, 128), 128, 0, ctx.stream>>>(m, mus, nus);
    QD_LAUNCH_CHECK();
    blockmul(ctx, n, X, m, m, Ss, m, m, Tm, m, 1.0, 0.0);  // Ritz vectors X S
    blockmul(ctx, n, Y, m, m, Ss, m, m, Z, m, 1.0, 0.0);   // H^{-1} X S
    std::vector<cplx> hr(m);
    std::vector<double> hnu(m);
    if (tau_s != 0.0) {
      // complex Rayleigh quotients mu_i = x_i^H (H^{-1} x_i) and the
      // residuals ||H^{-1} x_i - mu_i x_i||
      cplx* muc = cm.as<cplx>();
      cplx* negmu = muc + m;
      cplx* ones = negmu + m;
      blas::dots(ctx, 1, n, m, Tm, 0, Z, 0, muc);
      std::vector<cplx> hmu(m), hneg(m), hone(m, mkc(1.0, 0.0));
      QD_CUDA(cudaMemcpyAsync(hmu.data(), muc, m * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
      QD_CUDA(cudaStreamSynchronize(ctx.stream));
      for (int i = 0; i < m; ++i) {
        hneg[i] = mkc(-hmu[i].x, -hmu[i].y);
        const double a2 = hmu[i].x * hmu[i].x + hmu[i].y * hmu[i].y;
        hnu[i] = std::sqrt(a2);
        theta[i] = a2 > 0.0 ? hmu[i].x / a2 : 0.0;  // Re 1/mu
      }
      QD_CUDA(cudaMemcpyAsync(negmu, hneg.data(), m * sizeof(cplx), cudaMemcpyHostToDevice, ctx.stream));
      QD_CUDA(cudaMemcpyAsync(ones, hone.data(), m * sizeof(cplx), cudaMemcpyHostToDevice, ctx.stream));
      blas::copy(ctx, (int64_t)n * m, Z, Rb.as<cplx>());
      blas::axpby(ctx, n, m, negmu, Tm, ones, Rb.as<cplx>());
      blas::dots(ctx, 1, n, m, Rb.as<cplx>(), 0, Rb.as<cplx>(), 0, resid.as<cplx>());
      QD_CUDA(cudaMemcpyAsync(hr.data(), resid.as<cplx>(), m * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
      QD_CUDA(cudaStreamSynchronize(ctx.stream));
    } else {
      eig_residuals(ctx, n, m, Z, Tm, nus, resid.as<cplx>());
      QD_CUDA(cudaMemcpyAsync(hr.data(), resid.as<cplx>(), m * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
      QD_CUDA(cudaMemcpyAsync(theta.data(), mus, m * sizeof(double), cudaMemcpyDeviceToHost, ctx.stream));
      QD_CUDA(cudaMemcpyAsync(hnu.data(), nus, m * sizeof(double), cudaMemcpyDeviceToHost, ctx.stream));
      QD_CUDA(cudaStreamSynchronize(ctx.stream));
    }
    double worst = 0.0;
    for (int i = 0; i < k; ++i) {
      const double rel = std::sqrt(hr[i].x) / (std::fabs(hnu[i]) > 0 ? std::fabs(hnu[i]) : 1.0);
      if (!(rel <= worst)) worst = rel;
    }
    if (worst <= eig_tol || it + 1 == maxit) {
      blas::copy(ctx, (int64_t)n * m, Tm, X);
      ++it;
      break;
    }
    blas::copy(ctx, (int64_t)n * m, Z, X);
    cholqr2(ctx, n, m, X, Tm, small);
  }
  iters_out = it;
}

// Raised by the eigensolver's inner solves when the inverter stagnates or
// misses its tolerance (Sec. 3.2).
struct InverterStagnated {};

// ---------------------------------------------------------------------------
void defl_build(qd_defl& d, const double* injected) {
  qd_ctx& ctx = *d.ctx;
  const int k = d.p.k;
  QD_REQUIRE(k >= 1, "deflation rank k must be >= 1");
  if (d.kind == QD_DEFL_MG_OBLIQUE) {
    QD_REQUIRE(d.mg != nullptr, "Algorithm 2 deflation needs a multigrid hierarchy");
    // the coarsest level: W is the composite prolongator W_0 ... W_{L-1}
    // (Table 2 sizes the Algorithm 2 eigenproblem by the coarsest level)
    d.level = d.mg->nlevels;
  } else {
    QD_REQUIRE(d.kind == QD_DEFL_EIG_ORTHO, "unknown deflation kind");
    d.level = 0;
  }
  const LevelGeom& geo = d.level == 0 ? d.gauge->geo : d.mg->geom(d.level);
  const int dof = d.level == 0 ? 12 : d.mg->dof(d.level);
  d.nb = geo.nsites * (int64_t)dof;
  QD_REQUIRE(k <= d.nb, "deflation rank exceeds the dimension");
  d.Ubar.resize((size_t)d.nb * k * sizeof(cplx));
  std::unique_ptr<Op<cplx>> op;
  if (d.level >= 1)
    op = d.mg->op<cplx>(d.level);
  else
    op.reset(new WilsonOp<cplx>(d.gauge, d.gauge->links.as<cplx>(), d.m0, d.tau, false));
  d.mu.assign(k, 0.0);
  d.iterations = 0;
  if (injected) {
    QD_CUDA(cudaMemcpyAsync(d.Ubar.as<cplx>(), injected, (size_t)d.nb * k * sizeof(cplx), cudaMemcpyDeviceToDevice,
                            ctx.stream));
  } else {
    int m = k + (d.p.guard > 0 ? d.p.guard : 0);
    if (m > d.nb) m = (int)d.nb;
    DevBuf X((size_t)d.nb * m * sizeof(cplx));
    const cplx* inv = d.level >= 1 ? d.mg->Cinv<cplx>(d.level) : nullptr;
    const double stol = d.p.solve_tol;
    const int srestart = d.p.solve_restart > 0 ? d.p.solve_restart : 32;
    std::vector<double> theta;
    d.tau_eig = 0.0;
    d.restarts = 0;
    for (int attempt = 0;; ++attempt) {
      // the eigensolver's operator: A + i (tau + tau_eig) gamma5 and its
      // multigrid inverter (rebuilt for the shift after a restart)
      std::unique_ptr<Op<cplx>> opx;
      Precond<cplx>* M = nullptr;
      if (d.level == 0) {
        opx.reset(new WilsonOp<cplx>(d.gauge, d.gauge->links.as<cplx>(), d.m0, d.tau + d.tau_eig, false));
        if (d.tau_eig != 0.0 && d.mg_shift) M = d.mg_shift->pre64.get();
        else if (d.tau_eig == 0.0 && d.mg) M = d.mg->pre64.get();
      }
      const Op<cplx>& A = d.level == 0 ? *opx : *op;
      GCR<cplx> solver;
      solver.stag_window = d.p.stag_window;
      bool first = true;
      SolveFn fn = [&](const cplx* Xin, cplx* Wout, int mm) {
        if (inv) {
          // direct coarsest solve, corrected to FP64 accuracy (each correction
          // gains ~4 digits; two reach the 1e-10 of the eigensolver's solves)
          coarsest_solve_refined(ctx, *d.mg->L[d.level - 1], mm, Xin, Wout, 2);
          return;
        }
        if (first && attempt < d.p.fail_first) throw InverterStagnated();  // test hook
        first = false;
        SolveInfo info;
        solver.solve(ctx, A, M, Xin, Wout, mm, stol, 20000, srestart, &info);
        if (info.stagnated || info.converged < mm) throw InverterStagnated();
      };
      try {
        subspace_eig(ctx, A, fn, geo, m, k, d.p.eig_tol, d.p.maxit, d.p.seed, X.as<cplx>(), theta, d.iterations,
                     d.level == 0 ? d.tau_eig : 0.0);
        break;
      } catch (const InverterStagnated&) {
        if (d.level != 0 || attempt >= d.p.max_restarts)
          fail(QD_ERR_NOT_CONVERGED, "eigensolver: the inverter stagnated (restarts " + std::to_string(attempt) +
                                         ", shift " + std::to_string(d.tau_eig) + ")");
        // Sec. 3.2: rebuild the multigrid inverter with a larger shift and
        // restart the eigensolver
        d.tau_eig = d.tau_eig > 0.0 ? 4.0 * d.tau_eig : d.p.tau_restart;
        ++d.restarts;
        d.mg_shift.reset();
        if (d.mg) {
          std::unique_ptr<qd_mg> ms(new qd_mg());
          ms->ctx = d.mg->ctx;
          ms->gauge = d.gauge;
          ms->m0 = d.m0;
          ms->tau = d.tau + d.tau_eig;
          ms->p = d.mg->p;
          mg_build(*ms, nullptr);
          d.mg_shift = std::move(ms);
        }
      }
    }
    for (int i = 0; i < k; ++i) d.mu[i] = theta[i];
    // U_bar = first k columns of X (ld m -> ld k)
    blockmul_identity_cols(ctx, d.nb, X.as<cplx>(), m, k, d.Ubar.as<cplx>());
  }
  if (d.kind == QD_DEFL_MG_OBLIQUE) {
    // G = U_bar^H gamma5^W C U_bar
    DevBuf t1((size_t)d.nb * k * sizeof(cplx)), t2((size_t)d.nb * k * sizeof(cplx));
    op->apply(ctx, d.Ubar.as<cplx>(), t1.as<cplx>(), k);
    blas::gamma5(ctx, geo.nsites, dof, k, t1.as<cplx>(), t2.as<cplx>());
    d.G.resize((size_t)k * k * sizeof(cplx));
    blockdot(ctx, d.nb, d.Ubar.as<cplx>(), k, k, t2.as<cplx>(), k, k, d.G.as<cplx>());
    hermitize(ctx, k, d.G.as<cplx>());
  } else {
    // Y = A^{-1}_xi U for t0 = sum u_i^H A^{-1}_xi u_i (Algorithm 1, step 2)
    d.AinvU.resize((size_t)d.nb * k * sizeof(cplx));
    GCR<cplx> solver;
    SolveInfo info;
    solver.solve(ctx, *op, d.mg ? d.mg->pre64.get() : nullptr, d.Ubar.as<cplx>(), d.AinvU.as<cplx>(), k,
                 d.p.solve_tol, 100000, 32, &info);
  }
  defl_set_rank(d, k);
}

void defl_set_rank(qd_defl& d, int r) {
  qd_ctx& ctx = *d.ctx;
  QD_REQUIRE(r >= 1 && r <= d.p.k, "rank must be in [1, k]");
  const int k = d.p.k;
  d.rank = r;
  const LevelGeom& geo = d.level == 0 ? d.gauge->geo : d.mg->geom(d.level);
  const int dof = d.level == 0 ? 12 : d.mg->dof(d.level);
  DevBuf dv(r * sizeof(cplx));
  if (d.kind == QD_DEFL_MG_OBLIQUE) {
    // step 3 on the leading r columns: G_r = U_hat Lambda U_hat^H
    DevBuf Gr((size_t)r * r * sizeof(cplx)), E((size_t)r * r * sizeof(cplx));
    copy_leading_block(ctx, k, r, d.G.as<cplx>(), Gr.as<cplx>());
    d.lam.resize(r * sizeof(double));
    jacobi_eigh(ctx, r, Gr.as<cplx>(), E.as<cplx>(), d.lam.as<double>(), nullptr);
    d.U.resize((size_t)d.nb * r * sizeof(cplx));
    blockmul(ctx, d.nb, d.Ubar.as<cplx>(), k, r, E.as<cplx>(), r, r, d.U.as<cplx>(), r, 1.0, 0.0);
    // step 4: t0 = sum_i u_i^H gamma5^W u_i / lambda_i
    DevBuf g((size_t)d.nb * r * sizeof(cplx));
    blas::gamma5(ctx, geo.nsites, dof, r, d.U.as<cplx>(), g.as<cplx>());
    blas::dots(ctx, 1, d.nb, r, d.U.as<cplx>(), 0, g.as<cplx>(), 0, dv.as<cplx>());
    sum_over_lambda(ctx, r, dv.as<cplx>(), d.lam.as<double>(), d.t0_dev());
  } else {
    // t0 = sum_{i<r} u_i^H (A^{-1}_xi u_i): column dots on the leading r columns
    DevBuf Ur((size_t)d.nb * r * sizeof(cplx)), Yr((size_t)d.nb * r * sizeof(cplx));
    blockmul_identity_cols(ctx, d.nb, d.Ubar.as<cplx>(), k, r, Ur.as<cplx>());
    blockmul_identity_cols(ctx, d.nb, d.AinvU.as<cplx>(), k, r, Yr.as<cplx>());
    blas::dots(ctx, 1, d.nb, r, Ur.as<cplx>(), 0, Yr.as<cplx>(), 0, dv.as<cplx>());
    sum_over_lambda(ctx, r, dv.as<cplx>(), nullptr, d.t0_dev());
    d.U.resize((size_t)d.nb * r * sizeof(cplx));
    QD_CUDA(cudaMemcpyAsync(d.U.as<cplx>(), Ur.as<cplx>(), (size_t)d.nb * r * sizeof(cplx), cudaMemcpyDeviceToDevice,
                            ctx.stream));
  }
  QD_CUDA(cudaMemcpyAsync(d.t0, d.t0_dev(), sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaStreamSynchronize(ctx.stream));
}

// c = W^H z with the composite W = W_0 ... W_{L-1} (L = d.level), s columns
static void restrict_chain(qd_ctx& ctx, qd_defl& d, int s, const cplx* z, cplx* c) {
  const cplx* src = z;
  DevBuf* tmp = d.chain;
  for (int l = 0; l < d.level; ++l) {
    const Transfer& T = *d.mg->T[l];
    cplx* dst = c;
    if (l + 1 < d.level) {
      tmp[l & 1].resize((size_t)d.mg->geom(l + 1).nsites * T.Dc * s * sizeof(cplx));
      dst = tmp[l & 1].as<cplx>();
    }
    restrict_<cplx>(ctx, T, T.W.as<cplx>(), src, dst, s);
    src = dst;
  }
}

// f = W c with the composite W, s columns
static void prolong_chain(qd_ctx& ctx, qd_defl& d, int s, const cplx* c, cplx* f) {
  const cplx* src = c;
  DevBuf* tmp = d.chain;
  for (int l = d.level - 1; l >= 0; --l) {
    const Transfer& T = *d.mg->T[l];
    cplx* dst = f;
    if (l > 0) {
      tmp[l & 1].resize((size_t)d.mg->geom(l).nsites * T.Df * s * sizeof(cplx));
      dst = tmp[l & 1].as<cplx>();
    }
    prolongate<cplx>(ctx, T, T.W.as<cplx>(), src, dst, s);
    src = dst;
  }
}

// out = (I - P) z, s columns
void defl_project(qd_ctx& ctx, qd_defl& d, int s, const cplx* z, cplx* out) {
  const int r = d.rank;
  const int64_t nf = d.gauge->geo.nsites * 12;
  // work spaces kept on the object (grow-only): no allocation per batch
  DevBuf& a = d.pj[0];
  a.resize((size_t)r * s * sizeof(cplx));
  if (d.kind == QD_DEFL_MG_OBLIQUE) {
    const LevelGeom& cg = d.mg->geom(d.level);
    const int dc = d.mg->dof(d.level);
    DevBuf& c = d.pj[1];
    DevBuf& gc = d.pj[2];
    DevBuf& f = d.pj[3];
    c.resize((size_t)d.nb * s * sizeof(cplx));
    gc.resize((size_t)d.nb * s * sizeof(cplx));
    f.resize((size_t)nf * s * sizeof(cplx));
    restrict_chain(ctx, d, s, z, c.as<cplx>());
    blas::gamma5(ctx, cg.nsites, dc, s, c.as<cplx>(), gc.as<cplx>());
    blockdot(ctx, d.nb, d.U.as<cplx>(), r, r, gc.as<cplx>(), s, s, a.as<cplx>());  // U^H g5 W^H z
    scale_rows_inv(ctx, r, s, d.lam.as<double>(), a.as<cplx>());                  // Lambda^{-1}
    blockmul(ctx, d.nb, d.U.as<cplx>(), r, r, a.as<cplx>(), s, s, c.as<cplx>(), s, 1.0, 0.0);  // U (.)
    prolong_chain(ctx, d, s, c.as<cplx>(), f.as<cplx>());                              // W (.)
    // out = z - A W U Lambda^{-1} U^H g5 W^H z (fused residual kernel)
    wilson_apply<cplx>(ctx, d.gauge->geo, d.gauge->links.as<cplx>(), d.m0, d.tau, false, f.as<cplx>(), out, s, z);
  } else {
    blockdot(ctx, nf, d.U.as<cplx>(), r, r, z, s, s, a.as<cplx>());  // U^H z
    blas::copy(ctx, nf * s, z, out);
    blockmul(ctx, nf, d.U.as<cplx>(), r, r, a.as<cplx>(), s, s, out, s, -1.0, 1.0);
  }
}

// Sec. 2.2 matrices: kind 2: M1 = U_bar^H W^H Z (k x s), M2 = U_bar^H g5 W^H Z;
// kind 1: M1 = (A^{-1}_xi U)^H Z, M2 = U^H Z.
void defl_coeffs(qd_ctx& ctx, qd_defl& d, int s, const cplx* z, cplx* M1, cplx* M2) {
  const int k = d.p.k;
  if (d.kind == QD_DEFL_EIG_ORTHO) {
    blockdot(ctx, d.nb, d.AinvU.as<cplx>(), k, k, z, s, s, M1);
    blockdot(ctx, d.nb, d.Ubar.as<cplx>(), k, k, z, s, s, M2);
    return;
  }
  const LevelGeom& cg = d.mg->geom(d.level);
  DevBuf c((size_t)d.nb * s * sizeof(cplx)), gc((size_t)d.nb * s * sizeof(cplx));
  restrict_chain(ctx, d, s, z, c.as<cplx>());
  blas::gamma5(ctx, cg.nsites, d.mg->dof(d.level), s, c.as<cplx>(), gc.as<cplx>());
  blockdot(ctx, d.nb, d.Ubar.as<cplx>(), k, k, c.as<cplx>(), s, s, M1);
  blockdot(ctx, d.nb, d.Ubar.as<cplx>(), k, k, gc.as<cplx>(), s, s, M2);
}

// sin of the angle between each column of V and range(W), W = W_0 ... W_{L-1}
void mg_subspace_sines(qd_ctx& ctx, qd_mg& mg, int L, int k, const cplx* V, double* out) {
  const int64_t nf = mg.gauge->geo.nsites * 12;
  qd_defl tmp;  // only the chain fields are used
  tmp.mg = &mg;
  tmp.level = L;
  const int64_t nc = mg.geom(L).nsites * (int64_t)mg.dof(L);
  DevBuf c((size_t)nc * k * sizeof(cplx)), f((size_t)nf * k * sizeof(cplx)), nn((size_t)2 * k * sizeof(cplx));
  restrict_chain(ctx, tmp, k, V, c.as<cplx>());
  prolong_chain(ctx, tmp, k, c.as<cplx>(), f.as<cplx>());
  blas::sub(ctx, nf * k, V, f.as<cplx>(), f.as<cplx>());  // v - W W^H v
  blas::dots(ctx, 1, nf, k, f.as<cplx>(), 0, f.as<cplx>(), 0, nn.as<cplx>());
  blas::dots(ctx, 1, nf, k, V, 0, V, 0, nn.as<cplx>() + k);
  std::vector<cplx> h(2 * k);
  QD_CUDA(cudaMemcpyAsync(h.data(), nn.as<cplx>(), 2 * k * sizeof(cplx), cudaMemcpyDeviceToHost, ctx.stream));
  QD_CUDA(cudaStreamSynchronize(ctx.stream));
  for (int i = 0; i < k; ++i) out[i] = h[k + i].x > 0.0 ? std::sqrt(h[i].x / h[k + i].x) : 0.0;
}

// ---------------------------------------------------------------------------
// Small kernels
// ---------------------------------------------------------------------------
__global__ void k_copy_cols(int64_t n, const cplx* __restrict__ X, int ldx, int r, cplx* __restrict__ Y) {
  const int64_t tot = n * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % r);
    const int64_t i = e / r;
    Y[e] = X[i * ldx + c];
  }
}
void blockmul_identity_cols(qd_ctx& ctx, int64_t n, const cplx* X, int ldx, int r, cplx* Y) {
  int blocks = div_up(n * r, 256);
  if (blocks > 32 * kNumSMs) blocks = 32 * kNumSMs;
  k_copy_cols<<<blocks, 256, 0, ctx.stream>>>(n, X, ldx, r, Y);
  QD_LAUNCH_CHECK();
}
void copy_leading_block(qd_ctx& ctx, int k, int r, const cplx* G, cplx* Gr) {
  blockmul_identity_cols(ctx, r, G, k, r, Gr);
}

// out = sum_i d_i / lam_i (lam nullable -> 1), Neumaier-compensated, in order
__global__ void k_sum_over_lambda(int r, const cplx* __restrict__ dv, const double* __restrict__ lam,
                                  cplx* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double sr = 0, cr = 0, si = 0, ci = 0;
  for (int i = 0; i < r; ++i) {
    const double l = lam ? lam[i] : 1.0;
    const double xr = dv[i].x / l, xi = dv[i].y / l;
    double t = sr + xr;
    cr += (fabs(sr) >= fabs(xr)) ? (sr - t) + xr : (xr - t) + sr;
    sr = t;
    t = si + xi;
    ci += (fabs(si) >= fabs(xi)) ? (si - t) + xi : (xi - t) + si;
    si = t;
  }
  *out = mkc(sr + cr, si + ci);
}
void sum_over_lambda(qd_ctx& ctx, int r, const cplx* dv, const double* lam, cplx* out) {
  k_sum_over_lambda<<<1, 32, 0, ctx.stream>>>(r, dv, lam, out);
  QD_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// Estimator statistics on the device (a9): Neumaier sums in sample order.
// out: [0] mean re, [1] mean im, [2] var, [3] var_re, [4] stderr, [5] jk err
// ---------------------------------------------------------------------------
__device__ void neu_add(double& s, double& c, double x) {
  const double t = s + x;
  c += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
  s = t;
}

__global__ void k_trace_stats(int s, const cplx* __restrict__ t, double* __restrict__ out, double* __restrict__ loo) {
  // delete-one variances, one sample per thread
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    double mr = 0, cmr = 0, mi = 0, cmi = 0;
    for (int j = 0; j < s; ++j) {
      if (j == i) continue;
      neu_add(mr, cmr, t[j].x);
      neu_add(mi, cmi, t[j].y);
    }
    const double m_r = (mr + cmr) / (s - 1), m_i = (mi + cmi) / (s - 1);
    double v = 0, cv = 0;
    for (int j = 0; j < s; ++j) {
      if (j == i) continue;
      const double dr = t[j].x - m_r, di = t[j].y - m_i;
      neu_add(v, cv, dr * dr + di * di);
    }
    loo[i] = s > 2 ? (v + cv) / (s - 2) : 0.0;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double sr = 0, cr = 0, si = 0, ci = 0;
  for (int j = 0; j < s; ++j) {
    neu_add(sr, cr, t[j].x);
    neu_add(si, ci, t[j].y);
  }
  const double mr = (sr + cr) / s, mi = (si + ci) / s;
  double v = 0, cv = 0, vr = 0, cvr = 0;
  for (int j = 0; j < s; ++j) {
    const double dr = t[j].x - mr, di = t[j].y - mi;
    neu_add(v, cv, dr * dr + di * di);
    neu_add(vr, cvr, dr * dr);
  }
  const double var = s > 1 ? (v + cv) / (s - 1) : 0.0;
  const double var_re = s > 1 ? (vr + cvr) / (s - 1) : 0.0;
  double lm = 0, clm = 0;
  for (int j = 0; j < s; ++j) neu_add(lm, clm, loo[j]);
  const double lmean = (lm + clm) / s;
  double q = 0, cq = 0;
  for (int j = 0; j < s; ++j) neu_add(q, cq, (loo[j] - lmean) * (loo[j] - lmean));
  out[0] = mr;
  out[1] = mi;
  out[2] = var;
  out[3] = var_re;
  out[4] = s > 0 ? sqrt(var / s) : 0.0;
  out[5] = s > 2 ? sqrt((double)(s - 1) / s * (q + cq)) : 0.0;
}

void trace_stats(qd_ctx& ctx, int s, const cplx* t, double* out_dev, double* loo_dev) {
  k_trace_stats<<<1, 256, 0, ctx.stream>>>(s, t, out_dev, loo_dev);
  QD_LAUNCH_CHECK();
}

}  // namespace qd
