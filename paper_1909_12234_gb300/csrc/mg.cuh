// Solvers and the multigrid hierarchy object (Sec. 2 two-grid method and
// adaptive setup; Sec. 1 inexact solves).
#pragma once

#include "qd_internal.cuh"

namespace qd {

struct SolveInfo {
  int iterations = 0;
  int converged = 0;
  bool stagnated = false;  // stopped by the stagnation test (GCR::stag_window)
  double max_rel = 0.0;
  std::vector<int> iters;
  std::vector<double> true_rel;
};

// Flexible restarted GCR, batched over independent right-hand sides.
template <class C> class GCR {
 public:
  // Gram-Schmidt passes per iteration (2 = CGS2; 1 = classical, one pass).
  int orth_passes = 2;
  // > 0 (with a tolerance > 0): every stag_window iterations compare each
  // active column's residual with its value stag_window iterations before;
  // if one fell by less than the factor stag_ratio the solve stops with
  // SolveInfo::stagnated (the inverter stagnating, Sec. 3.2).
  int stag_window = 0;
  double stag_ratio = 0.9;
  // > 0 (fused FP32 form only): each direction P_i and the residual r sit at
  // offset `embed` (complex elements) inside a slot of embed + n nrhs
  // elements whose leading part of r is zero, so a preconditioner can read r
  // and write P_i as the second half of a larger field (the odd sites of a
  // full-lattice field in the even-odd solve) without copies.
  int64_t embed = 0;
  bool embeds(int restart) const;
  // x = A^{-1} b to ||b - A x|| <= tol ||b|| per column (x overwritten,
  // zero initial guess).  M (nullable) is a right preconditioner that may
  // change between calls.  `quiet` skips per-column statistics.
  void solve(qd_ctx& ctx, const Op<C>& A, Precond<C>* M, const C* b, C* x, int nrhs, double tol,
             int maxit, int restart, SolveInfo* info);
  // Device buffers the solve uses (their current addresses).
  void buffers(std::vector<const void*>& v) const;

 private:
  void ensure(int64_t n, int nrhs, int m, int64_t emb);
  DevBuf P_, Q_, r_, t_;
  int64_t cap_emb_ = -1;
  DevBuf sc_;   // cplx per-RHS scalars
  DevBuf tab_;  // cplx coefficient tables of the fused one-pass form
  DevBuf act_;  // int [nrhs + 1]: active flags, then the count of active
  int64_t cap_n_ = -1;
  int cap_rhs_ = -1, cap_m_ = -1;
};

// Minimal-residual steps on A x = b, batched.  Fixed number of steps with
// x0 = 0 (smoother), or until ||r|| <= tol ||r0|| per column (null vectors,
// x0 given).  steps (device int[nrhs], nullable) counts steps per column.
template <class C>
void mr_steps(qd_ctx& ctx, const Op<C>& A, const C* b, C* x, bool x_is_zero, int nrhs, int nsteps,
              double tol, C* rbuf, C* qbuf, int* steps_dev, DevBuf& scratch);
// nsteps minimal-residual steps on A e = res, accumulated into x; res is
// updated in place (smoother: no checks, no host synchronisation).  With
// rin and Az given (res = rin - A x on entry), the last step also writes
// Az = rin - res = A x.  keep_res = false: the last step's residual is not
// written back (the caller does not read res afterwards).
template <class C>
void mr_smooth(qd_ctx& ctx, const Op<C>& A, C* x, C* res, C* q, int nrhs, int nsteps, DevBuf& scratch,
               const C* rin = nullptr, C* Az = nullptr, bool keep_res = true);

}  // namespace qd

struct qd_mg;

namespace qd {

// V-cycle preconditioner for level `level` of a hierarchy (Sec. 2 two-grid
// method: coarse-grid correction, then smoothing; deeper levels precondition
// the coarse GCR with the next V-cycle; no recursion below the coarsest,
// where the solve is GCR or, when the coarsest operator was inverted in
// setup, one dense product).
template <class C> class MGPrecond : public Precond<C> {
 public:
  MGPrecond(qd_mg* mg, int level);
  MGPrecond(const MGPrecond&) = delete;
  MGPrecond& operator=(const MGPrecond&) = delete;
  ~MGPrecond();
  void apply(qd_ctx& ctx, const C* r, C* z, int nrhs) override;
  bool apply_az(qd_ctx& ctx, const Op<C>& A, const C* r, C* z, C* Az, int nrhs) override;
  void buffers(std::vector<const void*>& v) const;
  bool sync_free() const;
  // z = W C^{-1} W^H r only (no smoothing).
  void coarse_correction(qd_ctx& ctx, const C* r, C* z, int nrhs);

 private:
  void ensure_buffers(int nrhs);
  void run(qd_ctx& ctx, const C* r, C* z, C* Az, int nrhs);
  void body(qd_ctx& ctx, const C* r, C* z, C* Az, int nrhs);
  bool ends_on_residual() const;
  void drop_graphs();
  qd_mg* mg_;
  int level_;
  std::unique_ptr<MGPrecond<C>> next_;
  GCR<C> coarse_;
  DevBuf rc_, ec_, t_, res_, q_, d_, scratch_;
  int cap_ = -1;
  // Captured fine-level V-cycles, one per (input, output) pair at one nrhs;
  // valid while every buffer in `ptrs` keeps its address.
  struct Graph {
    const void* r = nullptr;
    void* z = nullptr;
    void* Az = nullptr;
    int nrhs = 0;
    std::vector<const void*> ptrs;
    long long kernels = 0;
    cudaGraphExec_t exec = nullptr;
  };
  std::vector<Graph> graphs_;
  struct Seen {
    const void* r;
    void* z;
    void* Az;
  };
  std::vector<Seen> seen_;  // (input, outputs) met once (eager so far)
  int warm_nrhs_ = -1;
  cudaStream_t cap_stream_ = nullptr;  // capture only; nothing runs on it
};

// Odd-site Schur complement of the Wilson operator (the even-odd
// preconditioned fine solves the paper's multigrid uses, Sec. 4):
//   S = A_oo - A_oe A_ee^{-1} A_eo = M - (1/4) H_oe M^{-1} H_eo
// with A = M - H/2, M = 4 + m0 + i tau gamma5, on half fields of the odd
// sites.
template <class C> struct SchurOp : public Op<C> {
  const qd_gauge* g;
  const C* links;
  double m0, tau;
  mutable DevBuf t;  // even-site scratch
  SchurOp(const qd_gauge* gauge, const C* lk, double m, double ta) : g(gauge), links(lk), m0(m), tau(ta) {}
  int64_t nsites() const override;
  int dof() const override { return 12; }
  void apply(qd_ctx& ctx, const C* in, C* out, int nrhs) const override;
};

// Preconditioner of the Schur system from a full-lattice V-cycle: the odd
// block of M_V (0, r_o) (the odd-odd block of A^{-1} is S^{-1}).  The
// embedding buffers persist, so the V-cycle's captured graphs are reused.
template <class C> class SchurPrecond : public Precond<C> {
 public:
  MGPrecond<C>* mg = nullptr;
  const LevelGeom* geo = nullptr;
  // r and z are the odd halves of full fields whose even half of r is zero
  // (GCR::embed): the V-cycle runs on them in place
  bool embedded = false;
  void apply(qd_ctx& ctx, const C* r, C* z, int nrhs) override;

 private:
  DevBuf R_, Z_;
  int cap_ = -1;
};

// A x = b on the full lattice through the Schur complement: b_o' = b_o -
// A_oe A_ee^{-1} b_e; S x_o = b_o' by flexible GCR (tolerance tol relative
// to ||b_o'||, preconditioner pre: nullable); x_e = A_ee^{-1} (b_e - A_eo
// x_o).  b and x full fields (even half first); scratch grow-only.
template <class C>
void schur_solve(qd_ctx& ctx, const qd_gauge& g, const C* links, double m0, double tau, SchurPrecond<C>* pre,
                 GCR<C>& gcr, DevBuf& scratch, const C* b, C* x, int nrhs, double tol, int maxit, int restart,
                 SolveInfo* info);

// Learned gauge-covariant smoother of the fine level (an extension; the
// paper has no counterpart): (S r)(x) = sum_d w_d (T_d r)(x), with T_0 the
// identity, T_{1+mu} r(x) = U_mu(x) r(x+mu), T_{5+mu} r(x) = U_mu(x-mu)^H
// r(x-mu), and w_d 4x4 spin matrices (colour moved by links only).
// With layers > 1, S = S_L ... S_1, each S_l a layer of the same form
// (weights w_l): reach L hops, L applications per use.
struct LearnedSmoother {
  bool enabled = false;
  int mr_steps = 2;                 // minimal-residual steps after S in the V-cycle
  int layers = 1;
  std::vector<cplx> w;              // [layers][9][4][4] FP64 (fitted)
  DevBuf w64;                       // device copy of w
  DevBuf w32;                       // w rounded to FP16, held as float2 (FP32 V-cycle)
  mutable DevBuf t[2];              // intermediate fields of a layered apply (grow-only)
  mutable DevBuf tune_scratch;      // output of the launch-shape timing (released after it)
  double err_learned = 0.0, err_plain = 0.0;
};

void smoother_set_weights(qd_mg& mg, const cplx* w);
// layers x 144 weights (layer-major).
void smoother_set_layers(qd_mg& mg, int layers, const cplx* w);
void smoother_fit(qd_mg& mg, int s, const cplx* e, const cplx* r);
void smoother_train(qd_mg& mg, int s, double solve_tol, uint64_t seed, int mr_steps, int layers, double* err_learned,
                    double* err_plain, int* enabled);
// out = S in (accumulate: out += S in) on the fine level, nrhs columns.
template <class C>
void smoother_apply(qd_ctx& ctx, qd_mg& mg, int nrhs, const C* in, C* out, bool accumulate);

}  // namespace qd

struct qd_mg {
  qd_ctx* ctx = nullptr;
  const qd_gauge* gauge = nullptr;
  double m0 = 0.0, tau = 0.0;
  qd_mg_params p{};
  int nlevels = 0;  // coarse levels
  std::vector<std::unique_ptr<qd::Transfer>> T;     // T[l]: level l -> l+1
  std::vector<std::unique_ptr<qd::CoarseLevel>> L;  // L[l-1]: level l >= 1
  std::unique_ptr<qd::MGPrecond<qd::cplx>> pre64;
  std::unique_ptr<qd::MGPrecond<qd::cplxf>> pre32;
  std::unique_ptr<qd::LearnedSmoother> ls;  // fine-level learned smoother (nullable)

  const qd::LevelGeom& geom(int level) const { return level == 0 ? gauge->geo : L[level - 1]->geo; }
  int dof(int level) const { return level == 0 ? 12 : L[level - 1]->D; }
  // Operator of a level in precision C (caller owns the returned object).
  template <class C> std::unique_ptr<qd::Op<C>> op(int level);
  template <class C> const C* W(int level);
  // Dense inverse of coarse level `level` (>= 1), or nullptr.
  template <class C> const C* Cinv(int level);
};
