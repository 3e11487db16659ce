/*
 * qdtrace.h -- C ABI of libqdtrace, a single-GPU (sm_103a) library for the
 * deflated Hutchinson estimator of tr(A^{-1}) for the 4-D Wilson-Dirac
 * operator A, following "Multigrid deflation for Lattice QCD" (Romero,
 * Stathopoulos, Orginos, arXiv:1909.12234).
 *
 * ---------------------------------------------------------------------------
 * Conventions (all entry points)
 * ---------------------------------------------------------------------------
 * Status:    every function returns QD_OK (0) or a negative qd_status code.
 *            qd_last_error() returns a message for the last failure on the
 *            calling host thread.  No C++ exception crosses this ABI.
 * Streams:   every device computation is issued on the stream given to
 *            qd_ctx_create().  Functions that return host results
 *            (statistics, solve stats, eigenvalues) synchronise that stream;
 *            the others are asynchronous unless stated.
 * Ownership: pointers passed in are owned by the caller and never freed by
 *            the library.  Device buffers must stay valid until the stream
 *            has finished the call.  Opaque handles (qd_ctx, qd_gauge, qd_mg,
 *            qd_defl) are owned by the library and freed by *_destroy.
 *            The library allocates its own device work space on first use.
 * Threads:   a qd_ctx, and the qd_gauge / qd_mg / qd_defl handles used with
 *            it, serve one host thread at a time.  qd_hutchinson_batch runs
 *            its own worker threads and streams internally.  Process-wide
 *            state (the launch counter, the autotuner table, kernels'
 *            shared-memory limits) is guarded for concurrent use.
 * Numbers:   complex numbers are two doubles (re, im), FP64 (the *_f32
 *            entry points take two floats).
 *
 * Lattice:   dims = {Lx, Ly, Lz, Lt}, periodic; Lx must be even.
 *            lexicographic site  lex = x + Lx*(y + Ly*(z + Lz*t));
 *            parity p = (x+y+z+t) mod 2;
 *            even-odd site       eo  = p * V/2 + lex/2   (V = Lx Ly Lz Lt).
 *            Direction mu = 0..3 is x, y, z, t.
 *
 * Field layout ("qd layout"), used by every device field argument:
 *   fine level   : element (eo site i, a, r) at complex offset
 *                  (i * 12 + a) * nrhs + r,  a = 3*spin + colour,
 *                  r = right-hand side 0..nrhs-1 (innermost);
 *   coarse level l>=1: element (coarse lex site i, d, r) at
 *                  (i * dc + d) * nrhs + r,  dc = 2*nv[l-1]; coarse sites are
 *                  lexicographic on the coarse lattice dims / block;
 *                  d < nv is chirality +1, d >= nv chirality -1.
 * Spin basis: chiral, gamma5 = diag(1, 1, -1, -1).
 *
 * The operator (no paper passage writes it out; the paper uses the Wilson
 * operator and its gamma5-Hermiticity, Sec. 2.1 and Sec. 3):
 *   (A x)(n) = (4 + m0) x(n)
 *              - 1/2 sum_mu [(1 - gamma_mu) U_mu(n) x(n+mu)
 *                            + (1 + gamma_mu) U_mu(n-mu)^H x(n-mu)]
 *              + i tau gamma5 x(n)          (tau: shift of Sec. 3.2)
 */
#ifndef QDTRACE_H
#define QDTRACE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QD_ABI_VERSION 6
#define QD_MAX_LEVELS 4 /* fine level + up to 3 coarse levels */

typedef enum {
  QD_OK = 0,
  QD_ERR_INVALID = -1,       /* bad argument, size or layout */
  QD_ERR_CUDA = -2,          /* a CUDA runtime call failed */
  QD_ERR_OOM = -3,           /* device allocation failed */
  QD_ERR_NOT_CONVERGED = -4, /* solver hit maxit; stats are still filled */
  QD_ERR_NONFINITE = -5,     /* NaN/Inf met in an input or a reduction */
  QD_ERR_TIMEOUT = -6,       /* a bounded device wait gave up */
  QD_ERR_INTERNAL = -7
} qd_status;

typedef struct qd_ctx qd_ctx;
typedef struct qd_gauge qd_gauge;
typedef struct qd_mg qd_mg;
typedef struct qd_defl qd_defl;

/* ------------------------------------------------------------------------ */
/* Context and errors                                                        */
/* ------------------------------------------------------------------------ */

/* ABI version of the loaded library (QD_ABI_VERSION it was built with). */
int qd_abi_version(void);

/* Message of the last failure on this host thread ("" if none). */
const char* qd_last_error(void);

/* Create a context on CUDA device `device`, issuing work on `stream`
 * (a cudaStream_t; NULL = legacy default stream). */
int qd_ctx_create(qd_ctx** ctx, int device, void* stream);
int qd_ctx_destroy(qd_ctx* ctx);

/* ------------------------------------------------------------------------ */
/* Geometry (Sec. 1 red-black partitioning; even-odd layout)                 */
/* ------------------------------------------------------------------------ */

/* Host-only: eo_of_lex[lex] = even-odd index of every site (V entries,
 * caller-allocated host array).  QD_ERR_INVALID for odd Lx or dims < 1. */
int qd_eo_index(const int dims[4], int64_t* eo_of_lex);

/* ------------------------------------------------------------------------ */
/* Gauge field                                                               */
/* ------------------------------------------------------------------------ */

/* Upload links.  links_host: host array [V][4][3][3] complex, lexicographic
 * sites, U_mu(n)[row][col] on the link n -> n + mu.  Copied; the caller may
 * free it on return.  Synchronous. */
int qd_gauge_create(qd_ctx* ctx, const int dims[4], const double* links_host,
                    qd_gauge** gauge);
int qd_gauge_destroy(qd_gauge* gauge);

/* Reorder fields between the canonical host order [r][V lex][12] (each
 * right-hand side a contiguous lexicographic vector) and the qd layout.
 * to_qd != 0: canon -> qd; 0: qd -> canon.  Both are device buffers of
 * 12 V nrhs complex numbers and must not overlap. */
int qd_field_reorder(qd_ctx* ctx, const qd_gauge* gauge, int nrhs, int to_qd,
                     const double* in, double* out);

/* ------------------------------------------------------------------------ */
/* a1: Rademacher noise (Sec. 1, Eq. 1: x_j with entries +-1)                */
/* ------------------------------------------------------------------------ */

/* out (qd layout, nrhs columns): real +-1 noise for global samples
 * sample_offset .. sample_offset+nrhs-1.  Dof i = 12*lex + a of sample j is
 * bit (i mod 128) of Philox4x32-10(counter = (i/128, j, 0, 0),
 * key = (seed & 0xffffffff, seed >> 32)) (word (i mod 128)/32, bit i mod 32);
 * bit 0 -> +1, bit 1 -> -1; imaginary part 0.  Bit-exact on any device. */
int qd_rademacher(qd_ctx* ctx, const qd_gauge* gauge, uint64_t seed,
                  int64_t sample_offset, int nrhs, double* out);

/* ------------------------------------------------------------------------ */
/* a2: Wilson-Dirac operator (Sec. 2 two-grid method acts with A; Sec. 3.2   */
/* shift i tau gamma5)                                                       */
/* ------------------------------------------------------------------------ */

/* out = A in (dagger = 0) or A^H in (dagger != 0), nrhs columns, qd layout.
 * in and out must not overlap.  Asynchronous. */
int qd_dirac_apply(qd_ctx* ctx, const qd_gauge* gauge, double m0, double tau,
                   int dagger, int nrhs, const double* in, double* out);

/* The same operator in FP32 (the arithmetic of the mixed-precision inner
 * solves): in/out are interleaved complex float (re, im) in qd layout,
 * links rounded once to FP32 and cached on the gauge (the first call
 * allocates that copy, so gauge is not const).  Same errors as
 * qd_dirac_apply; a bounded wait of the stencil's bulk-staged launch shape
 * that gives up is reported as QD_ERR_TIMEOUT by the next synchronising
 * call on the gauge (qd_dirac_schur_apply_f32, qd_solve,
 * qd_hutchinson_trace).  Asynchronous. */
int qd_dirac_apply_f32(qd_ctx* ctx, qd_gauge* gauge, double m0, double tau,
                       int dagger, int nrhs, const float* in, float* out);

/* r = b - A x (or b - A^H x) in FP32, the residual form of the same
 * stencil (the subtraction in the kernel's epilogue, as the mixed-precision
 * inner solves use it).  b, x, r: interleaved complex float in qd layout;
 * r must not overlap b or x.  A bounded wait of the bulk-staged form of the
 * FP32 stencil that gives up is reported as QD_ERR_TIMEOUT by the next
 * synchronising call on the gauge (qd_dirac_schur_apply_f32, qd_solve,
 * qd_hutchinson_trace).  Asynchronous. */
int qd_dirac_residual_f32(qd_ctx* ctx, qd_gauge* gauge, double m0, double tau,
                          int dagger, int nrhs, const float* b,
                          const float* x, float* r);

/* out = S in with S = A_oo - A_oe A_ee^{-1} A_eo, the Schur complement of A
 * on the odd sites (the even-odd solves of Sec. 4; qd_solver_params.schur).
 * in/out: half fields of the odd sites, (site - V/2, 12, nrhs) for the odd
 * half of the qd layout (sites V/2 .. V-1).  in and out must not overlap.
 * Returns after the stream has finished the product. */
int qd_dirac_schur_apply(qd_ctx* ctx, const qd_gauge* gauge, double m0,
                         double tau, int nrhs, const double* in, double* out);
/* The same in FP32 (interleaved complex float, links as
 * qd_dirac_apply_f32); QD_ERR_TIMEOUT when a bounded wait of the stencil
 * gave up in this or an earlier FP32 stencil call on the gauge. */
int qd_dirac_schur_apply_f32(qd_ctx* ctx, qd_gauge* gauge, double m0,
                             double tau, int nrhs, const float* in,
                             float* out);

/* ------------------------------------------------------------------------ */
/* a10: adaptive multigrid setup (Sec. 2 "adaptive setup" and "blocking";    */
/* Sec. 4 tolerance 1e-2 / 200 iterations; Algorithm 2 step 1)              */
/* ------------------------------------------------------------------------ */

typedef struct {
  int nlevels;                  /* coarse levels to build, 1..QD_MAX_LEVELS-1 */
  int block[QD_MAX_LEVELS][4];  /* block[l] = aggregate shape on level l */
  int nv[QD_MAX_LEVELS];        /* null vectors on level l (coarse dof 2 nv) */
  double null_tol;              /* relative residual of A y = 0 (1e-2) */
  int null_maxit;               /* minimal-residual steps cap (200) */
  uint64_t seed;                /* level l uses seed + l for its starts */
  int smoother_steps;           /* minimal-residual post-smoothing steps */
  double coarse_tol;            /* relative tolerance of coarse GCR */
  int coarse_maxit;             /* iteration cap of coarse GCR; with
                                   coarse_tol <= 0 exactly this many
                                   iterations, no convergence checks */
  int coarse_restart;           /* restart length of coarse GCR */
  int coarsest_direct;          /* > 0: invert the coarsest operator densely
                                   (FP32 Gauss-Jordan with partial pivoting
                                   in setup) when its dimension is <= this
                                   value (at most 16384); every coarsest
                                   solve in a V-cycle is then one dense
                                   product.  0: coarsest GCR */
  int coarsest_bf16;            /* with a dense coarsest inverse: != 0 lets
                                   the FP32 V-cycle apply it as one BF16
                                   tcgen05 tensor-core GEMM (FP32
                                   accumulate); 0 uses FP32 CUDA cores */
  int use_graphs;               /* != 0: when the V-cycle needs no host
                                   synchronisation (dense coarsest inverse
                                   below the first coarse level, and
                                   coarse_tol <= 0 on the levels between),
                                   each fine-level V-cycle is captured once
                                   per (input, output, nrhs) as a CUDA graph
                                   and replayed; the result is the same as
                                   the eager launches.  Off while profiling */
  int coarse_tc;                /* != 0: the FP32 V-cycle applies coarse
                                   stencils with dof 8, 16, 24 or 32
                                   (qd_coarse_apply_tc) and restrictions with
                                   fine dof 12, 16, 24 or 32 and coarse dof
                                   16, 24 or 32 (qd_restrict_tc) on the
                                   tcgen05 tensor cores (split-BF16 operands,
                                   FP32 accumulate); 0: FP32 CUDA cores */
  int coarse_smoother_steps;    /* minimal-residual post-smoothing steps of
                                   the V-cycles on coarse levels; < 0: the
                                   same as smoother_steps */
  int null_f32;                 /* 1: the null-vector iterations run in FP32
                                   (FP32 operators; the vectors only need
                                   null_tol, 1e-2); 0 (default): FP64, the
                                   oracle's arithmetic */
} qd_mg_params;

/* Fill `p` with this library's defaults (1 level, 2^4 blocks, nv 12,
 * 1e-2 / 200, 4 smoothing steps, coarse GCR to 0.1 / 256 / 16, direct
 * coarsest solve on, BF16 tensor cores for the coarsest solve and the coarse
 * stencils of the FP32 V-cycle, CUDA graphs on). */
void qd_mg_params_default(qd_mg_params* p);

/* Build the hierarchy for A(m0, tau).  Null-vector starts are complex
 * +-1 +-i signs: re from bit 2(i mod 64), im from bit 2(i mod 64)+1 of
 * Philox(counter = (i/64, v, 1, 0), key = seed + level) with i the dof index
 * lex_site * dof + d of that level.  injected_null (nullable): device array
 * of the level-0 null vectors in qd layout with nrhs = nv[0]; when given the
 * level-0 iteration is skipped (used to compare implementations).
 * Synchronous. */
int qd_mg_setup(qd_ctx* ctx, const qd_gauge* gauge, double m0, double tau,
                const qd_mg_params* params, const double* injected_null,
                qd_mg** mg);
int qd_mg_destroy(qd_mg* mg);

/* Sizes of level l (0 = fine): dims[4], dofs per site and number of sites.
 * Also the minimal-residual steps each level-l null vector took (host array
 * of nv[l] ints, nullable; zeros for injected vectors). */
int qd_mg_level_info(const qd_mg* mg, int level, int dims[4], int* dof,
                     int64_t* nsites, int* null_steps);

/* ------------------------------------------------------------------------ */
/* a3: prolongation W c and restriction W^H x (Sec. 2 two-grid step 1)       */
/* ------------------------------------------------------------------------ */

/* fine (level l, qd layout) = W_l coarse (level l+1).  Asynchronous. */
int qd_prolongate(qd_mg* mg, int level, int nrhs, const double* coarse,
                  double* fine);
/* coarse (level l+1) = W_l^H fine (level l).  Asynchronous. */
int qd_restrict(qd_mg* mg, int level, int nrhs, const double* fine,
                double* coarse);
/* fine = W_l coarse in FP32, the kernel of the FP32 V-cycle: W rounded to
 * FP32, FP32 products summed over the nv vectors of the component's
 * chirality in index order.  coarse and fine: FP32 complex (re, im) device
 * fields, layouts as qd_prolongate.  Asynchronous. */
int qd_prolongate_f32(qd_mg* mg, int level, int nrhs, const float* coarse,
                      float* fine);

/* coarse (level l+1) = W_l^H fine (level l) in FP32 on the tcgen05 tensor
 * cores (the form the FP32 V-cycle uses with qd_mg_params.coarse_tc): per
 * aggregate and chunk of <= 128 right-hand sides one real GEMM over the
 * aggregate's fine sites, each operand split into two BF16 terms
 * (hi = bf16(v), lo = bf16(v - hi)), products hi*hi + hi*lo + lo*hi with FP32
 * accumulation (error about 3 * 2^-16 sum |W||fine| per output).  Needs fine
 * dof 12, 16, 24 or 32, coarse dof 16, 24 or 32, 16-byte aligned interleaved
 * complex float fields, nrhs even above 128 (QD_ERR_INVALID otherwise).
 * Timeouts as qd_coarse_apply_tc.  Asynchronous. */
int qd_restrict_tc(qd_mg* mg, int level, int nrhs, const float* fine, float* coarse);

/* ------------------------------------------------------------------------ */
/* a4: coarse operator C_l = W^H A W (Sec. 2, "V^H A V")                     */
/* ------------------------------------------------------------------------ */

/* out = C_level in, level >= 1, 9-point block stencil.  Asynchronous. */
int qd_coarse_apply(qd_mg* mg, int level, int nrhs, const double* in,
                    double* out);

/* The same stencil in FP32 (the arithmetic of the mixed-precision V-cycle):
 * in/out are interleaved complex float in the level's qd layout; the FP32
 * copy of C_level is made on first use.  Same errors as qd_coarse_apply.
 * Asynchronous. */
int qd_coarse_apply_f32(qd_mg* mg, int level, int nrhs, const float* in,
                        float* out);

/* The same stencil as a dense contraction on the tcgen05 tensor cores (the
 * form the FP32 V-cycle uses with qd_mg_params.coarse_tc): per coarse site
 * and chunk of <= 128 right-hand sides one real GEMM (M = right-hand sides,
 * N = 2 dof, K = 9 x 2 dof).  Each operand is split into two BF16 terms
 * (hi = bf16(v), lo = bf16(v - hi)) and the product formed as
 * hi*hi + hi*lo + lo*hi with FP32 accumulation, so each output's error is
 * about 3 * 2^-16 sum |C||in| (plain BF16, 2^-7, perturbs the small singular
 * values of a near-critical coarse operator too much).  The level's dof must
 * be 8, 16, 24 or 32, in/out 16-byte aligned interleaved complex float,
 * nrhs even when above 128 (QD_ERR_INVALID otherwise).  A bounded wait that gives up is reported as QD_ERR_TIMEOUT by
 * the next synchronising call on the hierarchy (qd_coarse_solve*, qd_solve,
 * qd_hutchinson_trace).  Asynchronous. */
int qd_coarse_apply_tc(qd_mg* mg, int level, int nrhs, const float* in,
                       float* out);
/* Residual form of the same kernel, r = b - C x (the subtraction in the
 * kernel's epilogue, in FP32: the same bits as b - (C x) stored first).
 * b, x, r distinct.  Asynchronous. */
int qd_coarse_residual_tc(qd_mg* mg, int level, int nrhs, const float* b,
                          const float* x, float* r);

/* out = C_level^{-1} in, level >= 1: the coarse solve of the V-cycle (a5).
 * On the coarsest level with a dense inverse: the product with the inverse
 * followed by three residual corrections with the FP64 operator (FP64
 * accuracy for coarse condition numbers up to ~1e5); otherwise GCR on
 * C_level to coarse_tol (preconditioned by the next level's V-cycle when
 * there is one).  Synchronous. */
int qd_coarse_solve(qd_mg* mg, int level, int nrhs, const double* in,
                    double* out);

/* The coarse solve of the FP32 V-cycle used by QD_PREC_MIXED: in and out are
 * complex FP32 (2 floats) in the level's qd layout.  On the coarsest level
 * with a dense inverse this is the BF16 tensor-core product (coarsest_bf16)
 * or the FP32 CUDA-core one; otherwise QD_ERR_INVALID.  Returns
 * QD_ERR_TIMEOUT if a bounded device wait of the tensor-core kernel gave
 * up.  Synchronous. */
int qd_coarse_solve_f32(qd_mg* mg, int level, int nrhs, const float* in,
                        float* out);

/* ------------------------------------------------------------------------ */
/* a5/a6: solves A x = b to ||b - A x|| <= tol ||b|| (Sec. 1, inexact solve; */
/* Sec. 2 multigrid preconditioning, GCR)                                    */
/* ------------------------------------------------------------------------ */

enum {
  QD_PREC_F64 = 0,   /* FP64 flexible GCR, FP64 V-cycle */
  QD_PREC_MIXED = 1  /* FP64 true-residual refinement around FP32 flexible
                        GCR with an FP32 V-cycle */
};

typedef struct {
  double tol;        /* xi: stop when ||b - A x|| <= tol ||b|| (FP64 residual) */
  int maxit;         /* iteration cap (outer GCR, or inner GCR per refinement) */
  int restart;       /* GCR restart length */
  int precision;     /* QD_PREC_* */
  double inner_tol;  /* QD_PREC_MIXED: relative tolerance of each FP32 solve */
  int max_refine;    /* QD_PREC_MIXED: cap on refinement steps */
  int stag_window;   /* > 0: stagnation test (Sec. 3.2, the inverter that
                        "stagnates at an error level well above xi"): every
                        stag_window iterations, a column whose residual fell
                        by less than 10 % since the previous check stops the
                        solve with QD_ERR_NOT_CONVERGED and
                        qd_solve_stats.stagnated = 1; 0: off */
  int schur;         /* 1: even-odd solve (Sec. 4, the even-odd
                        preconditioned fine solves): GCR on the odd-site
                        Schur complement S = A_oo - A_oe A_ee^{-1} A_eo,
                        preconditioned by the odd block of the V-cycle, then
                        x_e = A_ee^{-1} (b_e - A_eo x_o); with QD_PREC_MIXED
                        each FP32 correction is solved this way.  The
                        tolerance still applies to the full FP64 residual.
                        0 (default): GCR on A itself */
} qd_solver_params;

/* Fills *p with the defaults given beside each field above (NULL: no-op). */
void qd_solver_params_default(qd_solver_params* p);

typedef struct {
  int iterations;                /* max outer iterations over the columns */
  int converged;                 /* columns whose TRUE residual met tol */
  double max_true_rel_residual;  /* max over columns of ||b-Ax||/||b|| */
  int* iters_per_rhs;            /* optional host [nrhs] */
  double* true_rel_residual;     /* optional host [nrhs] */
  int stagnated;                 /* 1: stopped by the stagnation test */
} qd_solve_stats;

/* Solve A(m0, tau) x = b for nrhs columns.  QD_PREC_F64: flexible
 * restarted GCR right-preconditioned by the FP64 V-cycle of `mg` (nullable:
 * unpreconditioned).  QD_PREC_MIXED: x = 0, r = b; repeat { solve
 * A e = r / ||r|| in FP32 (flexible GCR, FP32 V-cycle) to inner_tol;
 * x += ||r|| e; r = b - A x in FP64 } until the FP64 residual meets tol.
 * With mg the operator is mg's.  x is overwritten.  Returns
 * QD_ERR_NOT_CONVERGED if a column missed tol (stats filled).
 * Synchronous. */
int qd_solve(qd_ctx* ctx, const qd_gauge* gauge, qd_mg* mg, double m0,
             double tau, int nrhs, const double* b, double* x,
             const qd_solver_params* params, qd_solve_stats* stats);

/* ------------------------------------------------------------------------ */
/* a7: deflation space (Algorithm 1 step 1; Algorithm 2 steps 1-4)           */
/* ------------------------------------------------------------------------ */

enum {
  QD_DEFL_EIG_ORTHO = 1,  /* Algorithm 1: k eigenvectors of A gamma5 */
  QD_DEFL_MG_OBLIQUE = 2  /* Algorithm 2: k eigenvectors of C gamma5^W */
};

typedef struct {
  int kind;          /* QD_DEFL_* */
  int k;             /* rank of the deflation space */
  int guard;         /* extra subspace-iteration vectors (>= 0) */
  double eig_tol;    /* stop when ||H u - mu u|| <= eig_tol |mu| for all k */
  double solve_tol;  /* xi of the inner solves H^{-1} */
  int maxit;         /* subspace iterations cap */
  uint64_t seed;     /* starting block: Philox random starts, this key */
  /* Sec. 3.2, eigensolver tuning (kind 1, whose eigensolver runs inexact
   * multigrid solves with the fine operator): when an inner solve
   * stagnates (stag_window iterations without a 10 % residual drop) or
   * fails to converge, the multigrid inverter is rebuilt for the shifted
   * operator A + i tau_eig gamma5 and the eigensolver restarts, with
   * tau_eig = tau_restart at the first restart and 4x larger at each next
   * one, at most max_restarts times.  (A gamma5 + i tau)^{-1} has the
   * eigenvectors of A gamma5, so the space deflates the unshifted A; the
   * Rayleigh-Ritz step then works on the Hermitian Y^H Y of
   * Y = (A gamma5 + i tau)^{-1} X (eigenvalues 1/(lambda^2 + tau^2)), and
   * lambda = Re 1/mu from the Rayleigh quotient mu of Y. */
  double tau_restart;  /* first shift (0.1) */
  int max_restarts;    /* (3) */
  int stag_window;     /* inner-solve stagnation window (100); 0: off */
  int solve_restart;   /* restart length of the inner GCR (32) */
  int fail_first;      /* test hook: report the first fail_first attempts
                          as stagnated without solving (0) */
} qd_defl_params;

/* Fills *p with the defaults given beside each field above (NULL: no-op). */
void qd_defl_params_default(qd_defl_params* p);

/* Build a deflation space for A(m0, tau) (tau taken from mg for kind 2).
 * kind 1 needs mg only as the solver's preconditioner (nullable); kind 2
 * needs mg (level 1 is used).  injected_basis (nullable device array):
 * kind 2: U_bar in level-1 qd layout with nrhs = k; kind 1: U in level-0 qd
 * layout with nrhs = k (orthonormal columns); skips the eigensolver.
 * Synchronous. */
int qd_defl_create(qd_ctx* ctx, const qd_gauge* gauge, qd_mg* mg, double m0,
                   double tau, const qd_defl_params* params,
                   const double* injected_basis, qd_defl** defl);
int qd_defl_destroy(qd_defl* defl);

/* Set the active rank r <= k (Algorithm 2 step 3 on the leading r columns;
 * Algorithm 1 keeps the first r vectors) and return t0 (complex, 2 doubles).
 * Synchronous. */
int qd_defl_set_rank(qd_defl* defl, int rank, double* t0);

/* Host copies: eigenvalues mu of the eigensolve (k, nullable), Lambda of
 * the active rank (rank, nullable), iterations taken (nullable). */
int qd_defl_info(const qd_defl* defl, double* mu, double* lambda,
                 int* iterations);

/* The eigensolver's shift after its restarts (0 without one) and the number
 * of restarts it took (Sec. 3.2; qd_defl_params.tau_restart). */
int qd_defl_shift_info(const qd_defl* defl, double* tau_eig, int* restarts);

/* Kind 2: G = U_bar^H gamma5^W C U_bar (host, k x k complex, row major),
 * the matrix whose leading r x r block gives the rank-r correction of
 * qd_deflate_coeffs (Sec. 2.2).  QD_ERR_INVALID for kind 1 (G = I). */
int qd_defl_gram(const qd_defl* defl, double* G);

/* Copy the k basis vectors (kind 1: U on the fine level; kind 2: U_bar on
 * the coarsest level), qd layout with nrhs = k, to the caller's device
 * buffer `out`.  Asynchronous. */
int qd_defl_basis(const qd_defl* defl, double* out);

/* ------------------------------------------------------------------------ */
/* a8: deflation projection (Algorithm 1 step 3, Algorithm 2 step 5,         */
/* Sec. 2.2 a-posteriori filtering)                                          */
/* ------------------------------------------------------------------------ */

/* out = (I - P) z on the fine level, nrhs columns, qd layout:
 *   kind 2: P = A W U Lambda^{-1} U^H gamma5^W W^H (K = gamma5 projector);
 *   kind 1: P = U U^H.
 * Uses the active rank.  z and out must not overlap (QD_ERR_INVALID).
 * Asynchronous. */
int qd_deflate_project(qd_defl* defl, int nrhs, const double* z, double* out);

/* The paper has no counterpart to this entry point.  It serves callers that
 * cannot let the library allocate device memory during a call: an
 * application that gives all device memory to its own pool up front (a
 * cudaMalloc inside the call would then fail), or a latency-critical loop
 * that must not pay for cudaMalloc and cudaFree (both can synchronise the
 * device).  qd_deflate_project allocates and frees small device buffers for
 * U^H z on every call; this variant computes the same result for a space of
 * orthonormal eigenvectors (QD_DEFL_EIG_ORTHO) at its active rank,
 *     out = (I - U U^H) z,
 * but keeps its scratch (the rank x nrhs coefficients and their partial
 * sums) in one fixed 8 MiB __device__ array compiled into the library.  It
 * calls no cudaMalloc, cudaFree or other allocating routine: qd_alloc_count()
 * does not move across a call.
 *   - QD_DEFL_EIG_ORTHO spaces only; QD_ERR_INVALID for other kinds, when
 *     rank * nrhs > 262144 (the array's limit) and when z and out overlap.
 *   - The array exists once per device that loads the library and stays
 *     allocated until the process exits.  qd_ctx_create takes it: with the
 *     context's device current it looks up the array's device address
 *     (cudaGetSymbolAddress, which also loads the module holding the array,
 *     so that is when its 8 MiB are allocated) and loads the kernels this
 *     call launches.  The call itself uses the address kept in the context
 *     that `defl` was created with.
 *   - Every call on a device uses the same array and leaves the last call's
 *     values in it: calls whose GPU work overlaps (other streams, threads or
 *     contexts on the same device) race; issue them on one stream.
 * Asynchronous, like qd_deflate_project. */
int qd_deflate_project_static(qd_defl* defl, int nrhs, const double* z,
                              double* out);

/* Sec. 2.2 matrices for an a-posteriori rank sweep, host outputs,
 * row-major complex, over all k columns of the space:
 *   kind 2: ZhV [nrhs][k] = Z^H W U_bar, UhKZ [k][nrhs] = U_bar^H gamma5^W
 *           W^H Z; the rank-r correction of sample j is
 *           ZhV[j][:r] G_r^{-1} UhKZ[:r][j], G = U_bar^H gamma5^W C U_bar;
 *   kind 1: ZhV [nrhs][k] = Z^H A^{-1}_xi U (the solves of Algorithm 1,
 *           step 2), UhKZ [k][nrhs] = U^H Z (K = I); the rank-r correction
 *           is sum_{i<r} ZhV[j][i] UhKZ[i][j].
 * With qd_defl_set_rank's t0 at rank r, t0 + mean_j (t_j - correction_j)
 * is the rank-r estimate from undeflated t_j = z_j^H A^{-1}_xi z_j.
 * Synchronous. */
int qd_deflate_coeffs(qd_defl* defl, int nrhs, const double* z, double* ZhV,
                      double* UhKZ);

/* Sec. 4.1 (Fig. 3, right): sin of the angle between each of the k columns
 * v_i of V (fine level, qd layout, device, k columns) and the range of the
 * composite prolongator W = W_0 ... W_{depth-1} (orthonormal):
 * sin_out[i] = ||v_i - W W^H v_i|| / ||v_i|| (host array of k doubles).
 * depth in [1, nlevels].  Synchronous. */
int qd_mg_subspace_sines(qd_mg* mg, int depth, int k, const double* V, double* sin_out);

/* ------------------------------------------------------------------------ */
/* a9: deflated Hutchinson estimator (Eq. 1; Algorithms 1 and 2)             */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint64_t seed;          /* noise key */
  int64_t sample_offset;  /* first global sample index */
  int nsamples;           /* s, solved together as one multi-RHS batch */
  qd_solver_params solver;/* xi = solver.tol and the solve's settings */
  int dilution;           /* 0: none (H = I); 12: spin-colour dilution, the
                             probing basis H of Algorithms 1 and 2 with its 12
                             spin-colour vectors: every sample z_j becomes the
                             12 vectors z_jh (entries of z_j with 3 spin +
                             colour = h) and t_j = sum_h z_jh^H A^{-1}_xi
                             (I - P) z_jh, 12 s right-hand sides solved
                             together */
} qd_trace_params;

typedef struct {
  double t0[2];            /* deterministic part (0 without deflation) */
  double mean[2];          /* (1/s) sum_j t_j */
  double estimate[2];      /* t0 + mean */
  double var;              /* (1/(s-1)) sum |t_j - mean|^2 */
  double var_re;           /* same for Re t_j */
  double stderr_mean;      /* sqrt(var / s) */
  double var_jackknife_err;/* delete-one jackknife error of var */
  int nsamples;
  int iterations;          /* outer GCR iterations (max over samples) */
  double max_true_rel_residual;
  double* t_samples;       /* optional host [nsamples][2]: t_j */
  double* ZhV;             /* optional host [nsamples][k][2] (kind 2) */
  double* UhKZ;            /* optional host [k][nsamples][2] (kind 2) */
} qd_trace_result;

/* One batch of the deflated estimator: z_j = Rademacher(seed, offset + j),
 * b_j = (I - P) z_j (defl nullable: P = 0), x_j = A^{-1}_xi b_j by qd_solve
 * with mg (nullable), t_j = z_j^H x_j (with dilution: the sum over the 12
 * spin-colour parts of z_j); statistics accumulated on the device with
 * compensated FP64 sums in a fixed order.  ZhV / UhKZ (kind 1 or 2) are not
 * available with dilution (QD_ERR_INVALID).  Synchronous.  Returns
 * QD_ERR_NOT_CONVERGED (result filled) if any solve missed tol. */
int qd_hutchinson_trace(qd_ctx* ctx, const qd_gauge* gauge, qd_mg* mg,
                        qd_defl* defl, double m0, double tau,
                        const qd_trace_params* params,
                        qd_trace_result* result);

/* One estimator problem of a batch: the arguments of qd_hutchinson_trace,
 * plus its outcome. */
typedef struct {
  const qd_gauge* gauge;
  qd_mg* mg;               /* nullable; distinct across the batch */
  qd_defl* defl;           /* nullable; distinct across the batch */
  double m0, tau;
  qd_trace_params params;
  qd_trace_result* result; /* host, filled as by qd_hutchinson_trace */
  int status;              /* out: QD_OK, QD_ERR_NOT_CONVERGED or the
                              item's own error code */
} qd_batch_item;

/* Independent estimators of uneven size (different lattices, masses and
 * sample counts: Eq. 1 with Algorithm 1 or 2 per item) solved concurrently
 * on one device: nstreams (1..64) worker streams, each driven by its own
 * host thread, take the items largest first (V x nsamples).  Every item's
 * arithmetic is that of qd_hutchinson_trace on the same inputs, so its
 * results are bit-identical to a lone call.  Items may share a gauge; an mg
 * or defl handle may appear in one item only (QD_ERR_INVALID otherwise).
 * Work is ordered after everything already queued on ctx's stream.
 * Synchronous.  Returns QD_OK when every item is QD_OK, else the first
 * failing item's code (QD_ERR_NOT_CONVERGED when that is the only kind of
 * failure); per-item codes are in items[i].status. */
int qd_hutchinson_batch(qd_ctx* ctx, int nitems, qd_batch_item* items,
                        int nstreams);

/* ------------------------------------------------------------------------ */
/* Learned gauge-covariant smoother of the fine level (an extension of the  */
/* V-cycle's smoothing step; the paper has no counterpart)                   */
/* ------------------------------------------------------------------------ */
/* (S r)(x)_{o,a} = sum_{d=0..8} sum_i w[d][o][i] (T_d r)(x)_{i,a}: T_0 = 1,
 * T_{1+mu} r(x) = U_mu(x) r(x+mu), T_{5+mu} r(x) = U_mu(x-mu)^H r(x-mu),
 * w[d] 4x4 spin matrices (144 complex weights; colour is moved only by the
 * links, so S is gauge covariant).  With the smoother enabled the fine
 * V-cycle smooths by z += S (r - A z) followed by mr_steps minimal-residual
 * steps instead of smoother_steps plain ones; the FP32 V-cycle applies the
 * weights rounded to FP16 with FP32 arithmetic. */

typedef struct {
  int nsamples;      /* training pairs; the held-out set has as many (8) */
  double solve_tol;  /* relative residual of the solves e = A^{-1} r (1e-6) */
  uint64_t seed;     /* Philox key of the random vectors (4242) */
  int mr_steps;      /* minimal-residual steps after S in the V-cycle (2) */
  int layers;        /* 1 (default) - 4: S = S_L ... S_1, a stack of layers of
                        the form above (L-hop reach, L applications per use),
                        trained layer by layer: S_l fits e ~ S_l (S_{l-1} ...
                        S_1 r) with the layers below fixed */
} qd_smoother_params;

typedef struct {
  double err_learned;  /* held-out mean ||e - x|| / ||e|| after S + mr_steps */
  double err_plain;    /* the same after smoother_steps plain MR steps */
  int enabled;         /* err_learned < err_plain: the V-cycle now uses S */
} qd_smoother_info;

/* Fills *p with the defaults given beside each field above (NULL: no-op). */
void qd_smoother_params_default(qd_smoother_params* p);

/* Train on pairs the solver generates: for random vectors v (Philox starts,
 * key seed), r = v - A W C^{-1} W^H v is the residual the smoother sees and
 * e = A^{-1} r (FP64 MG-preconditioned GCR to solve_tol); w minimises
 * sum ||e - S r||^2 (linear least squares), then a held-out set judges S
 * against the plain smoother and enables S only if it leaves a smaller
 * error.  Synchronous. */
int qd_smoother_train(qd_mg* mg, const qd_smoother_params* p, qd_smoother_info* info);

/* Least-squares weights for caller pairs (device, fine qd layout, nrhs
 * columns each); the enabled state is unchanged.  Synchronous. */
int qd_smoother_fit(qd_mg* mg, int nrhs, const double* e, const double* r);

/* Host weights w[9][4][4] (complex, 2 doubles each): set (one layer) /
 * read (the first layer). */
int qd_smoother_set_weights(qd_mg* mg, const double* w);
int qd_smoother_get_weights(const qd_mg* mg, double* w);
/* Layered form: layers (1-4) x 144 complex weights, first layer first (the
 * layer applied first to r). */
int qd_smoother_set_layer_weights(qd_mg* mg, int layers, const double* w);
/* Number of layers of the current weights (0: none), and their weights
 * (layers x 144 complex, host). */
int qd_smoother_layers(const qd_mg* mg);
int qd_smoother_get_layer_weights(const qd_mg* mg, double* w);

/* Use S in the V-cycle (enabled != 0, weights must be set) with mr_steps
 * minimal-residual steps after it, or go back to the plain smoother. */
int qd_smoother_enable(qd_mg* mg, int enabled, int mr_steps);

/* out = S in, FP64, nrhs columns in fine qd layout.  Asynchronous. */
int qd_smoother_apply(qd_mg* mg, int nrhs, const double* in, double* out);
/* The same in FP32 with the FP16-rounded weights (the FP32 V-cycle's form):
 * in/out interleaved complex float.  Asynchronous. */
int qd_smoother_apply_f32(qd_mg* mg, int nrhs, const float* in, float* out);

/* ------------------------------------------------------------------------ */
/* Launch-shape autotuner (the paper has no counterpart)                     */
/* ------------------------------------------------------------------------ */

/* mode 1 (default): the first call of a tunable kernel for a new problem
 * shape times each valid launch shape on the caller's stream and keeps the
 * fastest for the rest of the process (coarse stencil: rows per thread and
 * block width; FP32 Wilson: one or two right-hand sides per thread).  All
 * coarse-stencil shapes give bit-identical results; the Wilson shapes agree
 * to FP32 rounding.  mode 0: fixed defaults, nothing timed.  Process-wide. */
void qd_autotune_set(int mode);
/* Clear the stored choices. */
void qd_autotune_clear(void);
/* Testing aid: candidate k >= 0 of every tunable kernel where k applies
 * (the default where it does not), nothing timed or stored; -1 (initial)
 * returns to the mode above.  Process-wide.  Lets a test compare every
 * launch shape of a kernel (coarse stencil on tensor cores: 0-3 input split
 * into operand tiles first, at most 8/4/3/2 operand slots; 4-6 input
 * converted in the kernel, 2/3/4 staging slots; 7-8 split tiles, at most 8/4
 * slots, one bulk copy per 4 KB tile region; 9-10 split tiles, two CTAs per
 * SM). */
void qd_autotune_force(int candidate);
/* The table as text, one line per shape key: the key, the chosen candidate,
 * then each candidate's best time in ms (-1: not applicable).  Writes at most
 * len bytes (NUL-terminated) to buf (nullable) and returns the full length
 * including the NUL. */
int qd_autotune_report(char* buf, int len);

/* ------------------------------------------------------------------------ */
/* Kernel timing (measurement support; the paper has no counterpart)         */
/* ------------------------------------------------------------------------ */

/* Number of kernels this library has launched since it was loaded (all
 * contexts and threads). */
long long qd_launch_count(void);

/* Number of device allocations (cudaMalloc) this library has made since it
 * was loaded (all contexts and threads). */
long long qd_alloc_count(void);

/* Kernel kinds: operator x precision. */
enum {
  QD_PROF_WILSON_F64 = 0,   /* a2 stencil, FP64 */
  QD_PROF_WILSON_F32 = 1,   /* a2 stencil, FP32 */
  QD_PROF_COARSE_F64 = 2,   /* a4 coarse stencil, FP64 */
  QD_PROF_COARSE_F32 = 3,   /* a4 coarse stencil, FP32 */
  QD_PROF_PROLONG_F64 = 4,  /* a3 W c, FP64 */
  QD_PROF_PROLONG_F32 = 5,
  QD_PROF_RESTRICT_F64 = 6, /* a3 W^H x, FP64 */
  QD_PROF_RESTRICT_F32 = 7,
  QD_PROF_DIRECT_F64 = 8,   /* coarsest dense solve C^{-1} R, FP64 */
  QD_PROF_DIRECT_F32 = 9,
  QD_PROF_DIRECT_BF16 = 10, /* coarsest dense solve on tcgen05 tensor cores */
  QD_PROF_BLAS_F64 = 11,    /* FP64 reductions and vector updates */
  QD_PROF_DOTS_F32 = 12,    /* FP32 per-column reductions (Gram-Schmidt, smoother) */
  QD_PROF_AXPY_F32 = 13,    /* FP32 multi-vector updates (Gram-Schmidt) */
  QD_PROF_UPDATE_F32 = 14,  /* FP32 fused GCR / minimal-residual updates */
  QD_PROF_SMOOTHER_F64 = 15,/* learned smoother S r, FP64 */
  QD_PROF_SMOOTHER_F32 = 16,/* learned smoother S r, FP32 (FP16 weights) */
  QD_PROF_COARSE_TC = 17,   /* a4 coarse stencil on tcgen05 (split-BF16 operands) */
  QD_PROF_RESTRICT_TC = 18, /* a3 W^H x on tcgen05 (split-BF16 operands) */
  QD_PROF_NKINDS = 19
};

/* enable != 0: record a CUDA event pair on the context stream around every
 * launch of the kinds above, with the launch's algorithmic flops and bytes;
 * enable == 0: stop recording.  Recording adds host work per launch. */
int qd_prof_enable(qd_ctx* ctx, int enable);

/* Totals for one kind since the last reset: launches, summed device time
 * (ms) of those launches, algorithmic flops and bytes.  Synchronises the
 * stream.  reset != 0 clears the totals of that kind afterwards. */
int qd_prof_read(qd_ctx* ctx, int kind, int64_t* launches, double* ms,
                 double* flops, double* bytes, int reset);

/* Statistics of per-sample values t_j (device array of s complex numbers),
 * as qd_hutchinson_trace computes them (Eq. 1; Sec. 4.1 jackknife): fills
 * t0, mean, estimate = t0 + mean, var, var_re, stderr_mean,
 * var_jackknife_err and nsamples of `result` (other fields untouched).
 * Used to merge the samples of several ranks or batches.  Synchronous. */
int qd_trace_stats(qd_ctx* ctx, int s, const double* t, const double t0[2],
                   qd_trace_result* result);

#ifdef __cplusplus
}
#endif

#endif /* QDTRACE_H */
