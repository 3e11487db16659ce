// Internal object model of libqdtrace: context, lattice levels, operators,
// multigrid hierarchy, deflation space.  Not part of the C ABI.
#pragma once

#include <memory>

#include "qd_common.cuh"

// ---------------------------------------------------------------------------
// Context: device, stream and small reusable scratch.
// ---------------------------------------------------------------------------
namespace qd {
// Per-kind kernel timing (qd_prof_*): event pairs folded into totals.
struct ProfTotals {
  int64_t launches = 0;
  double ms = 0.0, flops = 0.0, bytes = 0.0;
};
struct ProfPending {
  int kind;
  cudaEvent_t e0, e1;
};
}  // namespace qd

struct qd_ctx {
  bool prof = false;
  qd::ProfTotals prof_tot[QD_PROF_NKINDS];
  std::vector<qd::ProfPending> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  int device = 0;
  cudaStream_t stream = nullptr;
  qd::DevBuf red_partials;  // reduction partial sums (double2)
  qd::DevBuf small;         // small device scratch (per-RHS scalars)
  int* host_pinned = nullptr;  // 64 pinned ints for flag read-back
  void* static_scratch = nullptr;  // device address of the fixed scratch array (noalloc.cu)
  std::shared_ptr<void> cache;  // solver work spaces reused across calls
};

namespace qd {

// Fold recorded event pairs into the totals (synchronises their events).
void prof_flush(qd_ctx& c);

// RAII: records an event pair around the launches in its scope when the
// context's profiling is on; flops / bytes are the algorithmic work.
class ProfScope {
 public:
  ProfScope(qd_ctx& c, int kind, double flops, double bytes);
  ~ProfScope();

 private:
  qd_ctx& c_;
  int kind_;
  cudaEvent_t e1_ = nullptr;
};

// Per-RHS scalar work area reserved from qd_ctx::small (double2 units).
inline cplx* ctx_small(qd_ctx& c, size_t n_complex) {
  c.small.resize(n_complex * sizeof(cplx));
  return c.small.as<cplx>();
}

// ---------------------------------------------------------------------------
// Lattice level geometry.
//   fine level : sites in even-odd order (eo = parity * V/2 + lex/2)
//   coarse     : sites in lexicographic order of the coarse lattice
//   nbr[s][h]  : h = 0..3 -> site + mu, h = 4..7 -> site - mu
// ---------------------------------------------------------------------------
struct LevelGeom {
  int dims[4] = {0, 0, 0, 0};
  int64_t nsites = 0;
  bool eo = false;
  std::vector<int> h_nbr;          // [nsites][8]
  std::vector<int> h_lex_of_site;  // [nsites]
  std::vector<int> h_site_of_lex;  // [nsites]
  DevBuf nbr;                      // int32 [nsites][8]
  DevBuf lex_of_site;              // int32 [nsites]
  DevBuf site_of_lex;              // int32 [nsites]
  // Stencil traversal order: visit[k] = site index of the k-th site when
  // 4^4 tiles are taken in turn (Morton order inside a tile), so that the
  // sites in flight at one time form compact 4-D regions whose neighbours
  // stay in L2.
  std::vector<int> h_visit;
  DevBuf visit;                    // int32 [nsites]
  // The same order restricted to the sites of one parity (even-odd
  // lattices): visit_par[p] holds nsites/2 site indices, all in
  // [p nsites/2, (p+1) nsites/2).
  DevBuf visit_par[2];
  // int, 0 until a bounded wait of the bulk-staged FP32 stencil gives up
  mutable DevBuf bulk_err;
  void build(const int d[4], bool even_odd);
  void coords(int64_t lex, int c[4]) const {
    c[0] = (int)(lex % dims[0]);
    c[1] = (int)((lex / dims[0]) % dims[1]);
    c[2] = (int)((lex / ((int64_t)dims[0] * dims[1])) % dims[2]);
    c[3] = (int)(lex / ((int64_t)dims[0] * dims[1] * dims[2]));
  }
  int64_t lex(const int c[4]) const {
    return c[0] + (int64_t)dims[0] * (c[1] + (int64_t)dims[1] * (c[2] + (int64_t)dims[2] * c[3]));
  }
};

// ---------------------------------------------------------------------------
// Linear operators on fields with `dof` complex numbers per site, nrhs
// columns, RHS innermost: element (site, d, r) at (site*dof + d)*nrhs + r.
// The first dof/2 components of a site have chirality +1, the rest -1.
// ---------------------------------------------------------------------------
template <class C> struct Op {
  virtual ~Op() {}
  virtual int64_t nsites() const = 0;
  virtual int dof() const = 0;
  int64_t n() const { return nsites() * (int64_t)dof(); }
  virtual void apply(qd_ctx& ctx, const C* in, C* out, int nrhs) const = 0;
  // r = b - A x; r must not alias x.  Default: apply into r, then subtract.
  virtual void residual(qd_ctx& ctx, const C* b, const C* x, C* r, int nrhs) const;
  // True when o is the same operator (same data, parameters and form).
  virtual bool same(const Op<C>& o) const { return false; }
};

template <class C> struct Precond {
  virtual ~Precond() {}
  virtual void apply(qd_ctx& ctx, const C* r, C* z, int nrhs) = 0;
  // z = M r and, when M ends on a residual of A (minimal-residual smoothing
  // keeps res = r - A z), also Az = A z = r - res without a product with A;
  // returns false with Az untouched when it cannot.
  virtual bool apply_az(qd_ctx& ctx, const Op<C>& A, const C* r, C* z, C* Az, int nrhs) {
    (void)A;
    (void)Az;
    apply(ctx, r, z, nrhs);
    return false;
  }
};

}  // namespace qd

// ---------------------------------------------------------------------------
// Gauge field: links in even-odd site order, [4][V][3][3] complex.
// ---------------------------------------------------------------------------
struct qd_gauge {
  qd_ctx* ctx = nullptr;
  qd::LevelGeom geo;
  qd::DevBuf links;   // cplx  [4][V][9]
  qd::DevBuf linksf;  // cplxf [4][V][9] (made on first FP32 use)
  const qd::cplxf* links_f32();
};

namespace qd {

// Wilson-Dirac operator A(m0, tau) (or A^H) in precision C.
template <class C> struct WilsonOp : public Op<C> {
  const qd_gauge* g;
  const C* links;
  double m0, tau;
  bool dagger;
  WilsonOp(const qd_gauge* gauge, const C* lk, double m, double t, bool dag)
      : g(gauge), links(lk), m0(m), tau(t), dagger(dag) {}
  int64_t nsites() const override { return g->geo.nsites; }
  int dof() const override { return 12; }
  void apply(qd_ctx& ctx, const C* in, C* out, int nrhs) const override;
  void residual(qd_ctx& ctx, const C* b, const C* x, C* r, int nrhs) const override;
  bool same(const Op<C>& o) const override {
    const WilsonOp<C>* w = dynamic_cast<const WilsonOp<C>*>(&o);
    return w && w->g == g && w->links == links && w->m0 == m0 && w->tau == tau && w->dagger == dagger;
  }
};

// Launchers (wilson.cu).  b != nullptr: out = b - A in (fused residual).
template <class C>
void wilson_apply(qd_ctx& ctx, const LevelGeom& geo, const C* links, double m0, double tau,
                  bool dagger, const C* in, C* out, int nrhs, const C* b = nullptr);
// Parity-restricted hopping (wilson.cu): for the sites n of parity p,
// out(n) = Q1 z(n) + Q2 (H in)(n) with A = M - H/2, Q1 and Q2 spin-diagonal
// (q[0] upper spins, q[1] lower); in a half field of parity 1 - p, z
// (nullable) and out half fields of parity p.
template <class C>
void wilson_eo(qd_ctx& ctx, const LevelGeom& geo, const C* links, int p, const cplx q1[2], const cplx q2[2],
               const C* in, const C* z, C* out, int nrhs);
// Nonzero when a bounded wait of the bulk-staged FP32 stencil gave up on
// this geometry (synchronises the stream).
int wilson_bulk_error(qd_ctx& ctx, const LevelGeom& geo);
// out = Q in on a half field of nh sites.
template <class C>
void spin_diag(qd_ctx& ctx, int64_t nh, int nrhs, const cplx q[2], const C* in, C* out);
void gauge_import(qd_ctx& ctx, qd_gauge& g, const double* links_host);
void links_to_f32(qd_ctx& ctx, const cplx* in, cplxf* out, int64_t n);

// Rademacher noise and setup starts (core.cu).
void rademacher_fill(qd_ctx& ctx, const LevelGeom& geo, uint64_t seed, int64_t sample_offset,
                     int nrhs, cplx* out);
void random_starts_fill(qd_ctx& ctx, const LevelGeom& geo, int dof, uint64_t key, int nvec,
                        cplx* out);
void field_reorder(qd_ctx& ctx, const LevelGeom& geo, int nrhs, bool to_qd, const cplx* in,
                   cplx* out);

// ---------------------------------------------------------------------------
// Multigrid: coarse levels and transfers.
// ---------------------------------------------------------------------------
struct Transfer {
  int nv = 0;         // null vectors per chirality
  int Df = 0;         // dofs per fine site (12 or 2 nv of the level above)
  int Dc = 0;         // dofs per coarse site = 2 nv
  int block[4] = {1, 1, 1, 1};
  int bsites = 0;     // fine sites per aggregate
  int64_t nfine = 0;  // fine sites
  int64_t ncoarse = 0;
  DevBuf agg_of;      // int32 [nfine]: coarse site of each fine site
  DevBuf members;     // int32 [ncoarse][bsites]: fine sites of an aggregate
  DevBuf hopdir;      // int8  [nfine][8]: coarse stencil direction of each hop
  DevBuf W;           // cplx  [nfine][Df][nv]
  DevBuf Wf;          // cplxf copy
  bool use_tc = false;     // FP32 V-cycle restricts on tensor cores
  mutable DevBuf Wtc;      // uint32 [nfine][2][Df][nv]: split-BF16 (hi, lo) W
  mutable DevBuf rtc_err;  // int: bounded-wait error of the tensor-core restriction
  std::vector<int> null_steps;
};

struct CoarseLevel {
  LevelGeom geo;      // lexicographic coarse lattice
  int D = 0;          // dofs per site
  DevBuf Cm;          // cplx  [nsites][9][D][D]; dir 0 self, 1+mu: +mu, 5+mu: -mu
  DevBuf Cmf;         // cplxf copy
  bool use_tc = false;      // FP32 V-cycle applies the stencil on tensor cores
  mutable DevBuf Cmb;       // uint32 [nsites][9][D][D]: (re, im) BF16 pairs
  mutable DevBuf ctc_err;   // int: bounded-wait error of the tensor-core stencil
  mutable DevBuf sten_src;  // int32 [nsites][9]: the site, then its 8 neighbours
  mutable DevBuf ctc_tiles; // split-BF16 operand tiles of the stencil's input (grow-only)
  int ndense = 0;     // > 0: Cinv holds the dense inverse (coarsest level)
  DevBuf Cinv;        // cplx  [n][n], n = nsites * D
  DevBuf Cinvf;       // cplxf copy
  // tensor-core form of Cinv (tc_gemm.cu): BF16 [Mp][Kp], TMA maps, buffers
  bool tc = false;
  int tc_Mp = 0, tc_Kp = 0, tc_mapB_N = 0;
  alignas(64) unsigned char tc_mapA[128];
  alignas(64) unsigned char tc_mapB[128];
  DevBuf tc_A, tc_B, tc_part, tc_err, tc_xc, tc_yc;
  // scratch of the FP64-corrected coarsest solve (grow-only)
  mutable DevBuf rs_f[2], rs_d[2];
};

template <class C> struct CoarseOp : public Op<C> {
  const CoarseLevel* lv;
  const C* mat;
  CoarseOp(const CoarseLevel* l, const C* m) : lv(l), mat(m) {}
  int64_t nsites() const override { return lv->geo.nsites; }
  int dof() const override { return lv->D; }
  void apply(qd_ctx& ctx, const C* in, C* out, int nrhs) const override;
  void residual(qd_ctx& ctx, const C* b, const C* x, C* r, int nrhs) const override;
  bool same(const Op<C>& o) const override {
    const CoarseOp<C>* c = dynamic_cast<const CoarseOp<C>*>(&o);
    return c && c->lv == lv && c->mat == mat;
  }
};

// Launchers (coarse.cu).
template <class C>
void coarse_apply(qd_ctx& ctx, const CoarseLevel& lv, const C* mat, const C* in, C* out, int nrhs);
template <class C>
void prolongate(qd_ctx& ctx, const Transfer& T, const C* W, const C* coarse, C* fine, int nrhs);
template <class C>
void restrict_(qd_ctx& ctx, const Transfer& T, const C* W, const C* fine, C* coarse, int nrhs);
void build_transfer_tables(Transfer& T, const LevelGeom& fine, const int block[4],
                           LevelGeom& coarse_geo);
void block_orthonormalize(qd_ctx& ctx, Transfer& T, const cplx* Y);
void coarse_build_from_wilson(qd_ctx& ctx, const Transfer& T, const qd_gauge& g, double m0,
                              double tau, CoarseLevel& out);
void coarse_build_from_coarse(qd_ctx& ctx, const Transfer& T, const CoarseLevel& fine,
                              CoarseLevel& out);
void to_f32(qd_ctx& ctx, const cplx* in, cplxf* out, int64_t n);
void to_f64(qd_ctx& ctx, const cplxf* in, cplx* out, int64_t n);

}  // namespace qd
