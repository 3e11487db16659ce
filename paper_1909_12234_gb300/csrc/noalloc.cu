// qd_deflate_project_static: out = (I - U U^H) z for an orthonormal
// eigenvector space, with its scratch in a fixed device array instead of
// memory the library would allocate per call.  For callers that cannot let
// the library allocate during a call (an application that gives all device
// memory to its own pool up front, or a loop that must not pay cudaMalloc /
// cudaFree).
#include "defl.cuh"
#include "dense.cuh"

namespace {

// Scratch shared by every call on a device: the U^H z coefficients and the
// per-chunk partial sums of that product.  Every element a call reads is
// written by the same call first, so nothing needs clearing between calls.
constexpr size_t kStaticScratchBytes = size_t(8) << 20;  // 8 MiB
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

}  // namespace

namespace qd {

size_t static_scratch_bytes() { return kStaticScratchBytes; }

// Device address of the scratch array on the current device.  In host code
// the symbol is only a stand-in; cudaGetSymbolAddress returns the device
// address and, under lazy module loading, loads the module that holds the
// array (which is when its 8 MiB are taken).  Called by qd_ctx_create with
// the context's device current, together with the load of the kernels the
// projection launches, so that a later call loads and allocates nothing.
void* static_scratch_resolve() {
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
  if (e != cudaSuccess || ptr == nullptr)
    fail(QD_ERR_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
  preload_projection_kernels();
  return ptr;
}

void defl_project_static(qd_defl& d, int s, const cplx* z, cplx* out) {
  QD_REQUIRE(d.kind == QD_DEFL_EIG_ORTHO,
             "qd_deflate_project_static supports QD_DEFL_EIG_ORTHO spaces only");
  qd_ctx& ctx = *d.ctx;
  QD_REQUIRE(ctx.static_scratch != nullptr, "context has no static scratch address");
  const int r = d.rank;
  const int64_t nf = d.gauge->geo.nsites * 12;
  const int64_t cap = (int64_t)(kStaticScratchBytes / sizeof(cplx));
  const int64_t coef = (int64_t)r * s;
  QD_REQUIRE(2 * coef <= cap, "rank x nrhs too large for the static scratch (8 MiB: rank * nrhs <= 262144)");
  cplx* base = static_cast<cplx*>(ctx.static_scratch);
  cplx* a = base;                // r x s coefficients U^H z
  cplx* partials = base + coef;  // per-chunk partial sums
  if (!blockdot_into(ctx, nf, d.U.as<cplx>(), r, r, z, s, s, a, partials, cap - coef))
    fail(QD_ERR_INVALID, "rank x nrhs too large for the static scratch");
  QD_CUDA(cudaMemcpyAsync(out, z, (size_t)nf * s * sizeof(cplx), cudaMemcpyDeviceToDevice, ctx.stream));
  blockmul(ctx, nf, d.U.as<cplx>(), r, r, a, s, s, out, s, -1.0, 1.0);
}

}  // namespace qd
