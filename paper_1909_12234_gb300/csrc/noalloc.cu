// qd_deflate_project_static: the Algorithm 1 projection (I - U U^H) z with
// its scratch in a fixed device array instead of memory the library would
// allocate per call.  See include/qdtrace.h for who needs this and its
// limits.
#include <map>
#include <mutex>

#include "defl.cuh"
#include "dense.cuh"

namespace {

// Scratch shared by every call on a device: the U^H z coefficients and the
// per-chunk partial sums of that product.  Every element a call reads is
// written by the same call first, so nothing needs clearing between calls.
constexpr size_t kStaticScratchBytes = size_t(8) << 20;  // 8 MiB
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_addr_mu;
std::map<int, void*> g_addr;  // device -> device address of g_static_scratch

// Device address of the scratch array on the current device (resolved on the
// first call per device; in host code the symbol itself is only a stand-in).
void* scratch_address(int device) {
  std::lock_guard<std::mutex> lock(g_addr_mu);
  auto it = g_addr.find(device);
  if (it != g_addr.end()) return it->second;
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
  if (e != cudaSuccess || ptr == nullptr)
    qd::fail(QD_ERR_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
  g_addr[device] = ptr;
  return ptr;
}

}  // namespace

namespace qd {

size_t static_scratch_bytes() { return kStaticScratchBytes; }

void defl_project_static(qd_defl& d, int s, const cplx* z, cplx* out) {
  QD_REQUIRE(d.kind == QD_DEFL_EIG_ORTHO,
             "qd_deflate_project_static supports Algorithm 1 (QD_DEFL_EIG_ORTHO) only");
  qd_ctx& ctx = *d.ctx;
  const int r = d.rank;
  const int64_t nf = d.gauge->geo.nsites * 12;
  const int64_t cap = (int64_t)(kStaticScratchBytes / sizeof(cplx));
  const int64_t coef = (int64_t)r * s;
  QD_REQUIRE(2 * coef <= cap, "rank x nrhs too large for the static scratch (8 MiB: rank * nrhs <= 262144)");
  cplx* base = static_cast<cplx*>(scratch_address(ctx.device));
  cplx* a = base;               // r x s coefficients U^H z
  cplx* partials = base + coef;  // per-chunk partial sums
  if (!blockdot_into(ctx, nf, d.U.as<cplx>(), r, r, z, s, s, a, partials, cap - coef))
    fail(QD_ERR_INVALID, "rank x nrhs too large for the static scratch");
  QD_CUDA(cudaMemcpyAsync(out, z, (size_t)nf * s * sizeof(cplx), cudaMemcpyDeviceToDevice, ctx.stream));
  blockmul(ctx, nf, d.U.as<cplx>(), r, r, a, s, s, out, s, -1.0, 1.0);
}

}  // namespace qd
