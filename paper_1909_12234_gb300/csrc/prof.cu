// Kernel timing support (qd_prof_enable / qd_prof_read): an event pair per
// instrumented launch, folded into per-kind totals in batches.
#include <map>
#include <mutex>
#include <utility>
#include "qd_internal.cuh"

namespace qd {

void ensure_smem_limit(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> limit;
  int dev = 0;
  QD_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = limit[{kernel, dev}];
  if (bytes <= cur) return;
  QD_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  cur = bytes;
}

std::atomic<long long>& launch_counter() {
  static std::atomic<long long> n{0};
  return n;
}

std::atomic<long long>& alloc_counter() {
  static std::atomic<long long> n{0};
  return n;
}

static cudaEvent_t take_event(qd_ctx& c) {
  if (c.prof_pool.empty()) {
    cudaEvent_t e;
    QD_CUDA(cudaEventCreate(&e));
    return e;
  }
  cudaEvent_t e = c.prof_pool.back();
  c.prof_pool.pop_back();
  return e;
}

void prof_flush(qd_ctx& c) {
  for (auto& p : c.prof_pending) {
    QD_CUDA(cudaEventSynchronize(p.e1));
    float ms = 0.f;
    QD_CUDA(cudaEventElapsedTime(&ms, p.e0, p.e1));
    c.prof_tot[p.kind].ms += ms;
    c.prof_pool.push_back(p.e0);
    c.prof_pool.push_back(p.e1);
  }
  c.prof_pending.clear();
}

ProfScope::ProfScope(qd_ctx& c, int kind, double flops, double bytes) : c_(c), kind_(kind) {
  if (!c.prof) return;
  if (c.prof_pending.size() >= 2048) prof_flush(c);
  cudaEvent_t e0 = take_event(c);
  e1_ = take_event(c);
  QD_CUDA(cudaEventRecord(e0, c.stream));
  c.prof_pending.push_back({kind, e0, e1_});
  c.prof_tot[kind].launches += 1;
  c.prof_tot[kind].flops += flops;
  c.prof_tot[kind].bytes += bytes;
}

ProfScope::~ProfScope() {
  if (e1_) cudaEventRecord(e1_, c_.stream);
}

}  // namespace qd

