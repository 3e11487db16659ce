// Launch-shape autotuner (see tune.cuh).
#include <atomic>
#include <map>
#include <mutex>
#include <sstream>
#include <vector>

#include "tune.cuh"

namespace qd {

namespace {

struct Entry {
  int choice = 0;
  std::vector<float> ms;
};

std::mutex g_mu;
std::map<std::string, Entry>& table() {
  static std::map<std::string, Entry> t;
  return t;
}
std::atomic<int> g_mode{1};
std::atomic<int> g_force{-1};

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  QD_CUDA(cudaStreamIsCapturing(s, &st));
  return st != cudaStreamCaptureStatusNone;
}

}  // namespace

void tune_set_mode(int mode) { g_mode.store(mode ? 1 : 0); }
void tune_force(int candidate) { g_force.store(candidate >= 0 ? candidate : -1); }
int tune_mode() { return g_mode.load(); }

int tune_lookup(const std::string& key) {
  const int forced = g_force.load();
  if (forced >= 0) return forced;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = table().find(key);
  return it != table().end() ? it->second.choice : -1;
}

bool tune_can_time(qd_ctx& ctx) { return g_force.load() < 0 && g_mode.load() != 0 && !capturing(ctx.stream); }

void tune_clear() {
  std::lock_guard<std::mutex> lk(g_mu);
  table().clear();
}

std::string tune_report() {
  std::lock_guard<std::mutex> lk(g_mu);
  std::ostringstream os;
  for (const auto& kv : table()) {
    os << kv.first << " " << kv.second.choice;
    for (float m : kv.second.ms) os << " " << m;
    os << "\n";
  }
  return os.str();
}

int tune_pick(qd_ctx& ctx, const std::string& key, int ncand, const std::function<bool(int)>& launch) {
  const int forced = g_force.load();
  if (forced >= 0) return forced < ncand ? forced : -1;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = table().find(key);
    if (it != table().end()) return it->second.choice;
  }
  if (g_mode.load() == 0 || capturing(ctx.stream)) return -1;  // caller uses its default
  constexpr int reps = 3;
  Entry e;
  e.ms.assign(ncand, -1.0f);
  cudaEvent_t a, b;
  QD_CUDA(cudaEventCreate(&a));
  QD_CUDA(cudaEventCreate(&b));
  float best = 0.0f;
  int choice = -1;
  for (int c = 0; c < ncand; ++c) {
    if (!launch(c)) continue;  // not applicable, nothing enqueued
    float m = -1.0f;
    for (int r = 0; r < reps; ++r) {
      QD_CUDA(cudaEventRecord(a, ctx.stream));
      launch(c);
      QD_CUDA(cudaEventRecord(b, ctx.stream));
      QD_CUDA(cudaEventSynchronize(b));
      float t = 0.0f;
      QD_CUDA(cudaEventElapsedTime(&t, a, b));
      if (m < 0.0f || t < m) m = t;
    }
    e.ms[c] = m;
    if (choice < 0 || m < best) {
      best = m;
      choice = c;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (choice < 0) return -1;
  e.choice = choice;
  std::lock_guard<std::mutex> lk(g_mu);
  auto ins = table().emplace(key, e);
  return ins.first->second.choice;
}

}  // namespace qd
