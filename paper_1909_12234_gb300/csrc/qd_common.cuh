// Internal definitions shared by the libqdtrace translation units:
// complex arithmetic on double2, error handling, device buffers, Philox.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdio>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/qdtrace.h"

namespace qd {

// ---------------------------------------------------------------------------
// Errors: internal code throws qd::Error; the C ABI turns it into a status.
// ---------------------------------------------------------------------------
struct Error : public std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

[[noreturn]] inline void fail(int code, const std::string& msg) { throw Error(code, msg); }

inline void cuda_check(cudaError_t e, const char* what, const char* file, int line) {
  if (e != cudaSuccess) {
    int code = (e == cudaErrorMemoryAllocation) ? QD_ERR_OOM : QD_ERR_CUDA;
    fail(code, std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" +
                   std::to_string(line) + ")");
  }
}
// Kernels launched by this library since load (qd_launch_count()).
std::atomic<long long>& launch_counter();
// Device allocations (cudaMalloc) this library has made since load
// (qd_alloc_count()).
std::atomic<long long>& alloc_counter();
// Raise a kernel's dynamic shared-memory limit on the current device to at
// least `bytes`.  The limit only ever grows (a launch that fits an earlier,
// smaller request still fits), so threads launching the same kernel with
// different sizes cannot undercut each other.  Thread safe.
void ensure_smem_limit(const void* kernel, size_t bytes);

#define QD_CUDA(call) ::qd::cuda_check((call), #call, __FILE__, __LINE__)
#define QD_LAUNCH_CHECK()                                                      \
  do {                                                                         \
    ::qd::launch_counter().fetch_add(1, std::memory_order_relaxed);           \
    ::qd::cuda_check(cudaGetLastError(), "kernel launch", __FILE__, __LINE__); \
  } while (0)
#define QD_REQUIRE(cond, msg)                                  \
  do {                                                         \
    if (!(cond)) ::qd::fail(QD_ERR_INVALID, std::string(msg)); \
  } while (0)

// ---------------------------------------------------------------------------
// Device buffer (owning, grow-only).
// ---------------------------------------------------------------------------
class DevBuf {
 public:
  DevBuf() = default;
  explicit DevBuf(size_t bytes) { resize(bytes); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p_(o.p_), n_(o.n_) { o.p_ = nullptr; o.n_ = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p_ = o.p_; n_ = o.n_; o.p_ = nullptr; o.n_ = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void resize(size_t bytes) {
    if (bytes <= n_) return;
    release();
    if (bytes == 0) return;
    QD_CUDA(cudaMalloc(&p_, bytes));
    alloc_counter().fetch_add(1, std::memory_order_relaxed);
    n_ = bytes;
  }
  void release() {
    if (p_) cudaFree(p_);
    p_ = nullptr;
    n_ = 0;
  }
  template <class T> T* as() const { return reinterpret_cast<T*>(p_); }
  size_t bytes() const { return n_; }

 private:
  void* p_ = nullptr;
  size_t n_ = 0;
};

// ---------------------------------------------------------------------------
// Complex numbers on double2 (FP64 path) and float2 (FP32 inner path).
// ---------------------------------------------------------------------------
typedef double2 cplx;   // FP64 complex, the library's external type
typedef float2 cplxf;   // FP32 complex, inner solver storage

template <class C> struct CTraits;
template <> struct CTraits<double2> { typedef double R; };
template <> struct CTraits<float2> { typedef float R; };

template <class C>
__host__ __device__ __forceinline__ C mk(typename CTraits<C>::R r, typename CTraits<C>::R i) {
  C c;
  c.x = r;
  c.y = i;
  return c;
}
__host__ __device__ __forceinline__ cplx mkc(double r, double i) { return make_double2(r, i); }
template <class C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <class C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <class C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <class C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
  return mk<C>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <class C> __host__ __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
template <class C> __host__ __device__ __forceinline__ C cscale(typename CTraits<C>::R s, C a) {
  return mk<C>(s * a.x, s * a.y);
}
// i * a
template <class C> __host__ __device__ __forceinline__ C ctimesi(C a) { return mk<C>(-a.y, a.x); }
// acc += a * b
template <class C> __host__ __device__ __forceinline__ void cfma(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
// acc += conj(a) * b
template <class C> __host__ __device__ __forceinline__ void cfmac(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}
template <class C> __host__ __device__ __forceinline__ typename CTraits<C>::R cnorm2(C a) {
  return a.x * a.x + a.y * a.y;
}
template <class Cout, class Cin> __host__ __device__ __forceinline__ Cout ccast(Cin a) {
  return mk<Cout>((typename CTraits<Cout>::R)a.x, (typename CTraits<Cout>::R)a.y);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 4x32 counter, 2x32 key,
// ten rounds of two 32x32->64 products, Weyl-sequence key schedule.
// ---------------------------------------------------------------------------
struct U4 { uint32_t v[4]; };

__host__ __device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
  const uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint64_t pa = (uint64_t)kMulA * c.v[0];
    const uint64_t pb = (uint64_t)kMulB * c.v[2];
    U4 n;
    n.v[0] = (uint32_t)(pb >> 32) ^ c.v[1] ^ k0;
    n.v[1] = (uint32_t)pb;
    n.v[2] = (uint32_t)(pa >> 32) ^ c.v[3] ^ k1;
    n.v[3] = (uint32_t)pa;
    c = n;
    k0 += kWeylA;
    k1 += kWeylB;
  }
  return c;
}

// ---------------------------------------------------------------------------
// Launch helpers.
// ---------------------------------------------------------------------------
inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
constexpr int kNumSMs = 152;  // GB300: 2 dies x 76 SMs (grid sizing only)

}  // namespace qd
