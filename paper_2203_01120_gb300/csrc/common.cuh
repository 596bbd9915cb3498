// Shared device helpers for the tdlz library: complex arithmetic on
// double2/float2, error plumbing and small launch utilities.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

namespace tdlz {

template <class T> struct Cx;
template <> struct Cx<double> { using type = double2; };
template <> struct Cx<float> { using type = float2; };
template <class T> using cx = typename Cx<T>::type;

template <class T> __host__ __device__ __forceinline__ cx<T> mk(T re, T im) {
  cx<T> r;
  r.x = re;
  r.y = im;
  return r;
}
template <class T> __host__ __device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) {
  return mk<T>(a.x + b.x, a.y + b.y);
}
template <class T> __host__ __device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) {
  return mk<T>(a.x - b.x, a.y - b.y);
}
template <class T> __host__ __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <class T> __host__ __device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {
  return mk<T>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <class T> __host__ __device__ __forceinline__ cx<T> cscale(cx<T> a, T s) {
  return mk<T>(a.x * s, a.y * s);
}
// acc += a * b
template <class T> __host__ __device__ __forceinline__ void cfma(cx<T> &acc, cx<T> a, cx<T> b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
// acc += conj(a) * b
template <class T> __host__ __device__ __forceinline__ void cfmac(cx<T> &acc, cx<T> a, cx<T> b) {
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}
template <class T> __host__ __device__ __forceinline__ cx<T> czero() { return mk<T>(T(0), T(0)); }

struct Error {
  int status;
  std::string msg;
};

// Process-wide number of kernels the library has launched (defined in abi.cu).
extern std::atomic<long long> g_launches;

}  // namespace tdlz

#define TDLZ_CUDA_TRY(expr)                                                            \
  do {                                                                                 \
    cudaError_t _e = (expr);                                                           \
    if (_e != cudaSuccess)                                                             \
      throw ::tdlz::Error{3, std::string(#expr) + ": " + cudaGetErrorString(_e)};      \
  } while (0)

#define TDLZ_LAUNCH_CHECK()                                                            \
  do {                                                                                 \
    ::tdlz::g_launches.fetch_add(1, std::memory_order_relaxed);                        \
    cudaError_t _e = cudaGetLastError();                                               \
    if (_e != cudaSuccess)                                                             \
      throw ::tdlz::Error{3, std::string("kernel launch: ") + cudaGetErrorString(_e)}; \
  } while (0)

#define TDLZ_REQUIRE(cond, code, text)                                                 \
  do {                                                                                 \
    if (!(cond)) throw ::tdlz::Error{(code), std::string(text)};                       \
  } while (0)
