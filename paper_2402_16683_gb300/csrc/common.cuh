// Internal helpers shared by the library's translation units: status and error
// reporting, device allocation, complex arithmetic and block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <string>

#include "../../include/nre.h"

namespace nre {

// ---------------------------------------------------------------- errors
int set_error(int code, const char* fmt, ...);
void clear_error();

// Launch tracing (prof.cu): bracket every kernel launch; `bytes` is the
// launch's algorithmic traffic (unique bytes of its global inputs + outputs).
void prof_begin(const char* name, double bytes, cudaStream_t st);
void prof_end(cudaStream_t st);

#define NRE_TRY_CUDA(call)                                                     \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess)                                                     \
      return ::nre::set_error(NRE_ECUDA, "%s failed: %s (%s:%d)", #call,      \
                              cudaGetErrorString(e_), __FILE__, __LINE__);     \
  } while (0)

#define NRE_TRY(call)                                                          \
  do {                                                                         \
    int s_ = (call);                                                           \
    if (s_ != NRE_OK) return s_;                                               \
  } while (0)

#define NRE_CHECK_LAUNCH()                                                     \
  do {                                                                         \
    cudaError_t e_ = cudaGetLastError();                                       \
    if (e_ != cudaSuccess)                                                     \
      return ::nre::set_error(NRE_ECUDA, "kernel launch failed: %s (%s:%d)",   \
                              cudaGetErrorString(e_), __FILE__, __LINE__);     \
  } while (0)

// Device bytes held by DevBufs of this process (prof.cu).
std::atomic<long long>& dev_bytes();
// Kernels launched outside prof_begin (graph replays): adds to the launch count.
void prof_add_launches(unsigned long long n);

// Owning device allocation (freed in the destructor).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) {
      cudaFree(p);
      dev_bytes().fetch_sub((long long)bytes);
    }
    p = nullptr;
    bytes = 0;
  }
  int alloc(size_t n) {
    release();
    if (n == 0) n = 16;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      return set_error(NRE_ENOMEM, "cudaMalloc(%zu) failed: %s", n, cudaGetErrorString(e));
    }
    bytes = n;
    dev_bytes().fetch_add((long long)n);
    return NRE_OK;
  }
  int upload(const void* h, size_t n) {
    NRE_TRY(alloc(n));
    NRE_TRY_CUDA(cudaMemcpy(p, h, n, cudaMemcpyHostToDevice));
    return NRE_OK;
  }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

inline int dtype_size(int dtype) { return dtype == NRE_F64 ? 8 : 4; }

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// ---------------------------------------------------------------- complex
template <typename T> struct CplxT;
template <> struct CplxT<float> { typedef float2 type; };
template <> struct CplxT<double> { typedef double2 type; };

template <typename C> __device__ __forceinline__ C cmake(decltype(C::x) a, decltype(C::x) b) {
  C r; r.x = a; r.y = b; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// multiply by -i
template <typename C> __device__ __forceinline__ C cmul_mi(C a) { return cmake<C>(a.y, -a.x); }

// ---------------------------------------------------------------- reductions
// Sum over the block of one double per thread; deterministic order.  `red`
// must hold blockDim.x/32 doubles.  The result is returned to every thread.
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += red[i];
  __syncthreads();
  return t;
}

// sum_{c < n} p[c * stride] by one thread, fixed order, eight loads in flight
// (the partial-sum loops are otherwise a serial chain of L2 round trips).
__device__ __forceinline__ double sum_strided(const double* p, int n, int64_t stride) {
  double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int c = 0;
  for (; c + 8 <= n; c += 8) {
    double v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = p[(int64_t)(c + k) * stride];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] += v[k];
  }
  for (int k = 0; c < n; ++c, ++k) acc[k] += p[(int64_t)c * stride];
  return ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
}

// Sum of n doubles p[0..n) by the first warp of the block in a fixed order
// (lane-strided runs, then a shuffle tree); every thread gets the result.
// Must be called by all threads of the block.
__device__ __forceinline__ double block_sum_array(const double* p, int n) {
  __shared__ double res;
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) s += p[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) res = s;
  }
  __syncthreads();
  const double r = res;
  __syncthreads();
  return r;
}

}  // namespace nre
