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
// Whether per-launch tracing is on (callers that would run launches
// concurrently on several streams serialise them while it is).
bool prof_tracing();
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

// Streaming multiprocessors of the current device (queried once per device).
inline int sm_count() {
  static int cache[64] = {0};
  int d = 0;
  cudaGetDevice(&d);
  if (d < 0 || d >= 64) d = 0;
  if (cache[d] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 1;
    }
    cache[d] = n;
  }
  return cache[d];
}

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
  // Copy of n host bytes, landed on the device when this returns.  A plain
  // cudaMemcpy from pageable memory may return once the bytes are staged, with
  // the DMA still queued on the legacy stream, which kernels on non-blocking
  // streams do not wait for; hence a stream-ordered copy that is waited for.
  int upload(const void* h, size_t n) {
    NRE_TRY(alloc(n));
    NRE_TRY_CUDA(cudaMemcpyAsync(p, h, n, cudaMemcpyHostToDevice, cudaStreamPerThread));
    NRE_TRY_CUDA(cudaStreamSynchronize(cudaStreamPerThread));
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
// Sum of a float over the 32 lanes of a warp (every lane gets it).
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Dot product of two 16-byte float vectors.
__device__ __forceinline__ float dot4(float4 a, float4 b) { return (a.x * b.x + a.y * b.y) + (a.z * b.z + a.w * b.w); }

// Sum of two unevaluated pairs hi + lo of floats (double-float numbers,
// about 48 significant bits) in FP32 arithmetic: Knuth's two-sum of the high
// parts, the low parts added to its error term, renormalised.
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float s = a.x + b.x;
  const float bv = s - a.x;
  const float e = ((a.x - (s - bv)) + (b.x - bv)) + (a.y + b.y);
  const float hi = s + e;
  return make_float2(hi, e - (hi - s));
}

// A thread's running sum of many terms: compensated (Kahan) FP32 for FP32
// terms, plain FP64 for FP64 terms.  The FP64 units of this part run at a
// small fraction of the FP32 rate, so per-element FP64 adds and conversions
// in FP32 loops cost more than the loads they follow; the compensation keeps
// the FP32 sum's error at a few units in the last place whatever the number
// of terms.  block_sum() totals the block's sums (all threads must call it;
// the result is valid in thread 0): in FP64 for FP64, in double-float FP32
// arithmetic for FP32, converted to a double once.
template <typename T>
struct RunSum {
  double s = 0.0;
  __device__ __forceinline__ void add(T x) { s += double(x); }
  __device__ __forceinline__ double value() const { return s; }
  __device__ double block_sum() const;
};
template <>
struct RunSum<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return double(s) - double(c); }
  __device__ double block_sum() const {
    __shared__ float2 red[32];
    float2 v = make_float2(s, -c);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      v = df_add(v, make_float2(__shfl_down_sync(0xffffffffu, v.x, o), __shfl_down_sync(0xffffffffu, v.y, o)));
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x != 0) return 0.0;
    v = red[0];
    for (int i = 1; i < nw; ++i) v = df_add(v, red[i]);
    return double(v.x) + double(v.y);
  }
};

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

template <typename T>
__device__ double RunSum<T>::block_sum() const {
  __shared__ double red[32];
  return ::nre::block_sum(s, red);
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

// Raises kernel k's dynamic shared-memory limit to `dyn` bytes where its
// static plus dynamic shared memory exceed the default 48 KB (a kernel with
// static barriers or reduction slots needs the raise below 48 KB of dynamic
// memory already).
template <typename K>
int raise_smem(K k, size_t dyn) {
  if (dyn <= 40 * 1024) return NRE_OK;
  cudaFuncAttributes fa{};
  NRE_TRY_CUDA(cudaFuncGetAttributes(&fa, k));
  if (dyn + fa.sharedSizeBytes > 48 * 1024)
    NRE_TRY_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  return NRE_OK;
}

}  // namespace nre
