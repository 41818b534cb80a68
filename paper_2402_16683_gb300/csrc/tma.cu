// Host side of the bulk tensor copies: tensor maps through the driver's
// cuTensorMapEncodeTiled, looked up once through the runtime (no link-time
// dependence on the driver library).
#include <mutex>

#include "tma.cuh"

namespace nre {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

std::mutex g_tw_mu;
unsigned* g_tw[64] = {nullptr};

}  // namespace

unsigned* timeout_word() {
  int d = 0;
  cudaGetDevice(&d);
  if (d < 0 || d >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_tw_mu);
  if (!g_tw[d]) {
    void* p = nullptr;
    if (cudaMalloc(&p, 16) != cudaSuccess || cudaMemset(p, 0, 16) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
      cudaGetLastError();
      if (p) cudaFree(p);
      return nullptr;
    }
    g_tw[d] = static_cast<unsigned*>(p);
  }
  return g_tw[d];
}

int tmap_tiled(CUtensorMap* m, CUtensorMapDataType dt, int rank, const void* base, const uint64_t* dims,
               const uint64_t* strides_b, const uint32_t* box, int swizzle_bytes) {
  const PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return set_error(NRE_ECUDA, "cuTensorMapEncodeTiled is not available");
  if (rank < 1 || rank > 5) return set_error(NRE_EINVAL, "internal: tensor map rank %d", rank);
  if (reinterpret_cast<uintptr_t>(base) % 16 != 0)
    return set_error(NRE_EINVAL, "internal: tensor map base not 16-byte aligned");
  const int es = (dt == CU_TENSOR_MAP_DATA_TYPE_FLOAT64) ? 8 : 4;
  if ((box[0] * es) % 16 != 0) return set_error(NRE_EINVAL, "internal: tensor map box row not a 16-byte multiple");
  cuuint64_t gd[5], gs[4];
  cuuint32_t bx[5], el[5];
  for (int d = 0; d < rank; ++d) {
    if (box[d] < 1 || box[d] > 256) return set_error(NRE_EINVAL, "internal: tensor map box extent %u", box[d]);
    gd[d] = dims[d];
    bx[d] = box[d];
    el[d] = 1;
  }
  for (int d = 0; d + 1 < rank; ++d) {
    if (strides_b[d] % 16 != 0) return set_error(NRE_EINVAL, "internal: tensor map stride not a 16-byte multiple");
    gs[d] = strides_b[d];
  }
  CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_NONE;
  if (swizzle_bytes == 32) sw = CU_TENSOR_MAP_SWIZZLE_32B;
  else if (swizzle_bytes == 64) sw = CU_TENSOR_MAP_SWIZZLE_64B;
  else if (swizzle_bytes == 128) sw = CU_TENSOR_MAP_SWIZZLE_128B;
  else if (swizzle_bytes != 0) return set_error(NRE_EINVAL, "internal: swizzle of %d bytes", swizzle_bytes);
  if (swizzle_bytes && box[0] * es != (uint32_t)swizzle_bytes)
    return set_error(NRE_EINVAL, "internal: swizzled box rows must span the swizzle");
  const CUresult r = fn(m, dt, (cuuint32_t)rank, const_cast<void*>(base), gd, gs, bx, el,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(NRE_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return NRE_OK;
}

}  // namespace nre

extern "C" int nre_wait_timeouts(unsigned* count, int reset) {
  nre::clear_error();
  if (!count) return nre::set_error(NRE_EINVAL, "NULL argument");
  unsigned* w = nre::timeout_word();
  if (!w) return nre::set_error(NRE_ECUDA, "no timeout word on this device");
  NRE_TRY_CUDA(cudaDeviceSynchronize());
  NRE_TRY_CUDA(cudaMemcpy(count, w, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (reset) {
    NRE_TRY_CUDA(cudaMemset(w, 0, sizeof(unsigned)));
    NRE_TRY_CUDA(cudaDeviceSynchronize());
  }
  return NRE_OK;
}

namespace {

// A wait that nothing completes: the barrier expects 16 bytes that no copy
// delivers, so every thread's bounded wait runs out and thread 0 counts it.
__global__ void k_wait_selftest(unsigned limit, unsigned* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    nre::mbar_init(&bar, 1);
    nre::mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) nre::mbar_arrive_tx(&bar, 16u);
  const bool ok = nre::mbar_wait(&bar, 0u, limit);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) nre::note_timeout(status);
}

}  // namespace

extern "C" int nre_wait_selftest(unsigned limit, nre_stream_t stream) {
  nre::clear_error();
  if (limit < 1 || limit > (1u << 20)) return nre::set_error(NRE_EINVAL, "limit must be in [1, 2^20]");
  unsigned* w = nre::timeout_word();
  if (!w) return nre::set_error(NRE_ECUDA, "no timeout word on this device");
  k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(limit, w);
  NRE_CHECK_LAUNCH();
  return NRE_OK;
}
