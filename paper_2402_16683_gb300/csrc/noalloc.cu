// cf_forward_noalloc: the correlated-field forward transform with all of its
// intermediates in one fixed device array instead of plan workspaces.
//
// cf_forward grows the plan's workspaces (sweep intermediates and the
// amplitude model state) with cudaMalloc the first time a batch needs more.
// Some callers cannot allow that: cudaMalloc / cudaFree may synchronise the
// device and take unpredictable time inside a latency-bounded loop, and some
// host runtimes own the whole device-memory budget and hand it out only
// through their own pool.  This entry point runs the same kernels with the
// scratch carved from a file-scope device array (kNoAllocBytes) that exists
// once per device for the life of the process.
//
// The device address of the array is looked up with cudaGetSymbolAddress the
// first time the entry point runs on a device (with that device current) and
// cached per device ordinal: the cache assumes the device's primary context
// (the runtime API's default) and is not refreshed after cudaDeviceReset.  Every call shares the array and leaves its last contents
// in it; each call rewrites everything it reads, so nothing has to start at
// zero.  Calls whose work overlaps on the GPU (different streams, or different
// host threads without ordering) race on the array.
#include <mutex>
#include <vector>

#include "cf_internal.cuh"

namespace {

constexpr size_t kNoAllocBytes = size_t(16) << 20;  // 16 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
std::vector<void*> g_ptr;  // per device ordinal

int scratch_ptr(void** out) {
  int dev = 0;
  NRE_TRY_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  if ((int)g_ptr.size() <= dev) g_ptr.resize(dev + 1, nullptr);
  if (g_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return nre::set_error(NRE_ECUDA, "cudaGetSymbolAddress of the fixed scratch array failed: %s",
                            cudaGetErrorString(e));
    g_ptr[dev] = p;
  }
  *out = g_ptr[dev];
  return NRE_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

template <typename T>
int forward_t(nre_cf_plan* p, const T* xi, T* s, int B, cudaStream_t st) {
  using namespace nre;
  const int64_t N = p->N;
  const bool model = binned_model(p);
  const size_t tmp = align256((size_t)B * N * sizeof(T));
  const int ntmp = p->ndim == 3 ? 2 : (p->ndim == 2 ? 1 : 0);
  const int SS = model ? amp_state_size(p->n_bins) : 0;
  const size_t state = model ? align256((size_t)B * SS * sizeof(double)) : 0;
  const size_t need = ntmp * tmp + state;
  if (need > kNoAllocBytes)
    return set_error(NRE_EINVAL,
                     "cf_forward_noalloc: batch %d of this plan needs %zu bytes of scratch, the fixed array holds "
                     "%zu; use a smaller batch or cf_forward",
                     B, need, kNoAllocBytes);
  void* base = nullptr;
  NRE_TRY(scratch_ptr(&base));
  unsigned char* q = static_cast<unsigned char*>(base);
  T* tmp0 = reinterpret_cast<T*>(q);
  T* tmp1 = reinterpret_cast<T*>(q + (ntmp > 1 ? tmp : 0));
  double* stp = reinterpret_cast<double*>(q + ntmp * tmp);
  Pro<T> pro{};
  pro.mode = PRO_AMP;
  pro.x = xi;
  pro.xs = p->stride;
  Epi<T> epi{};
  epi.mode = EPI_OFFSET;
  epi.y = s;
  epi.ys = N;
  epi.offset = p->offset_mean;
  if (model) {
    NRE_TRY(amp_forward<T>(amp_prior_of(p), xi + N, p->stride, stp, B, st));
    pro.av = amp_view<T>(p, stp + as_A(p->n_bins), SS);
  } else {
    pro.av = amp_view<T>(p, nullptr, 0);
  }
  int np = 0;
  return run_hartley<T>(p, B, pro, epi, nullptr, tmp0, tmp1, nullptr, &np, st);
}

}  // namespace

extern "C" int cf_forward_noalloc(nre_cf_plan* plan, const void* xi, void* s, int batch, nre_stream_t stream) {
  nre::clear_error();
  if (!plan) return nre::set_error(NRE_EINVAL, "plan must not be NULL");
  if (batch < 0 || batch > 65535) return nre::set_error(NRE_EINVAL, "batch must be in [0, 65535]");
  if (batch == 0) return NRE_OK;
  if (!xi || !s) return nre::set_error(NRE_EINVAL, "NULL array argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->dtype == NRE_F64) return forward_t<double>(plan, (const double*)xi, (double*)s, batch, st);
  return forward_t<float>(plan, (const float*)xi, (float*)s, batch, st);
}
