// Launch tracing: every kernel launch of the library goes through
// prof_begin / prof_end.  A process-wide counter always counts launches; when
// tracing is enabled, each launch is also bracketed by a pair of CUDA events
// recorded on its own stream and tagged with the kernel name and the
// algorithmic bytes it must move (unique bytes of its global inputs and
// outputs), so that a caller can read per-kernel device time and achieved
// bandwidth for the region it traced.
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace nre {

namespace {
struct Rec {
  const char* name;
  double bytes;
  cudaEvent_t a, b;
};
std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_on{0};
std::mutex g_mu;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
thread_local int t_open = -1;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

std::atomic<long long>& dev_bytes() {
  static std::atomic<long long> b{0};
  return b;
}

void prof_add_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

bool prof_tracing() { return g_on.load(std::memory_order_relaxed) != 0; }

void prof_begin(const char* name, double bytes, cudaStream_t st) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Rec r{name, bytes, take_event(), take_event()};
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  t_open = (int)g_recs.size() - 1;
}

void prof_end(cudaStream_t st) {
  if (!g_on.load(std::memory_order_relaxed) || t_open < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEventRecord(g_recs[t_open].b, st);
  t_open = -1;
}

}  // namespace nre

using namespace nre;

extern "C" {

unsigned long long nre_launch_count(void) { return g_launches.load(); }

int nre_device_bytes(int64_t* bytes) {
  if (!bytes) return set_error(NRE_EINVAL, "bytes must not be NULL");
  *bytes = (int64_t)dev_bytes().load();
  return NRE_OK;
}

int nre_prof_enable(int on) {
  g_on.store(on ? 1 : 0);
  return NRE_OK;
}

// Synchronises the device, then writes a JSON object
// {"kernel": [launches, total_ms, bytes], ...} of the traced launches into buf
// and clears the record.  Returns NRE_EINVAL if buf is too small.
int nre_prof_report(char* buf, size_t len) {
  clear_error();
  if (!buf || len == 0) return set_error(NRE_EINVAL, "buffer must not be empty");
  NRE_TRY_CUDA(cudaDeviceSynchronize());
  std::lock_guard<std::mutex> lk(g_mu);
  std::map<std::string, std::vector<double>> acc;
  for (auto& r : g_recs) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    auto& v = acc[r.name];
    if (v.empty()) v.assign(3, 0.0);
    v[0] += 1;
    v[1] += ms;
    v[2] += r.bytes;
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  std::string out = "{";
  bool first = true;
  for (auto& kv : acc) {
    char tmp[256];
    snprintf(tmp, sizeof tmp, "%s\"%s\": [%.0f, %.6f, %.0f]", first ? "" : ", ", kv.first.c_str(),
             kv.second[0], kv.second[1], kv.second[2]);
    out += tmp;
    first = false;
  }
  out += "}";
  if (out.size() + 1 > len) return set_error(NRE_EINVAL, "report needs %zu bytes", out.size() + 1);
  memcpy(buf, out.c_str(), out.size() + 1);
  return NRE_OK;
}

}  // extern "C"
