// Request loop for sampling solves (serve_*): continuous batching of CG solves
// of correlated-field metrics with different grids and likelihoods.
//
// Every admitted request owns a "slot object" for its lifetime: a plan, a
// likelihood, a metric, input / output device buffers, a non-blocking CUDA
// stream, an event and a page-locked copy of its CG scalars.  Slot objects are
// kept after their request completes and reused by the next request with the
// same key (grid, amplitude prior, likelihood, samples, preconditioner), which
// re-linearises the metric in place, so steady-state serving allocates and
// frees nothing (cudaFree would synchronise the whole device).
//
// Host threads:
//   admission  (cfg.prep_threads of them, so that the host-side set-up of
//              several requests overlaps) FIFO over the queue; each admits the
//              head when a slot is free and its
//              footprint fits the budget (evicting idle slot objects first),
//              uploads the inputs, (re)linearises the metric, sets up the
//              preconditioner, forms the MGVI right-hand sides, starts CG and,
//              on first use of a slot object, captures one chunk of CG
//              iterations as a CUDA graph;
//   launcher   keeps every running request busy: when a request's previous
//              chunk has finished (event query, no blocking), it reads the
//              scalars copied to host memory by that chunk and either launches
//              the next chunk or hands the request on; for requests with
//              residual correction it enqueues the FP64 residual pass after a
//              solve and, while a system is above rtol, restarts CG on the
//              cast-down residual (refine.cu);
//   completion copies x to the caller's buffer, records the result and
//              returns the slot object to the idle pool.
// The device runs the chunks of all running requests concurrently on their
// streams.
#include <time.h>

#include <algorithm>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "metric_internal.cuh"

using namespace nre;

namespace {

double now_s() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return ts.tv_sec + 1e-9 * ts.tv_nsec;
}

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

struct Geom {
  int64_t N = 1, latent = 0, S = 0, qmax = 0;
  int nb = 0, nh = 0, Lmax = 0;
};

int request_geom(const nre_serve_req* r, Geom* g) {
  if (r->ndim < 1 || r->ndim > 3) return set_error(NRE_EINVAL, "ndim must be 1, 2 or 3");
  g->N = 1;
  g->qmax = 0;
  g->Lmax = 0;
  for (int d = 0; d < r->ndim; ++d) {
    const int64_t n = r->shape[d];
    if (!is_pow2(n) || n < 8 || n > 4096)
      return set_error(NRE_EINVAL, "shape[%d] = %lld must be a power of two in [8, 4096]", d, (long long)n);
    g->N *= n;
    g->qmax += (n / 2) * (n / 2);
    g->Lmax = std::max<int>(g->Lmax, (int)n);
  }
  if (r->amp.kind == NRE_AMP_POWER_MODEL || r->amp.kind == NRE_AMP_MATERN_MODEL) {
    if (r->amp.n_bins < 2 || r->amp.n_bins > 1024) return set_error(NRE_EINVAL, "n_bins must be in [2, 1024]");
    g->nb = r->amp.n_bins;
    g->nh = r->amp.kind == NRE_AMP_POWER_MODEL ? 4 + 2 * (g->nb - 1) : 3;
  } else if (r->amp.kind == NRE_AMP_MATERN_FIXED) {
    g->nb = 0;
    g->nh = 0;
  } else {
    return set_error(NRE_EINVAL, "serving takes POWER_MODEL, MATERN_MODEL or MATERN_FIXED amplitudes");
  }
  g->latent = g->N + g->nh;
  g->S = round_up(g->latent, 64);
  return NRE_OK;
}

// Upper bound of the device bytes one slot object holds (plan tables, metric,
// CG workspace, inputs and outputs), each buffer rounded to 256 bytes.
uint64_t footprint(const nre_serve_req* r, const Geom& g, int dtype) {
  const size_t E = dtype == NRE_F64 ? 8 : 4, B = (size_t)r->n_samples;
  const size_t N = (size_t)g.N, S = (size_t)g.S, nb = (size_t)g.nb, nh = (size_t)g.nh;
  const bool pc = r->precond != NRE_PRECOND_NONE;
  size_t b = 0;
  // plan: twiddles, fixed spectrum or bin tables, row groups (<= N / 2 rows, two ints each)
  b += a256(2 * E * g.Lmax);
  if (nb == 0) b += a256(N * E);
  else b += a256(2 * (size_t)(g.qmax + 1)) + 2 * a256(nb * 8);
  b += 2 * a256(N / 2 * sizeof(int) + 16);
  // metric
  b += a256(S * E) + a256(N * E) + 2 * a256(B * N * E);
  if (nb > 0)
    b += a256((size_t)amp_state_size((int)nb) * 8) + a256(B * nb * 8) + a256(B * 128 * nb * 8) + a256(N * E) +
         a256(N * 2);
  if (nb > 0 && E == 4)  // amplitude Jacobian of the FP32 metric, in-place bin sums and their counters
    b += 2 * a256(nb * nh * 4) + a256(nh * nh * E) + a256(nh * nb * 8) + a256(B * nb * 8) +
         a256(B * kGcntStride * 4);
  // CG workspace (r, p, q and z) and scalars
  b += (pc ? 4 : 3) * a256(B * S * E) + a256(B * CG_SC_N * 8) + a256(3 * B * 64 * 8 + B * 4);
  if (pc && nb > 0)
    b += a256(B * 64 * nb * 8) + a256(B * nb * 8) + 2 * a256(nh * nb * 4) + a256(nh * nh * 4) +
         a256((1 + (size_t)sm_count()) * (1 + nb) * 8) + a256(nh * nh * E) + a256(nh * nb * 8) + 2 * a256(N * E) +
         // the FP64 Schur block: its matrix and factor (n = min(nh, nb)), S^-1, the Woodbury product
         2 * a256(std::min(nh, nb) * std::min(nh, nb) * 8 + 16) + a256(nh * nh * 8) + a256(nh * nb * 8);
  else if (pc)
    b += a256(8 + 8) + a256(N * E);
  // slot buffers: xi_p, b, x (+ eta and the formed right-hand sides)
  b += a256(S * E) + 2 * a256(B * S * E);
  if (r->eta) b += a256(B * N * E) + a256(B * S * E);
  if (r->refine > 0) {
    // FP64 plan and metric (products only), xi_p / b / x in FP64, the
    // correction workspaces of both metrics and the inner solves' graph
    b += a256(16 * g.Lmax);
    if (nb == 0) b += a256(N * 8);
    else b += a256(2 * (size_t)(g.qmax + 1)) + 2 * a256(nb * 8);
    b += 2 * a256(N / 2 * sizeof(int) + 16);
    b += a256(S * 8) + a256(N * 8) + 2 * a256(B * N * 8);
    if (nb > 0)
      b += a256((size_t)amp_state_size((int)nb) * 8) + a256(B * nb * 8) + a256(B * 128 * nb * 8) + a256(N * 8) +
           a256(N * 2);
    b += a256(S * 8) + 2 * a256(B * S * 8);
    b += 2 * a256(B * S * 8) + a256((2 * B * 64 + 2 * B) * 8 + B * 4) + 2 * a256(B * S * E);
  }
  return (uint64_t)b + (1u << 20);
}

struct Key {
  int ndim;
  int64_t shape[3];
  nre_cf_amp_params amp;
  int lik_kind, response;
  double sig;
  int B, precond, mgvi, refine;
  bool operator==(const Key& o) const {
    if (ndim != o.ndim || lik_kind != o.lik_kind || response != o.response || sig != o.sig || B != o.B ||
        precond != o.precond || mgvi != o.mgvi || refine != o.refine)
      return false;
    for (int d = 0; d < ndim; ++d)
      if (shape[d] != o.shape[d]) return false;
    const nre_cf_amp_params &a = amp, &c = o.amp;
    return a.kind == c.kind && a.k0 == c.k0 && a.gamma == c.gamma && a.variance == c.variance &&
           a.zero_mode == c.zero_mode && a.fluct_mean == c.fluct_mean && a.fluct_std == c.fluct_std &&
           a.slope_mean == c.slope_mean && a.slope_std == c.slope_std && a.flex_mean == c.flex_mean &&
           a.flex_std == c.flex_std && a.asp_mean == c.asp_mean && a.asp_std == c.asp_std &&
           a.offset_mean == c.offset_mean && a.offset_std == c.offset_std && a.n_bins == c.n_bins &&
           a.scale_mean == c.scale_mean && a.scale_std == c.scale_std && a.cutoff_mean == c.cutoff_mean &&
           a.cutoff_std == c.cutoff_std && a.lls_mean == c.lls_mean && a.lls_std == c.lls_std;
  }
};

struct SlotObj {
  Key key{};
  Geom g;
  uint64_t est = 0;
  nre_cf_plan* plan = nullptr;
  nre_lik* lik = nullptr;
  nre_metric* m = nullptr;
  DevBuf dxi, db, dx, deta, drhs;
  // residual correction: FP64 plan and metric, xi_p / b / x in FP64, the
  // passes' sums on the host, the inner solves' chunk graph
  nre_cf_plan* plan64 = nullptr;
  nre_metric* m64 = nullptr;
  DevBuf dxi64, db64, dx64;
  double* h_rf = nullptr;  // page-locked [2 B]: r.r, b.b
  cudaGraphExec_t gexec_in = nullptr;
  double gin_rtol = -1.0;
  int gin_chunk = 0;
  unsigned long long gin_kernels = 0;
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  double* h_sc = nullptr;  // page-locked [B][CG_SC_N]
  cudaGraphExec_t gexec = nullptr;
  double g_rtol = -1.0;
  int g_chunk = 0;
  unsigned long long g_kernels = 0;
  uint64_t last_used = 0;
  ~SlotObj() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (gexec_in) cudaGraphExecDestroy(gexec_in);
    if (m64) metric_destroy(m64);
    if (plan64) cf_destroy(plan64);
    if (h_rf) cudaFreeHost(h_rf);
    if (m) metric_destroy(m);
    if (lik) lik_destroy(lik);
    if (plan) cf_destroy(plan);
    if (h_sc) cudaFreeHost(h_sc);
    if (ev) cudaEventDestroy(ev);
    if (st) cudaStreamDestroy(st);
  }
};

enum JobState { J_QUEUED, J_PREP, J_RUN, J_FIN, J_DONE };

struct Job {
  uint64_t id = 0;
  nre_serve_req req{};
  Key key{};
  Geom g;
  uint64_t est = 0;
  JobState state = J_QUEUED;
  SlotObj* so = nullptr;
  bool so_broken = false;
  int iters_done = 0;
  bool inflight = false;
  // residual correction: passes taken, a pass's residual in flight, the
  // tolerance of the running solve (rtol, then the inner one)
  int pass = 0;
  bool rf_inflight = false;
  double cur_rtol = 0.0;
  int its_total[64] = {0};
  nre_serve_result res{};
};

// Relative tolerance of the CG solves for the corrections after the first.
constexpr double kInnerRtol = 1e-2;

}  // namespace

struct nre_server {
  nre_serve_cfg cfg{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_prep, cv_work, cv_fin, cv_done;
  std::deque<Job*> pending, ready, finishing;
  std::unordered_map<uint64_t, Job*> jobs;
  std::vector<SlotObj*> idle;
  int active = 0;
  uint64_t reserved = 0, peak = 0, next_id = 1, tick = 0;
  uint64_t completed = 0, reused = 0, created = 0, evicted = 0, replays = 0, chunks = 0;
  bool stop = false, prep_done = false, work_done = false;
  int prep_alive = 0;
  std::vector<std::thread> t_prep;
  std::thread t_work, t_fin;

  void run_prep();
  void run_work();
  void run_fin();
  int prepare(Job* j);
  void fail(Job* j, int status, const char* msg);
};

namespace {

void set_msg(Job* j, int status, const char* msg) {
  j->res.status = status;
  std::snprintf(j->res.error, sizeof(j->res.error), "%s", msg ? msg : "");
}

int make_slot(const Job* j, int dtype, SlotObj** out) {
  SlotObj* so = new SlotObj();
  so->key = j->key;
  so->g = j->g;
  so->est = j->est;
  const nre_serve_req& r = j->req;
  const size_t E = dtype == NRE_F64 ? 8 : 4, B = (size_t)r.n_samples;
  auto bad = [&](int s) {
    delete so;
    return s;
  };
  double spacing[3];
  for (int d = 0; d < r.ndim; ++d) spacing[d] = 1.0 / (double)r.shape[d];
  int s = cf_create(&so->plan, r.ndim, r.shape, spacing, &r.amp, dtype);
  if (s != NRE_OK) return bad(s);
  s = lik_create(&so->lik, r.lik_kind, r.response, nullptr, so->g.N, r.sigma_or_scale);
  if (s != NRE_OK) return bad(s);
  // Smaller grids get higher stream priority: their CTAs are scheduled ahead
  // of the queued CTAs of large requests, so a short solve is not stuck behind
  // the long sweeps of the requests running beside it.
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  const int prio = so->g.N <= 8192 ? greatest : so->g.N <= 65536 ? (least + greatest) / 2 : least;
  if (cudaStreamCreateWithPriority(&so->st, cudaStreamNonBlocking, prio) != cudaSuccess ||
      cudaEventCreateWithFlags(&so->ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaHostAlloc((void**)&so->h_sc, B * CG_SC_N * sizeof(double), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return bad(set_error(NRE_ECUDA, "stream / event / host buffer creation failed"));
  }
  const size_t S = (size_t)so->g.S, N = (size_t)so->g.N;
  if ((s = so->dxi.alloc(S * E)) != NRE_OK || (s = so->db.alloc(B * S * E)) != NRE_OK ||
      (s = so->dx.alloc(B * S * E)) != NRE_OK)
    return bad(s);
  if (r.eta && ((s = so->deta.alloc(B * N * E)) != NRE_OK || (s = so->drhs.alloc(B * S * E)) != NRE_OK))
    return bad(s);
  if (r.refine > 0) {
    s = cf_create(&so->plan64, r.ndim, r.shape, spacing, &r.amp, NRE_F64);
    if (s != NRE_OK) return bad(s);
    if ((s = so->dxi64.alloc(S * 8)) != NRE_OK || (s = so->db64.alloc(B * S * 8)) != NRE_OK ||
        (s = so->dx64.alloc(B * S * 8)) != NRE_OK)
      return bad(s);
    if (cudaHostAlloc((void**)&so->h_rf, 2 * B * sizeof(double), cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return bad(set_error(NRE_ECUDA, "host buffer creation failed"));
    }
  }
  *out = so;
  return NRE_OK;
}

// FP32 -> FP64 copy of n entries.
__global__ void k_widen(const float* src, double* dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = double(src[i]);
}

int widen(const void* src, void* dst, int64_t n, cudaStream_t st) {
  prof_begin("serve_widen", (double)n * 12, st);
  k_widen<<<(int)std::min<int64_t>((n + 255) / 256, 1216), 256, 0, st>>>((const float*)src, (double*)dst, n);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  return NRE_OK;
}

// One chunk of `iters` CG iterations and the copy of the scalars to host.
int enqueue_chunk(SlotObj* so, int iters, double rtol) {
  const int B = so->key.B;
  NRE_TRY(cg_iterate(so->m, so->dx.p, B, iters, rtol, so->st));
  NRE_TRY_CUDA(cudaMemcpyAsync(so->h_sc, so->m->cg_sc.p, (size_t)B * CG_SC_N * sizeof(double),
                               cudaMemcpyDeviceToHost, so->st));
  return NRE_OK;
}

// Capture one chunk as a graph (the pointers of a slot object never change)
// into the first solve's graph or (inner) the correction solves' one.  A
// capture that fails leaves those solves on direct launches.
void capture_chunk(SlotObj* so, int chunk, double rtol, bool inner = false) {
  cudaGraphExec_t& gx = inner ? so->gexec_in : so->gexec;
  if (gx) {
    cudaGraphExecDestroy(gx);
    gx = nullptr;
  }
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(so->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const int s = enqueue_chunk(so, chunk, rtol);
  const cudaError_t e = cudaStreamEndCapture(so->st, &g);
  if (s != NRE_OK || e != cudaSuccess || !g) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    return;
  }
  size_t n = 0;
  cudaGraphGetNodes(g, nullptr, &n);
  std::vector<cudaGraphNode_t> nodes(n);
  unsigned long long kernels = 0;
  if (n > 0 && cudaGraphGetNodes(g, nodes.data(), &n) == cudaSuccess)
    for (size_t i = 0; i < n; ++i) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
    }
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
    cudaGetLastError();
    ex = nullptr;
  }
  cudaGraphDestroy(g);
  gx = ex;
  (inner ? so->gin_rtol : so->g_rtol) = rtol;
  (inner ? so->gin_chunk : so->g_chunk) = chunk;
  (inner ? so->gin_kernels : so->g_kernels) = kernels;
}

}  // namespace

void nre_server::fail(Job* j, int status, const char* msg) {
  set_msg(j, status, msg);
  j->res.t_done = now_s();
  j->state = J_DONE;
}

// Admission and set-up of the head of the queue (called without the lock).
int nre_server::prepare(Job* j) {
  const nre_serve_req& r = j->req;
  SlotObj* so = j->so;
  const int B = r.n_samples;
  const int dt = cfg.dtype;
  const size_t E = dt == NRE_F64 ? 8 : 4;
  const size_t S = (size_t)j->g.S, L = (size_t)j->g.latent, N = (size_t)j->g.N;
  NRE_TRY_CUDA(cudaMemcpyAsync(so->dxi.p, r.xi_p, L * E, cudaMemcpyHostToDevice, so->st));
  NRE_TRY_CUDA(cudaMemcpy2DAsync(so->db.p, S * E, r.b, L * E, L * E, B, cudaMemcpyHostToDevice, so->st));
  if (r.eta) NRE_TRY_CUDA(cudaMemcpyAsync(so->deta.p, r.eta, (size_t)B * N * E, cudaMemcpyHostToDevice, so->st));
  if (!so->m) {
    NRE_TRY(metric_create(&so->m, NRE_MODEL_CF, so->plan, so->lik, so->dxi.p, B, so->st));
  } else {
    NRE_TRY(metric_relinearize(so->m, so->dxi.p, so->st));
  }
  NRE_TRY(metric_set_precond(so->m, r.precond, so->st));
  const void* rhs = so->db.p;
  if (r.eta) {
    NRE_TRY(mgvi_rhs(so->m, so->db.p, so->deta.p, so->drhs.p, B, so->st));
    rhs = so->drhs.p;
  }
  if (r.refine > 0) {
    // the FP64 system at the same point: widened xi_p and right-hand sides
    NRE_TRY(widen(so->dxi.p, so->dxi64.p, (int64_t)S, so->st));
    if (!so->m64) NRE_TRY(metric_create(&so->m64, NRE_MODEL_CF, so->plan64, so->lik, so->dxi64.p, B, so->st));
    else NRE_TRY(metric_relinearize(so->m64, so->dxi64.p, so->st));
    NRE_TRY(widen(rhs, so->db64.p, (int64_t)B * S, so->st));
    NRE_TRY_CUDA(cudaMemsetAsync(so->dx64.p, 0, (size_t)B * S * 8, so->st));
  }
  j->pass = 0;
  j->rf_inflight = false;
  j->cur_rtol = r.rtol;
  for (int i = 0; i < B; ++i) j->its_total[i] = 0;
  NRE_TRY(cg_begin(so->m, rhs, so->dx.p, B, r.rtol, so->st));
  const int chunk = cfg.chunk_iters;
  if (cfg.use_graphs && (so->g_chunk != chunk || so->g_rtol != r.rtol || !so->gexec))
    capture_chunk(so, chunk, r.rtol);
  return NRE_OK;
}

void nre_server::run_prep() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    cv_prep.wait(lk, [&] { return stop || (!pending.empty() && active < cfg.max_slots); });
    if (stop) break;
    Job* j = pending.front();
    SlotObj* so = nullptr;
    for (size_t i = 0; i < idle.size(); ++i)
      if (idle[i]->key == j->key) {
        so = idle[i];
        idle.erase(idle.begin() + i);
        ++reused;
        break;
      }
    if (!so) {
      std::vector<SlotObj*> drop;
      while (reserved + j->est > cfg.hbm_budget_bytes && !idle.empty()) {
        auto it = std::min_element(idle.begin(), idle.end(),
                                   [](const SlotObj* a, const SlotObj* b) { return a->last_used < b->last_used; });
        reserved -= (*it)->est;
        drop.push_back(*it);
        idle.erase(it);
        ++evicted;
      }
      if (!drop.empty()) {
        lk.unlock();
        for (SlotObj* d : drop) delete d;
        lk.lock();
        // another admission thread may have taken the head of the queue (or
        // the last free slot) while the lock was released: start over
        continue;
      }
      if (reserved + j->est > cfg.hbm_budget_bytes) {
        // wait for a running request to release memory
        cv_prep.wait(lk);
        continue;
      }
      reserved += j->est;
      peak = std::max(peak, reserved);
    }
    pending.pop_front();
    ++active;
    j->state = J_PREP;
    j->res.t_start = now_s();
    j->res.device_bytes = j->est;
    lk.unlock();
    int s = NRE_OK;
    if (!so) {
      s = make_slot(j, cfg.dtype, &so);
      if (s == NRE_OK) {
        std::lock_guard<std::mutex> g2(mu);
        ++created;
      }
    }
    j->so = so;
    if (s == NRE_OK) s = prepare(j);
    if (s != NRE_OK) {
      const std::string msg = nre_last_error();
      lk.lock();
      set_msg(j, s, msg.c_str());
      j->so_broken = true;
      if (!so) reserved -= j->est;
      j->state = J_FIN;
      finishing.push_back(j);
      cv_fin.notify_one();
      continue;
    }
    lk.lock();
    j->state = J_RUN;
    ready.push_back(j);
    cv_work.notify_one();
  }
  // shutting down: requests that were never admitted fail
  while (!pending.empty()) {
    Job* j = pending.front();
    pending.pop_front();
    fail(j, NRE_EBUSY, "server destroyed before the request was admitted");
  }
  if (--prep_alive == 0) prep_done = true;
  cv_done.notify_all();
  cv_work.notify_all();
  cv_prep.notify_all();
}

void nre_server::run_work() {
  cudaSetDevice(device);
  std::vector<Job*> run;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(mu);
      while (!ready.empty()) {
        run.push_back(ready.front());
        ready.pop_front();
      }
      if (run.empty()) {
        if (prep_done) break;
        cv_work.wait(lk, [&] { return !ready.empty() || prep_done; });
        continue;
      }
    }
    bool progressed = false;
    std::vector<Job*> done;
    for (Job* j : run) {
      SlotObj* so = j->so;
      const nre_serve_req& r = j->req;
      const int B = r.n_samples;
      if (j->inflight) {
        const cudaError_t q = cudaEventQuery(so->ev);
        if (q == cudaErrorNotReady) continue;
        j->inflight = false;
        progressed = true;
        if (q != cudaSuccess) {
          set_msg(j, NRE_ECUDA, cudaGetErrorString(q));
          j->so_broken = true;
          done.push_back(j);
          continue;
        }
        int s = NRE_OK;
        if (j->rf_inflight) {
          // a residual pass finished: the true residuals decide
          j->rf_inflight = false;
          std::vector<int> act(B, 0);
          bool anyr = false;
          for (int i = 0; i < B; ++i) {
            const double bb = so->h_rf[B + i];
            const double rel = bb > 0 ? std::sqrt(so->h_rf[i] / bb) : 0.0;
            j->res.relres[i] = rel;
            act[i] = rel > r.rtol ? 1 : 0;
            anyr = anyr || act[i];
          }
          if (!anyr || j->pass >= r.refine) {
            done.push_back(j);
            continue;
          }
          // the next correction: CG on the cast-down residual of the systems above rtol
          void* rlo = nullptr;
          s = refine_down(so->m, so->m64, B, act.data(), &rlo, so->st);
          if (s == NRE_OK) s = cg_begin(so->m, rlo, so->dx.p, B, kInnerRtol, so->st);
          if (s == NRE_OK && cfg.use_graphs &&
              (!so->gexec_in || so->gin_chunk != cfg.chunk_iters || so->gin_rtol != kInnerRtol))
            capture_chunk(so, cfg.chunk_iters, kInnerRtol, true);
          ++j->pass;
          j->iters_done = 0;
          j->cur_rtol = kInnerRtol;
        } else {
          bool any = false;
          for (int i = 0; i < B; ++i) any |= so->h_sc[(size_t)i * CG_SC_N + CG_SC_ACTIVE] != 0.0;
          if (!any || j->iters_done >= r.maxiter) {
            if (r.refine <= 0) {
              done.push_back(j);
              continue;
            }
            // the solve of this pass is done: x64 += its result, r = b - M64 x64
            for (int i = 0; i < B; ++i) j->its_total[i] += (int)so->h_sc[(size_t)i * CG_SC_N + CG_SC_ITERS];
            double* sums = nullptr;
            s = refine_residual(so->m, so->m64, so->db64.as<double>(), so->dx64.as<double>(), so->dx.p, B,
                                j->pass == 0, &sums, so->st);
            if (s == NRE_OK &&
                (cudaMemcpyAsync(so->h_rf, sums, 2 * B * sizeof(double), cudaMemcpyDeviceToHost, so->st) !=
                     cudaSuccess ||
                 cudaEventRecord(so->ev, so->st) != cudaSuccess)) {
              cudaGetLastError();
              s = set_error(NRE_ECUDA, "residual pass: copy / event record failed");
            }
            if (s != NRE_OK) {
              set_msg(j, s, nre_last_error());
              j->so_broken = true;
              done.push_back(j);
              continue;
            }
            j->rf_inflight = true;
            j->inflight = true;
            continue;
          }
        }
        if (s != NRE_OK) {
          set_msg(j, s, nre_last_error());
          j->so_broken = true;
          done.push_back(j);
          continue;
        }
      }
      const int k = std::min(cfg.chunk_iters, r.maxiter - j->iters_done);
      const double rt = j->cur_rtol;
      cudaGraphExec_t gx = j->pass == 0 ? so->gexec : so->gexec_in;
      const int gchunk = j->pass == 0 ? so->g_chunk : so->gin_chunk;
      const double grt = j->pass == 0 ? so->g_rtol : so->gin_rtol;
      const unsigned long long gk = j->pass == 0 ? so->g_kernels : so->gin_kernels;
      int s = NRE_OK;
      bool graph = false;
      if (gx && k == gchunk && grt == rt) {
        const cudaError_t e = cudaGraphLaunch(gx, so->st);
        if (e != cudaSuccess) {
          cudaGetLastError();
          s = set_error(NRE_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
        }
        graph = true;
      } else {
        s = enqueue_chunk(so, k, rt);
      }
      if (s == NRE_OK && cudaEventRecord(so->ev, so->st) != cudaSuccess)
        s = set_error(NRE_ECUDA, "cudaEventRecord failed");
      if (s != NRE_OK) {
        set_msg(j, s, nre_last_error());
        j->so_broken = true;
        done.push_back(j);
        continue;
      }
      if (graph) prof_add_launches(gk);
      j->iters_done += k;
      j->inflight = true;
      progressed = true;
      std::lock_guard<std::mutex> g2(mu);
      ++chunks;
      if (graph) ++replays;
    }
    if (!done.empty()) {
      for (Job* j : done) run.erase(std::find(run.begin(), run.end(), j));
      std::lock_guard<std::mutex> lk(mu);
      for (Job* j : done) {
        j->state = J_FIN;
        finishing.push_back(j);
      }
      cv_fin.notify_one();
    }
    if (!progressed) {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait_for(lk, std::chrono::microseconds(50), [&] { return !ready.empty(); });
    }
  }
  std::lock_guard<std::mutex> lk(mu);
  work_done = true;
  cv_fin.notify_all();
}

void nre_server::run_fin() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    cv_fin.wait(lk, [&] { return !finishing.empty() || work_done; });
    if (finishing.empty()) {
      if (work_done) break;
      continue;
    }
    Job* j = finishing.front();
    finishing.pop_front();
    lk.unlock();
    SlotObj* so = j->so;
    const nre_serve_req& r = j->req;
    const int B = r.n_samples;
    if (so && !j->so_broken && r.refine > 0) {
      // FP64 solutions; relres already holds the true residuals
      const size_t S = (size_t)j->g.S, L = (size_t)j->g.latent;
      cudaError_t e = cudaMemcpy2DAsync(r.x64_out, L * 8, so->dx64.p, S * 8, L * 8, B, cudaMemcpyDeviceToHost, so->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(so->st);
      if (e != cudaSuccess) {
        cudaGetLastError();
        set_msg(j, NRE_ECUDA, cudaGetErrorString(e));
        j->so_broken = true;
      } else {
        bool conv = true;
        for (int i = 0; i < B; ++i) {
          j->res.iters[i] = j->its_total[i];
          if (j->res.relres[i] > r.rtol) conv = false;
        }
        if (!conv) set_msg(j, NRE_ENOTCONV, "some system missed rtol (true residual) after the correction passes");
      }
    } else if (so && !j->so_broken) {
      const size_t E = cfg.dtype == NRE_F64 ? 8 : 4;
      const size_t S = (size_t)j->g.S, L = (size_t)j->g.latent;
      cudaError_t e = cudaMemcpy2DAsync(r.x_out, L * E, so->dx.p, S * E, L * E, B, cudaMemcpyDeviceToHost, so->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(so->st);
      if (e != cudaSuccess) {
        cudaGetLastError();
        set_msg(j, NRE_ECUDA, cudaGetErrorString(e));
        j->so_broken = true;
      } else {
        bool conv = true;
        for (int i = 0; i < B; ++i) {
          const double* c = so->h_sc + (size_t)i * CG_SC_N;
          j->res.iters[i] = (int)c[CG_SC_ITERS];
          j->res.relres[i] = c[CG_SC_BB] > 0 ? std::sqrt(c[CG_SC_RR] / c[CG_SC_BB]) : 0.0;
          if (j->res.relres[i] > r.rtol) conv = false;
        }
        if (!conv) set_msg(j, NRE_ENOTCONV, "some system missed rtol within maxiter");
      }
    }
    SlotObj* drop = nullptr;
    lk.lock();
    if (so) {
      if (j->so_broken) {
        reserved -= so->est;
        drop = so;
      } else {
        so->last_used = ++tick;
        idle.push_back(so);
      }
    }
    j->so = nullptr;
    j->res.t_done = now_s();
    j->state = J_DONE;
    --active;
    ++completed;
    cv_done.notify_all();
    cv_prep.notify_one();
    if (drop) {
      lk.unlock();
      delete drop;
      lk.lock();
    }
  }
}

extern "C" {

int serve_footprint(const nre_serve_req* req, int dtype, uint64_t* bytes) {
  clear_error();
  if (!req || !bytes) return set_error(NRE_EINVAL, "NULL argument");
  if (dtype != NRE_F32 && dtype != NRE_F64) return set_error(NRE_EINVAL, "dtype must be NRE_F32 or NRE_F64");
  Geom g;
  NRE_TRY(request_geom(req, &g));
  if (req->n_samples < 1 || req->n_samples > 64) return set_error(NRE_EINVAL, "n_samples must be in [1, 64]");
  *bytes = footprint(req, g, dtype);
  return NRE_OK;
}

int serve_create(nre_server** out, const nre_serve_cfg* cfg) {
  clear_error();
  if (!out || !cfg) return set_error(NRE_EINVAL, "NULL argument");
  *out = nullptr;
  if (cfg->max_slots < 1 || cfg->max_slots > 256) return set_error(NRE_EINVAL, "max_slots must be in [1, 256]");
  if (cfg->dtype != NRE_F32 && cfg->dtype != NRE_F64) return set_error(NRE_EINVAL, "dtype must be NRE_F32 or NRE_F64");
  if (cfg->chunk_iters < 0 || cfg->chunk_iters > 1024) return set_error(NRE_EINVAL, "chunk_iters must be in [0, 1024]");
  if (cfg->prep_threads < 0 || cfg->prep_threads > 64) return set_error(NRE_EINVAL, "prep_threads must be in [0, 64]");
  nre_server* s = new nre_server();
  s->cfg = *cfg;
  if (s->cfg.chunk_iters == 0) s->cfg.chunk_iters = 8;
  if (s->cfg.prep_threads == 0) s->cfg.prep_threads = 8;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess && s->cfg.hbm_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    e = cudaMemGetInfo(&fr, &tot);
    s->cfg.hbm_budget_bytes = fr / 2;
  }
  if (e != cudaSuccess) {
    delete s;
    return set_error(NRE_ECUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
  }
  const int np = s->cfg.prep_threads;
  s->prep_alive = np;
  for (int i = 0; i < np; ++i) s->t_prep.emplace_back([s] { s->run_prep(); });
  s->t_work = std::thread([s] { s->run_work(); });
  s->t_fin = std::thread([s] { s->run_fin(); });
  *out = s;
  return NRE_OK;
}

int serve_submit(nre_server* s, const nre_serve_req* req, uint64_t* id) {
  clear_error();
  if (!s || !req || !id) return set_error(NRE_EINVAL, "NULL argument");
  Geom g;
  NRE_TRY(request_geom(req, &g));
  if (req->n_samples < 1 || req->n_samples > 64) return set_error(NRE_EINVAL, "n_samples must be in [1, 64]");
  if (!(req->rtol > 0.0) || req->maxiter < 1) return set_error(NRE_EINVAL, "rtol must be > 0 and maxiter >= 1");
  if (req->lik_kind != NRE_LIK_GAUSS && req->lik_kind != NRE_LIK_POISSON)
    return set_error(NRE_EINVAL, "unknown likelihood kind %d", req->lik_kind);
  if (!(req->sigma_or_scale > 0.0)) return set_error(NRE_EINVAL, "sigma / scale must be positive");
  if (req->response != NRE_RESP_EXP && req->response != NRE_RESP_IDENTITY)
    return set_error(NRE_EINVAL, "unknown response %d", req->response);
  if (req->lik_kind == NRE_LIK_POISSON && req->response != NRE_RESP_EXP)
    return set_error(NRE_EINVAL, "the Poisson likelihood uses the exponential response");
  if (req->precond != NRE_PRECOND_NONE && req->precond != NRE_PRECOND_HARMONIC)
    return set_error(NRE_EINVAL, "unknown preconditioner %d", req->precond);
  if (req->refine < 0 || req->refine > 16) return set_error(NRE_EINVAL, "refine must be in [0, 16]");
  if (req->refine > 0 && s->cfg.dtype != NRE_F32)
    return set_error(NRE_EINVAL, "residual correction needs an FP32 server");
  if (!req->xi_p || !req->b || (req->refine > 0 ? !req->x64_out : !req->x_out))
    return set_error(NRE_EINVAL, "NULL array in the request");
  const uint64_t est = footprint(req, g, s->cfg.dtype);
  if (est > s->cfg.hbm_budget_bytes)
    return set_error(NRE_EBUSY, "request needs %llu device bytes, the budget is %llu", (unsigned long long)est,
                     (unsigned long long)s->cfg.hbm_budget_bytes);
  Job* j = new Job();
  j->req = *req;
  j->g = g;
  j->est = est;
  Key& k = j->key;
  k.ndim = req->ndim;
  for (int d = 0; d < 3; ++d) k.shape[d] = d < req->ndim ? req->shape[d] : 1;
  k.amp = req->amp;
  k.amp.amp_array = nullptr;
  k.lik_kind = req->lik_kind;
  k.response = req->response;
  k.sig = req->sigma_or_scale;
  k.B = req->n_samples;
  k.precond = req->precond;
  k.mgvi = req->eta ? 1 : 0;
  k.refine = req->refine > 0 ? 1 : 0;
  j->res.t_submit = now_s();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    delete j;
    return set_error(NRE_EBUSY, "server is shutting down");
  }
  j->id = s->next_id++;
  s->jobs[j->id] = j;
  s->pending.push_back(j);
  *id = j->id;
  s->cv_prep.notify_one();
  return NRE_OK;
}

int serve_poll(nre_server* s, uint64_t id, nre_serve_result* res, int timeout_ms) {
  clear_error();
  if (!s || !res) return set_error(NRE_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return set_error(NRE_EINVAL, "unknown or already collected request id %llu", (unsigned long long)id);
  Job* j = it->second;
  auto done = [&] { return j->state == J_DONE; };
  if (!done()) {
    if (timeout_ms == 0) return NRE_EAGAIN;
    if (timeout_ms < 0) s->cv_done.wait(lk, done);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) return NRE_EAGAIN;
  }
  *res = j->res;
  s->jobs.erase(it);
  delete j;
  return NRE_OK;
}

int serve_stats(nre_server* s, nre_serve_stats* st) {
  clear_error();
  if (!s || !st) return set_error(NRE_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  st->budget = s->cfg.hbm_budget_bytes;
  st->reserved = s->reserved;
  st->peak_reserved = s->peak;
  st->active = s->active;
  st->queued = (int)s->pending.size();
  st->idle_objects = (int)s->idle.size();
  st->completed = s->completed;
  st->reused = s->reused;
  st->created = s->created;
  st->evicted = s->evicted;
  st->graph_replays = s->replays;
  st->chunks = s->chunks;
  return NRE_OK;
}

int serve_destroy(nre_server* s) {
  clear_error();
  if (!s) return NRE_OK;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    // let admitted work finish, then stop admitting
    s->cv_done.wait(lk, [&] { return s->active == 0 || s->prep_done; });
    s->stop = true;
  }
  s->cv_prep.notify_all();
  for (auto& t : s->t_prep) t.join();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->cv_work.notify_all();
  }
  s->t_work.join();
  s->t_fin.join();
  for (SlotObj* o : s->idle) delete o;
  for (auto& kv : s->jobs) delete kv.second;
  delete s;
  return NRE_OK;
}

}  // extern "C"
