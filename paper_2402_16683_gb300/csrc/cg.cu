// Batched conjugate gradients on the metric (the linear MGVI sample draw).
//
// Sec. "Variational Inference": draw_linear_kwargs / cg_kwargs - samples are
// drawn by CG on M_p (maxiter = 100 in the example).  Textbook Hestenes-Stiefel
// per system b: x_0 = 0, r_0 = b, p_0 = r_0; alpha = r.r / p.Mp;
// x += alpha p; r -= alpha Mp; beta = r'.r' / r.r; p = r' + beta p.  A system
// stops (x frozen) once ||r|| <= rtol ||b|| on the recursive residual; rtol = 0
// runs exactly maxiter iterations.  Inner products and alpha / beta are FP64;
// each thread folds short runs of products in the vector dtype into an FP64
// accumulator.
#include <cmath>

#include "metric_internal.cuh"

using namespace nre;

namespace {

constexpr int CG_THREADS = 256;
enum { SC_RR = 0, SC_BB = 1, SC_ALPHA = 2, SC_BETA = 3, SC_ACTIVE = 4, SC_ITERS = 5, SC_N = 8 };

// Blocks per system of the vector kernels.
int cg_blocks(int64_t n) {
  int64_t nb = (n + CG_THREADS * 8 - 1) / (CG_THREADS * 8);
  if (nb > 64) nb = 64;
  if (nb < 1) nb = 1;
  return (int)nb;
}

// Sum over the block, then one partial per (system, block).
__device__ void write_partial(double acc, double* part) {
  __shared__ double red[CG_THREADS / 32];
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

template <typename T>
__global__ void __launch_bounds__(CG_THREADS) k_cg_init(const T* b, T* x, T* r, T* p, int64_t n,
                                                       int64_t S, double* part) {
  const int64_t off = (int64_t)blockIdx.y * S;
  double acc = 0.0;
  T run = T(0);
  int cnt = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T v = b[off + i];
    x[off + i] = T(0);
    r[off + i] = v;
    p[off + i] = v;
    run += v * v;
    if (++cnt == 8) {
      acc += double(run);
      run = T(0);
      cnt = 0;
    }
  }
  acc += double(run);
  write_partial(acc, part);
}

__global__ void k_cg_start(double* sc, const double* part, int nblk, double rtol) {
  const int b = blockIdx.x;
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < nblk; ++i) s += part[b * nblk + i];
  double* c = sc + b * SC_N;
  c[SC_RR] = s;
  c[SC_BB] = s;
  c[SC_ALPHA] = 0.0;
  c[SC_BETA] = 0.0;
  c[SC_ITERS] = 0.0;
  c[SC_ACTIVE] = (s > 0.0 && (rtol <= 0.0 || sqrt(s) > rtol * sqrt(s))) ? 1.0 : 0.0;
}

template <typename T>
__global__ void __launch_bounds__(CG_THREADS) k_cg_dot(const T* a, const T* q, int64_t n, int64_t S,
                                                      double* part) {
  const int64_t off = (int64_t)blockIdx.y * S;
  double acc = 0.0;
  T run = T(0);
  int cnt = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    run += a[off + i] * q[off + i];
    if (++cnt == 8) {
      acc += double(run);
      run = T(0);
      cnt = 0;
    }
  }
  acc += double(run);
  write_partial(acc, part);
}

// alpha = r.r / p.Mp from the dot partials (every block sums them in the same
// order), then x += alpha p, r -= alpha q and partials of r'.r'.
template <typename T>
__global__ void __launch_bounds__(CG_THREADS) k_cg_update(T* x, T* r, const T* p, const T* q, int64_t n,
                                                         int64_t S, const double* sc, const double* pq_part,
                                                         double* rr_part) {
  const int b = blockIdx.y, nblk = gridDim.x;
  const double* c = sc + b * SC_N;
  const bool active = c[SC_ACTIVE] != 0.0;
  double pq = 0.0;
  for (int i = 0; i < nblk; ++i) pq += pq_part[b * nblk + i];
  const double alpha_d = active && pq != 0.0 ? c[SC_RR] / pq : 0.0;
  const T alpha = T(alpha_d);
  const int64_t off = (int64_t)b * S;
  double acc = 0.0;
  T run = T(0);
  int cnt = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T ri = r[off + i];
    if (active) {
      x[off + i] += alpha * p[off + i];
      ri -= alpha * q[off + i];
      r[off + i] = ri;
    }
    run += ri * ri;
    if (++cnt == 8) {
      acc += double(run);
      run = T(0);
      cnt = 0;
    }
  }
  acc += double(run);
  write_partial(acc, rr_part);
}

// beta = r'.r' / r.r; p = r' + beta p; bookkeeping of the scalars.  Block 0 of
// each system updates the scalars after all blocks have read them: the scalar
// update is deferred to k_cg_finish.
template <typename T>
__global__ void __launch_bounds__(CG_THREADS) k_cg_pupdate(T* p, const T* r, int64_t n, int64_t S,
                                                          const double* sc, const double* rr_part,
                                                          int nblk_rr) {
  const int b = blockIdx.y;
  const double* c = sc + b * SC_N;
  if (c[SC_ACTIVE] == 0.0) return;
  double rr_new = 0.0;
  for (int i = 0; i < nblk_rr; ++i) rr_new += rr_part[b * nblk_rr + i];
  const T beta = T(rr_new / c[SC_RR]);
  const int64_t off = (int64_t)b * S;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[off + i] = r[off + i] + beta * p[off + i];
}

__global__ void k_cg_finish(double* sc, const double* rr_part, int nblk, double rtol) {
  const int b = blockIdx.x;
  if (threadIdx.x != 0) return;
  double* c = sc + b * SC_N;
  if (c[SC_ACTIVE] == 0.0) return;
  double rr_new = 0.0;
  for (int i = 0; i < nblk; ++i) rr_new += rr_part[b * nblk + i];
  c[SC_BETA] = rr_new / c[SC_RR];
  c[SC_RR] = rr_new;
  c[SC_ITERS] += 1.0;
  if (rtol > 0.0 && sqrt(rr_new) <= rtol * sqrt(c[SC_BB])) c[SC_ACTIVE] = 0.0;
}

template <typename T>
int cg_t(nre_metric* m, const T* b, T* x, int B, double rtol, int maxiter, int* iters_out,
         double* relres_out, cudaStream_t st) {
  const int64_t n = m->latent, S = m->stride;
  NRE_TRY(ensure(m->cg_r, (size_t)B * S * sizeof(T)));
  NRE_TRY(ensure(m->cg_p, (size_t)B * S * sizeof(T)));
  NRE_TRY(ensure(m->cg_q, (size_t)B * S * sizeof(T)));
  NRE_TRY(ensure(m->cg_sc, (size_t)B * SC_N * sizeof(double)));
  const int nblk = cg_blocks(n);
  NRE_TRY(ensure(m->cg_part, (size_t)2 * B * nblk * sizeof(double)));
  T* r = m->cg_r.as<T>();
  T* p = m->cg_p.as<T>();
  T* q = m->cg_q.as<T>();
  double* sc = m->cg_sc.as<double>();
  double* part_a = m->cg_part.as<double>();
  double* part_b = part_a + (size_t)B * nblk;
  const dim3 grid(nblk, B);
  const double vb = (double)B * n * sizeof(T);
  prof_begin("cg_init", 4 * vb, st);
  k_cg_init<T><<<grid, CG_THREADS, 0, st>>>(b, x, r, p, n, S, part_a);
  prof_end(st);
  prof_begin("cg_scalars", 0.0, st);
  k_cg_start<<<B, 32, 0, st>>>(sc, part_a, nblk, rtol);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  m->cg_host.resize((size_t)B * SC_N);
  const int check_every = 8;
  for (int it = 0; it < maxiter; ++it) {
    NRE_TRY(metric_apply_impl(m, p, q, B, st));
    prof_begin("cg_dot", 2 * vb, st);
    k_cg_dot<T><<<grid, CG_THREADS, 0, st>>>(p, q, n, S, part_a);
    prof_end(st);
    prof_begin("cg_update", 6 * vb, st);
    k_cg_update<T><<<grid, CG_THREADS, 0, st>>>(x, r, p, q, n, S, sc, part_a, part_b);
    prof_end(st);
    prof_begin("cg_pupdate", 3 * vb, st);
    k_cg_pupdate<T><<<grid, CG_THREADS, 0, st>>>(p, r, n, S, sc, part_b, nblk);
    prof_end(st);
    prof_begin("cg_scalars", 0.0, st);
    k_cg_finish<<<B, 32, 0, st>>>(sc, part_b, nblk, rtol);
    prof_end(st);
    NRE_CHECK_LAUNCH();
    if (rtol > 0.0 && (it + 1) % check_every == 0 && it + 1 < maxiter) {
      NRE_TRY_CUDA(cudaMemcpyAsync(m->cg_host.data(), sc, (size_t)B * SC_N * sizeof(double),
                                   cudaMemcpyDeviceToHost, st));
      NRE_TRY_CUDA(cudaStreamSynchronize(st));
      bool any = false;
      for (int i = 0; i < B; ++i) any |= m->cg_host[(size_t)i * SC_N + SC_ACTIVE] != 0.0;
      if (!any) break;
    }
  }
  NRE_TRY_CUDA(cudaMemcpyAsync(m->cg_host.data(), sc, (size_t)B * SC_N * sizeof(double),
                               cudaMemcpyDeviceToHost, st));
  NRE_TRY_CUDA(cudaStreamSynchronize(st));
  bool conv = true;
  for (int i = 0; i < B; ++i) {
    const double* c = &m->cg_host[(size_t)i * SC_N];
    const double rel = c[SC_BB] > 0 ? std::sqrt(c[SC_RR] / c[SC_BB]) : 0.0;
    if (iters_out) iters_out[i] = (int)c[SC_ITERS];
    if (relres_out) relres_out[i] = rel;
    if (rtol > 0.0 && rel > rtol) conv = false;
  }
  if (!conv) return set_error(NRE_ENOTCONV, "CG: some system missed rtol=%g within maxiter=%d", rtol, maxiter);
  return NRE_OK;
}

}  // namespace

extern "C" int cg_solve(nre_metric* m, const void* b, void* x, int batch, double rtol, int maxiter,
                        int* iters_out, double* relres_out, nre_stream_t stream) {
  clear_error();
  if (!m) return set_error(NRE_EINVAL, "metric must not be NULL");
  if (batch < 0 || batch > m->max_batch) return set_error(NRE_EINVAL, "batch %d outside [0, max_batch=%d]", batch, m->max_batch);
  if (maxiter < 0 || !(rtol >= 0.0)) return set_error(NRE_EINVAL, "maxiter must be >= 0 and rtol >= 0");
  if (batch == 0) return NRE_OK;
  if (!b || !x) return set_error(NRE_EINVAL, "NULL array argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (m->dtype == NRE_F64)
    return cg_t<double>(m, (const double*)b, (double*)x, batch, rtol, maxiter, iters_out, relres_out, st);
  return cg_t<float>(m, (const float*)b, (float*)x, batch, rtol, maxiter, iters_out, relres_out, st);
}
