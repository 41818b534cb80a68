// Sample solves to a true (FP64) relative residual: residual correction
// (mixed-precision iterative refinement) around the batched CG.
//
// Sec. "Variational Inference": the linear sample draw solves M_p x = b by CG
// to a tolerance.  An FP32 solve stops on its recursive residual, and the true
// residual ||b - M x|| / ||b|| of its result is bounded below by the FP32
// operator's own error on x (about 1e-4 on the 2-D Poisson metrics).  Here x is
// kept in FP64 and corrected from FP64 residuals of an FP64 metric at the same
// expansion point:
//     x_0 = 0;  r_k = b - M64 x_k;  stop once ||r_k|| <= rtol ||b||;
//     solve M_lo d = r_k by CG to inner_rtol (recursive);  x_{k+1} = x_k + d.
// Each pass reduces the true residual by about max(inner_rtol, the low
// precision operator's relative error), so two or three passes reach 1e-5.
// The residual of x_0 = 0 is b itself (no product); every later pass costs one
// FP64 metric product.  Systems that have reached rtol are frozen (their
// right-hand side of the inner solve is zero, so d = 0).
#include <cmath>
#include <vector>

#include "metric_internal.cuh"

using namespace nre;

namespace {

constexpr int RF_THREADS = 256;

int rf_blocks(int64_t n) {
  int64_t nb = (n + RF_THREADS * 8 - 1) / (RF_THREADS * 8);
  if (nb > 64) nb = 64;
  return nb < 1 ? 1 : (int)nb;
}

// r = b - q (q == nullptr: r = b) over the latent entries of system
// blockIdx.y, and per-block partials of r.r and (bb != nullptr) b.b.
__global__ void __launch_bounds__(RF_THREADS) k_rf_residual(const double* b, const double* q, double* r, int64_t n,
                                                           int64_t S, double* rr_part, double* bb_part) {
  const int64_t off = (int64_t)blockIdx.y * S;
  double srr = 0.0, sbb = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double bv = b[off + i];
    const double rv = q ? bv - q[off + i] : bv;
    r[off + i] = rv;
    srr += rv * rv;
    sbb += bv * bv;
  }
  __shared__ double red[RF_THREADS / 32];
  const double t = block_sum(srr, red);
  if (threadIdx.x == 0) rr_part[blockIdx.y * gridDim.x + blockIdx.x] = t;
  if (bb_part) {
    const double u = block_sum(sbb, red);
    if (threadIdx.x == 0) bb_part[blockIdx.y * gridDim.x + blockIdx.x] = u;
  }
}

// Sums of the partials of each system, in block order.
__global__ void k_rf_sum(const double* part, int nblk, int B, double* out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double s = 0.0;
  for (int i = 0; i < nblk; ++i) s += part[b * nblk + i];
  out[b] = s;
}

// r_lo = T(r) for the systems still active (flag != 0), 0 for frozen ones.
template <typename T>
__global__ void k_rf_down(const double* r, T* rlo, int64_t n, int64_t S, const int* active) {
  const int64_t off = (int64_t)blockIdx.y * S;
  const bool act = active[blockIdx.y] != 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    rlo[off + i] = act ? T(r[off + i]) : T(0);
}

// x += double(d) (d of a frozen system is zero).
template <typename T>
__global__ void k_rf_up(double* x, const T* d, int64_t n, int64_t S) {
  const int64_t off = (int64_t)blockIdx.y * S;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[off + i] += double(d[off + i]);
}

// Workspaces of a pass: FP64 residual, product and sums in the FP64 metric,
// the low precision right-hand side and correction in the low one.
int rf_ensure(nre_metric* lo, nre_metric* hi, int B) {
  const int64_t S = hi->stride;
  const int nblk = rf_blocks(hi->latent);
  const size_t el = lo->dtype == NRE_F64 ? 8 : 4;
  NRE_TRY(ensure(hi->rf_r, (size_t)B * S * sizeof(double)));
  NRE_TRY(ensure(hi->rf_q, (size_t)B * S * sizeof(double)));
  NRE_TRY(ensure(hi->rf_part, ((size_t)2 * B * nblk + 2 * B) * sizeof(double) + (size_t)B * sizeof(int)));
  NRE_TRY(ensure(lo->rf_r, (size_t)B * S * el));
  NRE_TRY(ensure(lo->rf_q, (size_t)B * S * el));
  return NRE_OK;
}

template <typename T>
int refined_t(nre_metric* lo, nre_metric* hi, const double* b, double* x, int B, double rtol, int max_outer,
              double inner_rtol, int inner_maxiter, int* iters_out, double* relres_out, int* outer_out,
              cudaStream_t st) {
  const int64_t S = hi->stride;
  NRE_TRY(rf_ensure(lo, hi, B));
  T* rlo = lo->rf_r.as<T>();
  T* dlo = lo->rf_q.as<T>();
  NRE_TRY_CUDA(cudaMemsetAsync(x, 0, (size_t)B * S * sizeof(double), st));
  NRE_TRY_CUDA(cudaMemsetAsync(rlo, 0, (size_t)B * S * sizeof(T), st));  // padding stays zero
  std::vector<double> hs(2 * B);
  std::vector<int> act(B, 1), its(B, 0);
  int outer = 0;
  for (;; ++outer) {
    double* sums = nullptr;
    NRE_TRY(refine_residual(lo, hi, b, x, outer > 0 ? dlo : nullptr, B, outer == 0, &sums, st));
    NRE_TRY_CUDA(cudaMemcpyAsync(hs.data(), sums, 2 * B * sizeof(double), cudaMemcpyDeviceToHost, st));
    NRE_TRY_CUDA(cudaStreamSynchronize(st));
    bool any = false;
    for (int i = 0; i < B; ++i) {
      const double rel = hs[B + i] > 0 ? std::sqrt(hs[i] / hs[B + i]) : 0.0;
      if (relres_out) relres_out[i] = rel;
      act[i] = rel > rtol ? 1 : 0;
      any = any || act[i];
    }
    if (!any || outer == max_outer) break;
    NRE_TRY(refine_down(lo, hi, B, act.data(), nullptr, st));
    std::vector<int> inner(B, 0);
    const int s = cg_solve(lo, rlo, dlo, B, inner_rtol, inner_maxiter, inner.data(), nullptr, (nre_stream_t)st);
    if (s != NRE_OK && s != NRE_ENOTCONV) return s;
    for (int i = 0; i < B; ++i) its[i] += act[i] ? inner[i] : 0;
  }
  clear_error();
  if (iters_out)
    for (int i = 0; i < B; ++i) iters_out[i] = its[i];
  if (outer_out) *outer_out = outer;
  for (int i = 0; i < B; ++i)
    if (act[i])
      return set_error(NRE_ENOTCONV, "refined CG: some system missed rtol=%g after %d correction passes", rtol,
                       max_outer);
  return NRE_OK;
}

}  // namespace

namespace nre {
int refine_residual(nre_metric* lo, nre_metric* hi, const double* b, double* x, const void* d_lo, int B,
                    bool with_bb, double** sums_out, cudaStream_t st) {
  const int64_t n = hi->latent, S = hi->stride;
  const int nblk = rf_blocks(n);
  NRE_TRY(rf_ensure(lo, hi, B));
  double* r = hi->rf_r.as<double>();
  double* q = hi->rf_q.as<double>();
  double* rr_part = hi->rf_part.as<double>();
  double* bb_part = rr_part + (size_t)B * nblk;
  double* sums = bb_part + (size_t)B * nblk;  // [B] r.r, [B] b.b
  const dim3 grid(nblk, B);
  if (d_lo) {
    prof_begin("refine_update", (double)B * n * (16 + (lo->dtype == NRE_F64 ? 8 : 4)), st);
    if (lo->dtype == NRE_F64) k_rf_up<double><<<grid, RF_THREADS, 0, st>>>(x, (const double*)d_lo, n, S);
    else k_rf_up<float><<<grid, RF_THREADS, 0, st>>>(x, (const float*)d_lo, n, S);
    prof_end(st);
    NRE_CHECK_LAUNCH();
    NRE_TRY(metric_apply_impl(hi, x, q, B, st));
  }
  prof_begin("refine_residual", (double)B * n * (d_lo ? 24 : 16), st);
  k_rf_residual<<<grid, RF_THREADS, 0, st>>>(b, d_lo ? q : nullptr, r, n, S, rr_part, with_bb ? bb_part : nullptr);
  k_rf_sum<<<(B + 127) / 128, 128, 0, st>>>(rr_part, nblk, B, sums);
  if (with_bb) k_rf_sum<<<(B + 127) / 128, 128, 0, st>>>(bb_part, nblk, B, sums + B);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  if (sums_out) *sums_out = sums;
  return NRE_OK;
}

int refine_down(nre_metric* lo, nre_metric* hi, int B, const int* active_host, void** rlo_out, cudaStream_t st) {
  const int64_t n = hi->latent, S = hi->stride;
  const int nblk = rf_blocks(n);
  int* active = reinterpret_cast<int*>(hi->rf_part.as<double>() + (size_t)2 * B * nblk + 2 * B);
  NRE_TRY_CUDA(cudaMemcpyAsync(active, active_host, B * sizeof(int), cudaMemcpyHostToDevice, st));
  const dim3 grid(nblk, B);
  prof_begin("refine_down", (double)B * n * (8 + (lo->dtype == NRE_F64 ? 8 : 4)), st);
  if (lo->dtype == NRE_F64) k_rf_down<double><<<grid, RF_THREADS, 0, st>>>(hi->rf_r.as<double>(), lo->rf_r.as<double>(), n, S, active);
  else k_rf_down<float><<<grid, RF_THREADS, 0, st>>>(hi->rf_r.as<double>(), lo->rf_r.as<float>(), n, S, active);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  if (rlo_out) *rlo_out = lo->rf_r.p;
  return NRE_OK;
}
}  // namespace nre

extern "C" int cg_solve_refined(nre_metric* m_lo, nre_metric* m_hi, const void* b, void* x, int batch, double rtol,
                                int max_outer, double inner_rtol, int inner_maxiter, int* iters_out,
                                double* relres_out, int* outer_out, nre_stream_t stream) {
  clear_error();
  if (!m_lo || !m_hi) return set_error(NRE_EINVAL, "metrics must not be NULL");
  if (m_hi->dtype != NRE_F64) return set_error(NRE_EINVAL, "m_hi must be an FP64 metric");
  if (m_lo == m_hi) return set_error(NRE_EINVAL, "m_lo and m_hi must be different metric objects");
  if (m_lo->latent != m_hi->latent || m_lo->stride != m_hi->stride || m_lo->model_kind != m_hi->model_kind)
    return set_error(NRE_EINVAL, "m_lo and m_hi must have the same model and latent layout");
  if (batch < 0 || batch > m_lo->max_batch || batch > m_hi->max_batch)
    return set_error(NRE_EINVAL, "batch %d outside [0, max_batch of both metrics]", batch);
  if (max_outer < 0 || inner_maxiter < 0 || !(rtol > 0.0) || !(inner_rtol > 0.0) || !(inner_rtol < 1.0))
    return set_error(NRE_EINVAL, "need rtol > 0, 0 < inner_rtol < 1, max_outer >= 0, inner_maxiter >= 0");
  if (outer_out) *outer_out = 0;
  if (batch == 0) return NRE_OK;
  if (!b || !x) return set_error(NRE_EINVAL, "NULL array argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (m_lo->dtype == NRE_F64)
    return refined_t<double>(m_lo, m_hi, (const double*)b, (double*)x, batch, rtol, max_outer, inner_rtol,
                             inner_maxiter, iters_out, relres_out, outer_out, st);
  return refined_t<float>(m_lo, m_hi, (const double*)b, (double*)x, batch, rtol, max_outer, inner_rtol,
                          inner_maxiter, iters_out, relres_out, outer_out, st);
}
