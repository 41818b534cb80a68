// geoVI nonlinear update of sample residuals (Sec. "Variational Inference":
// geoVI, the successor of MGVI; the example's nonlinear sample update "SN", a
// Newton minimiser with xtol and maxiter = 5).
//
// Reading implemented here (the paper gives no formulas): with t the
// likelihood's standardising transform in data space (unit Fisher metric),
//     Gaussian (std sigma, mask m, response R):  t(cf) = sqrt(m) R(cf) / sigma,
//     Poisson (rate lambda = scale exp(cf)):     t(cf) = 2 sqrt(lambda),
// and J_p the Jacobian of xi -> t(cf(xi)) at the expansion point p
// (J_p^T J_p = J^T W J, the metric's likelihood part), a residual delta solves
//     F(delta) = delta + J_p^T [t(cf(p + delta)) - t(cf(p))] - b = 0,
// starting from the linear MGVI residual M_p^-1 b, by Newton iterations with
// M_p as the Jacobian: delta <- delta - M_p^-1 F(delta) (CG on the metric, with
// its preconditioner), until mean |step| <= xtol for every system or maxiter.
// Every evaluation of F is one batched cf_forward at p + delta, a pointwise
// kernel, one batched cf_vjp at p and a vector kernel.
#include <cmath>
#include <vector>

#include "metric_internal.cuh"

using namespace nre;

namespace {

constexpr int GV_THREADS = 256;

int gv_blocks(int64_t n) {
  int64_t nb = (n + GV_THREADS * 4 - 1) / (GV_THREADS * 4);
  if (nb > 128) nb = 128;
  return nb < 1 ? 1 : (int)nb;
}

// t(cf) and dt/dcf of the likelihood's standardising transform.
template <typename T>
__device__ __forceinline__ void std_transform(T c, int kind, int response, double sig_or_scale, T m, T* t, T* dt) {
  if (kind == NRE_LIK_POISSON) {
    const T sl = sqrt(T(sig_or_scale) * exp(c));  // sqrt(lambda)
    *t = T(2) * sl;
    *dt = sl;
  } else {
    const T is = T(1.0 / sig_or_scale) * sqrt(m);
    const T s = response == NRE_RESP_EXP ? exp(c) : c;
    *t = is * s;
    *dt = is * (response == NRE_RESP_EXP ? s : T(1));
  }
}

// t(cf_p) and dt/dcf at p.
template <typename T>
__global__ void k_gv_tp(const T* cfp, const T* mask, int64_t N, int kind, int response, double sig, T* tp, T* dtp) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (int64_t)gridDim.x * blockDim.x)
    std_transform<T>(cfp[x], kind, response, sig, mask ? mask[x] : T(1), &tp[x], &dtp[x]);
}

// y[b][x] = dt_p[x] (t(cf[b][x]) - t_p[x]).
template <typename T>
__global__ void k_gv_y(const T* cf, const T* tp, const T* dtp, const T* mask, int64_t N, int kind, int response,
                       double sig, T* y) {
  const int64_t off = (int64_t)blockIdx.y * N;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (int64_t)gridDim.x * blockDim.x) {
    T t, dt;
    std_transform<T>(cf[off + x], kind, response, sig, mask ? mask[x] : T(1), &t, &dt);
    y[off + x] = dtp[x] * (t - tp[x]);
  }
}

// out[b][i] = p[i] + d[b][i] (i < n), zero padding.
template <typename T>
__global__ void k_gv_shift(const T* p, const T* d, T* out, int64_t n, int64_t S) {
  const int64_t off = (int64_t)blockIdx.y * S;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (int64_t)gridDim.x * blockDim.x)
    out[off + i] = i < n ? T(p[i] + (d ? d[off + i] : T(0))) : T(0);
}

// F = delta + u - b on the latent entries (zero padding).
template <typename T>
__global__ void k_gv_F(const T* delta, const T* u, const T* b, T* F, int64_t n, int64_t S) {
  const int64_t off = (int64_t)blockIdx.y * S;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (int64_t)gridDim.x * blockDim.x)
    F[off + i] = i < n ? T(delta[off + i] + u[off + i] - b[off + i]) : T(0);
}

// delta -= step; per-block partials of |step|.
template <typename T>
__global__ void __launch_bounds__(GV_THREADS) k_gv_update(T* delta, const T* step, int64_t n, int64_t S,
                                                         double* part) {
  const int64_t off = (int64_t)blockIdx.y * S;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T s = step[off + i];
    delta[off + i] -= s;
    acc += fabs(double(s));
  }
  __shared__ double red[GV_THREADS / 32];
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

__global__ void k_gv_rows(const double* part, int nblk, int rows, double* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= rows) return;
  double s = 0.0;
  for (int i = 0; i < nblk; ++i) s += part[(int64_t)k * nblk + i];
  out[k] = s;
}

template <typename T>
int geovi_t(nre_metric* m, const T* b, T* delta, int B, double xtol, int maxiter, double cg_rtol, int cg_maxiter,
            int* iters_out, double* step_out, cudaStream_t st) {
  nre_cf_plan* p = m->cf;
  const int64_t N = p->N, n = m->latent, S = m->stride;
  const int nblk = gv_blocks(S);
  NRE_TRY(ensure(m->gv_pp, (size_t)B * S * sizeof(T)));
  NRE_TRY(ensure(m->gv_pts, (size_t)B * S * sizeof(T)));
  NRE_TRY(ensure(m->gv_u, (size_t)B * S * sizeof(T)));
  NRE_TRY(ensure(m->gv_F, (size_t)B * S * sizeof(T)));
  NRE_TRY(ensure(m->gv_step, (size_t)B * S * sizeof(T)));
  NRE_TRY(ensure(m->gv_cf, (size_t)B * N * sizeof(T)));
  NRE_TRY(ensure(m->gv_tp, (size_t)2 * N * sizeof(T)));
  NRE_TRY(ensure(m->gv_part, ((size_t)B * nblk + B) * sizeof(double)));
  const T* xp = m->xi_p.as<T>();
  T* pp = m->gv_pp.as<T>();
  T* pts = m->gv_pts.as<T>();
  T* u = m->gv_u.as<T>();
  T* F = m->gv_F.as<T>();
  T* step = m->gv_step.as<T>();
  T* cf = m->gv_cf.as<T>();
  T* tp = m->gv_tp.as<T>();
  T* dtp = tp + N;
  double* part = m->gv_part.as<double>();
  const T* mask = m->mask.p ? m->mask.as<T>() : nullptr;
  const int kind = m->lik.kind, resp = m->lik.response;
  const double sig = m->lik.sig_or_scale;
  const dim3 grid(nblk, B);
  // p replicated per system (the VJP's expansion points), cf(p), t(p), dt(p)
  prof_begin("geovi_setup", (double)B * S * sizeof(T), st);
  k_gv_shift<T><<<grid, GV_THREADS, 0, st>>>(xp, nullptr, pp, n, S);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  NRE_TRY(cf_forward(p, pp, cf, 1, (nre_stream_t)st));
  prof_begin("geovi_setup", (double)N * sizeof(T) * 3, st);
  k_gv_tp<T><<<gv_blocks(N), GV_THREADS, 0, st>>>(cf, mask, N, kind, resp, sig, tp, dtp);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  std::vector<double> h(B, 0.0);
  std::vector<int> conv_at(B, 0);  // first iteration whose step met xtol
  int it = 0;
  bool done = false;
  while (it < maxiter && !done) {
    prof_begin("geovi_shift", (double)B * S * sizeof(T) * 2, st);
    k_gv_shift<T><<<grid, GV_THREADS, 0, st>>>(xp, delta, pts, n, S);
    prof_end(st);
    NRE_CHECK_LAUNCH();
    NRE_TRY(cf_forward(p, pts, cf, B, (nre_stream_t)st));
    prof_begin("geovi_y", (double)B * N * sizeof(T) * 2 + 3.0 * N * sizeof(T), st);
    k_gv_y<T><<<dim3(gv_blocks(N), B), GV_THREADS, 0, st>>>(cf, tp, dtp, mask, N, kind, resp, sig, cf);
    prof_end(st);
    NRE_CHECK_LAUNCH();
    NRE_TRY(cf_vjp(p, pp, cf, u, B, (nre_stream_t)st));
    prof_begin("geovi_F", (double)B * S * sizeof(T) * 4, st);
    k_gv_F<T><<<grid, GV_THREADS, 0, st>>>(delta, u, b, F, n, S);
    prof_end(st);
    NRE_CHECK_LAUNCH();
    const int s = cg_solve(m, F, step, B, cg_rtol, cg_maxiter, nullptr, nullptr, (nre_stream_t)st);
    if (s != NRE_OK && s != NRE_ENOTCONV) return s;
    clear_error();
    prof_begin("geovi_update", (double)B * n * sizeof(T) * 3, st);
    k_gv_update<T><<<grid, GV_THREADS, 0, st>>>(delta, step, n, S, part);
    k_gv_rows<<<(B + 127) / 128, 128, 0, st>>>(part, nblk, B, part + (size_t)B * nblk);
    prof_end(st);
    NRE_CHECK_LAUNCH();
    NRE_TRY_CUDA(cudaMemcpyAsync(h.data(), part + (size_t)B * nblk, B * sizeof(double), cudaMemcpyDeviceToHost, st));
    NRE_TRY_CUDA(cudaStreamSynchronize(st));
    ++it;
    done = true;
    for (int i = 0; i < B; ++i) {
      h[i] /= (double)n;
      if (conv_at[i] == 0 && h[i] <= xtol) conv_at[i] = it;
      if (h[i] > xtol) done = false;
    }
  }
  if (iters_out)
    for (int i = 0; i < B; ++i) iters_out[i] = conv_at[i] ? conv_at[i] : it;
  if (step_out)
    for (int i = 0; i < B; ++i) step_out[i] = h[i];
  return NRE_OK;
}

}  // namespace

extern "C" int geovi_update(nre_metric* m, const void* b, void* delta, int batch, double xtol, int maxiter,
                            double cg_rtol, int cg_maxiter, int* iters_out, double* step_out, nre_stream_t stream) {
  clear_error();
  if (!m) return set_error(NRE_EINVAL, "metric must not be NULL");
  if (m->model_kind != NRE_MODEL_CF) return set_error(NRE_EINVAL, "geovi_update needs a correlated-field metric");
  if (batch < 0 || batch > m->max_batch) return set_error(NRE_EINVAL, "batch %d outside [0, max_batch=%d]", batch, m->max_batch);
  if (!(xtol >= 0.0) || maxiter < 0 || !(cg_rtol > 0.0) || cg_maxiter < 1)
    return set_error(NRE_EINVAL, "need xtol >= 0, maxiter >= 0, cg_rtol > 0, cg_maxiter >= 1");
  if (batch == 0 || maxiter == 0) return NRE_OK;
  if (!b || !delta) return set_error(NRE_EINVAL, "NULL array argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (m->dtype == NRE_F64)
    return geovi_t<double>(m, (const double*)b, (double*)delta, batch, xtol, maxiter, cg_rtol, cg_maxiter, iters_out,
                           step_out, st);
  return geovi_t<float>(m, (const float*)b, (float*)delta, batch, xtol, maxiter, cg_rtol, cg_maxiter, iters_out,
                        step_out, st);
}
