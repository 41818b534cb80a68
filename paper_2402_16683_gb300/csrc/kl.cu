// KL minimisation of MGVI by Newton-CG (Sec. "Variational Inference": the KL
// minimiser "M" of the example, a Newton-CG with xtol and maxiter = 35).
//
// Reading implemented here (the paper gives no formulas):
//   samples xi_s = xi_bar + delta_s with fixed residual samples delta_s;
//   E(xi_bar) = (1/S) sum_s [ NLL(d | cf(xi_s)) + |xi_s|^2 / 2 ],
//     Poisson (rate lambda = scale exp(cf)): NLL = sum lambda - d ln lambda,
//     Gaussian (response R, mask m, std sigma): NLL = sum m (d - R(cf))^2 / (2 sigma^2);
//   grad E = (1/S) sum_s [ xi_s + J_s^T dNLL/dcf(xi_s) ];
//   curvature: Mbar = I + (1/S) sum_s J_s^T W_s J_s (Fisher weights W_s at xi_s);
//   Newton-CG: D = -Mbar^-1 grad E by CG, backtracking line search (alpha = 1,
//   halved while the energy does not decrease, at most 30 times), stop once
//   mean |alpha D| <= xtol or after maxiter iterations.
//
// Every point's model evaluation runs as one batch of the correlated-field
// kernels (batch index = sample s, per-sample expansion points, amplitude
// states and Fisher weights): cf_forward for the energy, cf_vjp for the
// gradient, and for Mbar v the fused metric sweeps with t = w_s * y per sample,
// followed by the average over the samples.
#include <cmath>
#include <vector>

#include "metric_internal.cuh"

using namespace nre;

struct nre_kl {
  nre_cf_plan* plan = nullptr;
  nre_lik lik;
  int S = 0, dtype = NRE_F32;
  int64_t N = 0, latent = 0, stride = 0;
  int nblk = 1;
  nre::DevBuf deltas, data, mask;   // [S][stride], [N], [N] or empty
  nre::DevBuf xbar, grad, dir, rhs, trial;  // [stride]
  nre::DevBuf pts, g, outs;         // [S][stride]
  nre::DevBuf cf, w, r, tmp0, tmp1; // [S][N]
  nre::DevBuf states, dA, part, bpix;
  // FP32 power / Matern model: per-sample amplitude Jacobians at the points
  // (G [S][nb][nhp], Gt [S][nh][nbp]), their scratch, and the complete bin
  // sums with their arrival counters
  bool lin = false;
  int64_t gstr = 0, gtstr = 0;
  nre::DevBuf G, Gt, eye, Jt, gsum, gcnt;
  nre::DevBuf red;                  // partials and per-sample sums
  double energy = 0.0;
  bool have_pos = false;
  nre_metric* metric = nullptr;     // model kind NRE_MODEL_KL, owned here
  ~nre_kl() { delete metric; }
};

namespace {

constexpr int KL_THREADS = 256;

// Four consecutive values as 16-byte vectors (two for double).
template <typename T>
__device__ __forceinline__ void ld4v(const T* p, T* o) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(p), c = *reinterpret_cast<const double2*>(p + 2);
    o[0] = a.x; o[1] = a.y; o[2] = c.x; o[3] = c.y;
  }
}
template <typename T>
__device__ __forceinline__ void st4v(T* p, const T* o) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(o[2], o[3]);
  }
}

int kl_blocks(int64_t n) {
  int64_t nb = (n + KL_THREADS * 4 - 1) / (KL_THREADS * 4);
  if (nb > 128) nb = 128;
  return nb < 1 ? 1 : (int)nb;
}

// out[s][i] = x[i] + d[s][i] (i < n), zero padding up to the stride.
template <typename T>
__global__ void k_kl_points(const T* x, const T* d, T* out, int64_t n, int64_t S) {
  const int64_t off = (int64_t)blockIdx.y * S;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (int64_t)gridDim.x * blockDim.x)
    out[off + i] = i < n ? T(x[i] + d[off + i]) : T(0);
}

// Pointwise likelihood terms at the model values cf[s][x]: per-block FP64
// partials of the NLL; with r / w also dNLL/dcf and the Fisher weight.
template <typename T>
__global__ void __launch_bounds__(KL_THREADS) k_kl_lik(const T* cf, const T* data, const T* mask, int64_t N,
                                                      int kind, int response, double sig_or_scale, T* r, T* w,
                                                      double* part) {
  // pointwise terms in the plan's precision (FP64 transcendentals are slow on
  // this part), their sum in FP64; ln(lambda) = ln(scale) + cf
  const int64_t off = (int64_t)blockIdx.y * N;
  const T lsc = T(log(sig_or_scale)), sc = T(sig_or_scale), inv = T(1.0 / (sig_or_scale * sig_or_scale));
  double acc = 0.0;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (int64_t)gridDim.x * blockDim.x) {
    const T c = cf[off + x], d = data[x];
    T nll, dn, fw;
    if (kind == NRE_LIK_POISSON) {
      const T lam = sc * exp(c);
      nll = lam - d * (lsc + c);
      dn = lam - d;
      fw = lam;
    } else {
      const T m = mask ? mask[x] : T(1);
      const T s = response == NRE_RESP_EXP ? exp(c) : c;
      const T ds = response == NRE_RESP_EXP ? s : T(1);
      const T res = d - s;
      nll = T(0.5) * m * res * res * inv;
      dn = -m * res * ds * inv;
      fw = m * ds * ds * inv;
    }
    acc += double(nll);
    if (r) r[off + x] = T(dn);
    if (w) w[off + x] = T(fw);
  }
  __shared__ double red[KL_THREADS / 32];
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// Per-block partials of |x_s|^2 over the n latent entries of each sample.
template <typename T>
__global__ void __launch_bounds__(KL_THREADS) k_kl_sq(const T* x, int64_t n, int64_t S, double* part) {
  const int64_t off = (int64_t)blockIdx.y * S;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = double(x[off + i]);
    acc += v * v;
  }
  __shared__ double red[KL_THREADS / 32];
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// out[k] = sum of part[k][0..nblk) in order (one thread per row k).
__global__ void k_kl_rows(const double* part, int nblk, int rows, double* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= rows) return;
  double s = 0.0;
  for (int i = 0; i < nblk; ++i) s += part[(int64_t)k * nblk + i];
  out[k] = s;
}

// out[i] = (1/S) sum_s (a[s][i] + (b ? b[s][i] : 0)) for i < n, in sample order
// (the sum times the rounded 1/S);
// zero padding up to the stride.
// Four consecutive entries per thread and round (the stride is a multiple of
// 64 entries, the arrays 16-byte aligned), so every load is a 16-byte vector.
template <typename T>
__global__ void k_kl_mean(const T* a, const T* b, T* out, int64_t n, int64_t stride, int S) {
  for (int64_t i0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x); i0 < stride;
       i0 += 4 * (int64_t)gridDim.x * blockDim.x) {
    // in the plan's precision, samples in order (FP64 conversions and
    // divisions are slow on this part)
    T s[4] = {T(0), T(0), T(0), T(0)};
    for (int k = 0; k < S; ++k) {
      T av[4], bv[4] = {T(0), T(0), T(0), T(0)};
      ld4v(a + (int64_t)k * stride + i0, av);
      if (b) ld4v(b + (int64_t)k * stride + i0, bv);
#pragma unroll
      for (int e = 0; e < 4; ++e) s[e] += av[e] + bv[e];
    }
    const T invS = T(1) / T(S);
    T o[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) o[e] = i0 + e < n ? s[e] * invS : T(0);
    st4v(out + i0, o);
  }
}

// y = x + alpha d (alpha_neg: y = -x); per-block partials of |d| (when part).
template <typename T>
__global__ void __launch_bounds__(KL_THREADS) k_kl_axpy(const T* x, const T* d, double alpha, T* y, int64_t n,
                                                       int64_t stride, double* part) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < stride; i += (int64_t)gridDim.x * blockDim.x) {
    if (i >= n) {
      y[i] = T(0);
      continue;
    }
    const double dv = d ? double(d[i]) : 0.0;
    y[i] = T(double(x[i]) + alpha * dv);
    acc += fabs(dv);
  }
  if (part) {
    __shared__ double red[KL_THREADS / 32];
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}

template <typename T>
AmpView<T> kl_view(const nre_kl* k) {
  const nre_cf_plan* p = k->plan;
  if (!binned_model(p)) return amp_view<T>(p, nullptr, 0);
  const int SS = amp_state_size(p->n_bins);
  AmpView<T> v = amp_view<T>(p, k->states.as<double>() + as_A(p->n_bins), SS);
  if (p->ndim >= 2) {
    // per-pixel bins, A from each sample's per-bin table (the register
    // sweeps stage it in shared memory; the generic sweeps read it directly)
    v.mode = AMPV_PIX;
    v.afull = nullptr;
    v.bpix = k->bpix.as<int16_t>();
  }
  return v;
}

// Energy at the points already in pts (model values into cf); with lin also
// r = dNLL/dcf and the Fisher weights w.  Returns the energy on the host.
template <typename T>
int kl_energy_pts(nre_kl* k, T* pts, T* cf, bool lin, double* energy, cudaStream_t st) {
  nre_cf_plan* p = k->plan;
  const int S = k->S, nblk = k->nblk;
  NRE_TRY(cf_forward(p, pts, cf, S, (nre_stream_t)st));
  double* part = k->red.as<double>();
  double* sums = part + (size_t)2 * S * nblk;
  const dim3 grid(nblk, S);
  prof_begin("kl_likelihood", (double)S * k->N * sizeof(T) * (lin ? 3 : 1), st);
  k_kl_lik<T><<<grid, KL_THREADS, 0, st>>>(cf, k->data.as<T>(), k->mask.p ? k->mask.as<T>() : nullptr, k->N,
                                           k->lik.kind, k->lik.response, k->lik.sig_or_scale,
                                           lin ? k->r.as<T>() : nullptr, lin ? k->w.as<T>() : nullptr, part);
  k_kl_sq<T><<<grid, KL_THREADS, 0, st>>>(pts, k->latent, k->stride, part + (size_t)S * nblk);
  k_kl_rows<<<(2 * S + 127) / 128, 128, 0, st>>>(part, nblk, 2 * S, sums);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  std::vector<double> h(2 * S);
  NRE_TRY_CUDA(cudaMemcpyAsync(h.data(), sums, 2 * S * sizeof(double), cudaMemcpyDeviceToHost, st));
  NRE_TRY_CUDA(cudaStreamSynchronize(st));
  double e = 0.0;
  for (int s = 0; s < S; ++s) e += h[s] + 0.5 * h[S + s];
  *energy = e / S;
  return NRE_OK;
}

template <typename T>
int kl_set_position_t(nre_kl* k, const T* xbar, cudaStream_t st) {
  nre_cf_plan* p = k->plan;
  const int S = k->S;
  const int64_t SZ = k->stride;
  if (xbar != k->xbar.as<T>())
    NRE_TRY_CUDA(cudaMemcpyAsync(k->xbar.p, xbar, SZ * sizeof(T), cudaMemcpyDeviceToDevice, st));
  T* pts = k->pts.as<T>();
  prof_begin("kl_points", (double)S * SZ * sizeof(T) * 2, st);
  k_kl_points<T><<<dim3(k->nblk, S), KL_THREADS, 0, st>>>(k->xbar.as<T>(), k->deltas.as<T>(), pts, k->latent, SZ);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  NRE_TRY(kl_energy_pts<T>(k, pts, k->cf.as<T>(), true, &k->energy, st));
  // gradient: (1/S) sum_s (xi_s + J_s^T r_s)
  NRE_TRY(cf_vjp(p, pts, k->r.p, k->g.p, S, (nre_stream_t)st));
  prof_begin("kl_mean", (double)S * SZ * sizeof(T) * 2, st);
  k_kl_mean<T><<<304, 256, 0, st>>>(pts, k->g.as<T>(), k->grad.as<T>(), k->latent, SZ, S);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  // amplitude states of the points for the metric
  if (binned_model(p)) NRE_TRY(amp_forward<T>(amp_prior_of(p), pts + k->N, SZ, k->states.as<double>(), S, st));
  if (k->lin) {
    // FP32: each point's amplitude Jacobian, formed from FP64 JVPs
    const int SS = amp_state_size(p->n_bins);
    for (int s = 0; s < S; ++s)
      NRE_TRY(amp_jacobian<T>(amp_prior_of(p), k->states.as<double>() + (int64_t)s * SS, p->n_hyper, k->eye.as<T>(),
                              k->Jt.as<double>(), k->G.as<float>() + s * k->gstr, k->Gt.as<float>() + s * k->gtstr,
                              st));
  }
  k->have_pos = true;
  return NRE_OK;
}

int kl_set_position_impl(nre_kl* k, const void* xbar, cudaStream_t st) {
  if (k->dtype == NRE_F64) return kl_set_position_t<double>(k, (const double*)xbar, st);
  return kl_set_position_t<float>(k, (const float*)xbar, st);
}

// Mbar v for one vector (the metric object's batch is 1).
template <typename T>
int kl_metric_apply_t(nre_kl* k, const T* v, T* out, cudaStream_t st) {
  nre_cf_plan* p = k->plan;
  const int S = k->S, nb = p->n_bins;
  const int64_t N = k->N, SZ = k->stride;
  const bool model = binned_model(p);
  const int SS = model ? amp_state_size(nb) : 0;
  const AmpPrior pr = model ? amp_prior_of(p) : AmpPrior{};
  const int nh = model ? p->n_hyper : 0;
  if (k->lin)  // also zeroes the in-place bin sums of the epilogue
    NRE_TRY(amp_jvp_lin<T>(k->G.as<float>(), nb, nh, v + N, 0, k->dA.as<double>(), S, st, k->gsum.as<double>(),
                           k->gstr));
  else if (model)
    NRE_TRY(amp_jvp<T>(pr, k->states.as<double>(), SS, v + N, 0, k->dA.as<double>(), S, st));
  T* pts = k->pts.as<T>();
  Pro<T> pro{};
  pro.mode = PRO_AMP;
  pro.x = v;
  pro.xs = 0;  // every point applies to the same v
  pro.av = kl_view<T>(k);
  Epi<T> epi{};
  epi.mode = EPI_AMP;
  epi.y = k->outs.as<T>();
  epi.ys = SZ;
  epi.base = v;
  epi.bs = 0;
  epi.av = pro.av;
  if (model) {
    pro.dA = k->dA.as<double>();
    pro.nb = nb;
    pro.xi_p = pts;
    pro.ps = SZ;
    epi.bins = 1;
    epi.xi_p = pts;
    epi.ps = SZ;
    if (k->lin) {
      epi.gsum = k->gsum.as<double>();
      epi.gcnt = k->gcnt.as<unsigned>();
    }
  }
  Mid<T> mid{k->w.as<T>(), N};
  int np = 0;
  NRE_TRY(run_hartley<T>(p, S, pro, epi, &mid, k->tmp0.as<T>(), k->tmp1.as<T>(),
                         model ? k->part.as<double>() : nullptr, &np, st));
  if (k->lin)
    NRE_TRY(amp_vjp_lin<T>(k->Gt.as<float>(), nb, nh, k->gsum.as<double>(), v + N, 0, k->outs.as<T>() + N, SZ, S, st,
                           nullptr, k->gtstr));
  else if (model)
    NRE_TRY(amp_vjp<T>(pr, k->states.as<double>(), SS, k->part.as<double>(), np, v + N, 0, k->outs.as<T>() + N,
                       SZ, S, st));
  prof_begin("kl_mean", (double)S * SZ * sizeof(T), st);
  k_kl_mean<T><<<304, 256, 0, st>>>(k->outs.as<T>(), nullptr, out, k->latent, SZ, S);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  return NRE_OK;
}

template <typename T>
int kl_newton_t(nre_kl* k, double cg_rtol, int cg_maxiter, double* step, double* energy, int* cg_iters,
                cudaStream_t st) {
  const int64_t n = k->latent, SZ = k->stride;
  const int nb1 = kl_blocks(SZ);
  double* part = k->red.as<double>();
  T* dir = k->dir.as<T>();
  T* rhs = k->rhs.as<T>();
  T* trial = k->trial.as<T>();
  // rhs = -grad, dir = Mbar^-1 rhs
  k_kl_axpy<T><<<nb1, KL_THREADS, 0, st>>>(k->grad.as<T>(), k->grad.as<T>(), -2.0, rhs, n, SZ, nullptr);
  NRE_CHECK_LAUNCH();
  int its = 0;
  double rel = 0.0;
  const int s = cg_solve(k->metric, rhs, dir, 1, cg_rtol, cg_maxiter, &its, &rel, (nre_stream_t)st);
  if (s != NRE_OK && s != NRE_ENOTCONV) return s;
  clear_error();
  if (cg_iters) *cg_iters = its;
  // |D|_1 for the step size
  k_kl_axpy<T><<<nb1, KL_THREADS, 0, st>>>(k->xbar.as<T>(), dir, 0.0, trial, n, SZ, part);
  NRE_CHECK_LAUNCH();
  k_kl_rows<<<1, 32, 0, st>>>(part, nb1, 1, part + nb1);
  double l1 = 0.0;
  NRE_TRY_CUDA(cudaMemcpyAsync(&l1, part + nb1, sizeof(double), cudaMemcpyDeviceToHost, st));
  NRE_TRY_CUDA(cudaStreamSynchronize(st));
  const double e0 = k->energy;
  double alpha = 1.0;
  for (int ls = 0; ls <= 30; ++ls, alpha *= 0.5) {
    k_kl_axpy<T><<<nb1, KL_THREADS, 0, st>>>(k->xbar.as<T>(), dir, alpha, trial, n, SZ, nullptr);
    k_kl_points<T><<<dim3(k->nblk, k->S), KL_THREADS, 0, st>>>(trial, k->deltas.as<T>(), k->g.as<T>(), n, SZ);
    NRE_CHECK_LAUNCH();
    double e1 = 0.0;
    NRE_TRY(kl_energy_pts<T>(k, k->g.as<T>(), k->tmp0.as<T>(), false, &e1, st));
    if (e1 <= e0) {
      NRE_TRY(kl_set_position_t<T>(k, trial, st));
      *step = alpha * l1 / (double)n;
      *energy = k->energy;
      return NRE_OK;
    }
  }
  *step = 0.0;  // no decrease along the direction: the position stays
  *energy = e0;
  return NRE_OK;
}

int kl_check(const nre_kl* k) {
  if (!k) return set_error(NRE_EINVAL, "kl must not be NULL");
  if (!k->have_pos) return set_error(NRE_EINVAL, "kl_set_position must be called first");
  return NRE_OK;
}

}  // namespace

namespace nre {
int kl_metric_apply(nre_kl* k, const void* v, void* out, int batch, cudaStream_t st) {
  if (!k->have_pos) return set_error(NRE_EINVAL, "the KL metric needs a position (kl_set_position)");
  for (int b = 0; b < batch; ++b) {
    if (k->dtype == NRE_F64)
      NRE_TRY(kl_metric_apply_t<double>(k, (const double*)v + b * k->stride, (double*)out + b * k->stride, st));
    else
      NRE_TRY(kl_metric_apply_t<float>(k, (const float*)v + b * k->stride, (float*)out + b * k->stride, st));
  }
  return NRE_OK;
}
}  // namespace nre

extern "C" {

int kl_create(nre_kl** out, nre_cf_plan* plan, const nre_lik* lik, const double* data, int64_t n_data,
              const void* deltas, int n_samples, nre_stream_t stream) {
  clear_error();
  if (!out || !plan || !lik || !data || !deltas) return set_error(NRE_EINVAL, "NULL argument");
  *out = nullptr;
  if (n_samples < 1 || n_samples > 1024) return set_error(NRE_EINVAL, "n_samples must be in [1, 1024]");
  if (n_data != plan->N) return set_error(NRE_EINVAL, "n_data %lld must equal the grid's N %lld",
                                          (long long)n_data, (long long)plan->N);
  if (!lik->mask.empty() && (int64_t)lik->mask.size() != plan->N)
    return set_error(NRE_EINVAL, "the likelihood mask must cover the grid");
  cudaStream_t st = (cudaStream_t)stream;
  nre_kl* k = new nre_kl();
  auto fail = [&](int code) {
    delete k;
    return code;
  };
  k->plan = plan;
  k->lik = *lik;
  k->S = n_samples;
  k->dtype = plan->dtype;
  k->N = plan->N;
  k->latent = plan->latent;
  k->stride = plan->stride;
  k->nblk = kl_blocks(k->stride);
  const size_t es = plan->dtype == NRE_F64 ? 8 : 4;
  const int S = n_samples;
  const int64_t SZ = k->stride, N = k->N;
  int s;
  for (nre::DevBuf* b : {&k->xbar, &k->grad, &k->dir, &k->rhs, &k->trial})
    if ((s = b->alloc(SZ * es)) != NRE_OK) return fail(s);
  for (nre::DevBuf* b : {&k->deltas, &k->pts, &k->g, &k->outs})
    if ((s = b->alloc((size_t)S * SZ * es)) != NRE_OK) return fail(s);
  for (nre::DevBuf* b : {&k->cf, &k->w, &k->r, &k->tmp0, &k->tmp1})
    if ((s = b->alloc((size_t)S * N * es)) != NRE_OK) return fail(s);
  if ((s = k->red.alloc(((size_t)2 * S * k->nblk + 2 * S + 2 * 128 + 8) * sizeof(double))) != NRE_OK) return fail(s);
  cudaError_t e = cudaMemcpyAsync(k->deltas.p, deltas, (size_t)S * SZ * es, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return fail(set_error(NRE_ECUDA, "copy of the residual samples failed: %s", cudaGetErrorString(e)));
  if (plan->dtype == NRE_F64) {
    if ((s = k->data.upload(data, N * sizeof(double))) != NRE_OK) return fail(s);
    if (!lik->mask.empty() && (s = k->mask.upload(lik->mask.data(), N * sizeof(double))) != NRE_OK) return fail(s);
  } else {
    std::vector<float> d(data, data + N);
    if ((s = k->data.upload(d.data(), N * sizeof(float))) != NRE_OK) return fail(s);
    if (!lik->mask.empty()) {
      std::vector<float> mk(lik->mask.begin(), lik->mask.end());
      if ((s = k->mask.upload(mk.data(), N * sizeof(float))) != NRE_OK) return fail(s);
    }
  }
  if (binned_model(plan)) {
    const int nb = plan->n_bins;
    if ((s = k->states.alloc((size_t)S * amp_state_size(nb) * sizeof(double))) != NRE_OK) return fail(s);
    if ((s = k->dA.alloc((size_t)S * nb * sizeof(double))) != NRE_OK) return fail(s);
    if ((s = k->part.alloc((size_t)S * max_parts(plan) * nb * sizeof(double))) != NRE_OK) return fail(s);
    const int nh = plan->n_hyper;
    if (plan->dtype == NRE_F32 && nh <= 1024) {
      k->lin = true;
      k->gstr = (int64_t)nb * ((nh + 3) & ~3);
      k->gtstr = (int64_t)nh * ((nb + 3) & ~3);
      if ((s = k->G.alloc((size_t)S * k->gstr * sizeof(float))) != NRE_OK ||
          (s = k->Gt.alloc((size_t)S * k->gtstr * sizeof(float))) != NRE_OK ||
          (s = k->eye.alloc((size_t)nh * nh * sizeof(float))) != NRE_OK ||
          (s = k->Jt.alloc((size_t)nh * nb * sizeof(double))) != NRE_OK ||
          (s = k->gsum.alloc((size_t)S * nb * sizeof(double))) != NRE_OK ||
          (s = k->gcnt.alloc((size_t)S * kGcntStride * sizeof(unsigned))) != NRE_OK)
        return fail(s);
      // the sweeps leave the arrival counters zero
      e = cudaMemsetAsync(k->gcnt.p, 0, (size_t)S * kGcntStride * sizeof(unsigned), st);
      if (e != cudaSuccess) return fail(set_error(NRE_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e)));
    }
    // per-pixel bins (-1 at k = 0) for the register sweeps' tables
    std::vector<int64_t> shp(plan->ndim);
    std::vector<double> sp(plan->ndim);
    for (int d = 0; d < plan->ndim; ++d) {
      shp[d] = plan->n[d];
      sp[d] = 1.0 / plan->n[d];
    }
    std::vector<int32_t> b32(N);
    if ((s = cf_bin_map(plan->ndim, shp.data(), sp.data(), nb, b32.data())) != NRE_OK) return fail(s);
    std::vector<int16_t> b16(b32.begin(), b32.end());
    if ((s = k->bpix.upload(b16.data(), N * sizeof(int16_t))) != NRE_OK) return fail(s);
  }
  // the averaged metric as a metric object (cg_solve, metric_apply)
  nre_metric* m = new nre_metric();
  m->model_kind = NRE_MODEL_KL;
  m->cf = nullptr;
  m->kl = k;
  m->dtype = plan->dtype;
  m->max_batch = 1;
  m->n_data = N;
  m->latent = k->latent;
  m->stride = k->stride;
  m->lik = *lik;
  k->metric = m;
  *out = k;
  return NRE_OK;
}

int kl_destroy(nre_kl* k) {
  delete k;
  return NRE_OK;
}

int kl_set_position(nre_kl* k, const void* xi_bar, double* energy, nre_stream_t stream) {
  clear_error();
  if (!k || !xi_bar) return set_error(NRE_EINVAL, "NULL argument");
  NRE_TRY(kl_set_position_impl(k, xi_bar, (cudaStream_t)stream));
  if (energy) *energy = k->energy;
  return NRE_OK;
}

int kl_energy_gradient(nre_kl* k, double* energy, void* grad, nre_stream_t stream) {
  clear_error();
  NRE_TRY(kl_check(k));
  if (energy) *energy = k->energy;
  if (grad) {
    const size_t es = k->dtype == NRE_F64 ? 8 : 4;
    NRE_TRY_CUDA(cudaMemcpyAsync(grad, k->grad.p, k->stride * es, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  }
  return NRE_OK;
}

int kl_energy_at(nre_kl* k, const void* xi, double* energy, nre_stream_t stream) {
  clear_error();
  if (!k || !xi || !energy) return set_error(NRE_EINVAL, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  const dim3 grid(k->nblk, k->S);
  if (k->dtype == NRE_F64) {
    k_kl_points<double><<<grid, KL_THREADS, 0, st>>>((const double*)xi, k->deltas.as<double>(), k->g.as<double>(),
                                                     k->latent, k->stride);
    NRE_CHECK_LAUNCH();
    return kl_energy_pts<double>(k, k->g.as<double>(), k->tmp0.as<double>(), false, energy, st);
  }
  k_kl_points<float><<<grid, KL_THREADS, 0, st>>>((const float*)xi, k->deltas.as<float>(), k->g.as<float>(), k->latent,
                                                  k->stride);
  NRE_CHECK_LAUNCH();
  return kl_energy_pts<float>(k, k->g.as<float>(), k->tmp0.as<float>(), false, energy, st);
}

int kl_metric(nre_kl* k, nre_metric** metric) {
  clear_error();
  if (!k || !metric) return set_error(NRE_EINVAL, "NULL argument");
  *metric = k->metric;
  return NRE_OK;
}

int kl_position(nre_kl* k, void* xi_bar, nre_stream_t stream) {
  clear_error();
  NRE_TRY(kl_check(k));
  if (!xi_bar) return set_error(NRE_EINVAL, "NULL argument");
  const size_t es = k->dtype == NRE_F64 ? 8 : 4;
  NRE_TRY_CUDA(cudaMemcpyAsync(xi_bar, k->xbar.p, k->stride * es, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return NRE_OK;
}

int kl_newton_step(nre_kl* k, double cg_rtol, int cg_maxiter, double* mean_abs_step, double* energy,
                   int* cg_iters, nre_stream_t stream) {
  clear_error();
  NRE_TRY(kl_check(k));
  if (!(cg_rtol > 0.0) || cg_maxiter < 1) return set_error(NRE_EINVAL, "need cg_rtol > 0 and cg_maxiter >= 1");
  double step = 0.0, e = 0.0;
  const cudaStream_t st = (cudaStream_t)stream;
  if (k->dtype == NRE_F64) NRE_TRY(kl_newton_t<double>(k, cg_rtol, cg_maxiter, &step, &e, cg_iters, st));
  else NRE_TRY(kl_newton_t<float>(k, cg_rtol, cg_maxiter, &step, &e, cg_iters, st));
  if (mean_abs_step) *mean_abs_step = step;
  if (energy) *energy = e;
  return NRE_OK;
}

int kl_minimize(nre_kl* k, double xtol, int maxiter, double cg_rtol, int cg_maxiter, int* iters, double* energy,
                nre_stream_t stream) {
  clear_error();
  NRE_TRY(kl_check(k));
  if (!(xtol >= 0.0) || maxiter < 0) return set_error(NRE_EINVAL, "need xtol >= 0 and maxiter >= 0");
  int it = 0;
  double e = k->energy;
  while (it < maxiter) {
    double step = 0.0;
    NRE_TRY(kl_newton_step(k, cg_rtol, cg_maxiter, &step, &e, nullptr, stream));
    ++it;
    if (step <= xtol) break;
  }
  if (iters) *iters = it;
  if (energy) *energy = e;
  return NRE_OK;
}

}  // extern "C"
