// Likelihood weights, the metric M_p = J^T N^-1 J + 1 and the MGVI right-hand
// side for the correlated field.
//
// Sec. "Performance": the benchmarked operator is M_p := F_p + 1 with
// F_p = J^T N^-1 J (N^-1 the Fisher metric of the Poisson likelihood).  With the
// response Jacobian folded into a per-pixel weight w (likelihood.h comments in
// nre.h) one application is
//     u = A * v_field + dA(v_hyper) * xi_p      (harmonic prologue)
//     y = H u,  t = w * y,  r = H t             (two Hartley transforms)
//     out_field = v_field + A * r,
//     out_hyper = v_hyper + VJP_amp(sum_{k in bin} xi_p[k] r[k]).
// Sec. "Variational Inference": an MGVI right-hand side with covariance M_p is
// b = xi' + J^T (sqrt(w) * eta).
#include <cmath>
#include <cstring>

#include "metric_internal.cuh"

using namespace nre;

namespace {

// Per-pixel amplitude and bin of the expansion point (power model).
template <typename T>
__global__ void k_pix_tables(AmpView<T> av, T* apix, int16_t* bpix, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int bn = av.bin(i);
    apix[i] = av.amp(0, i, bn);
    bpix[i] = (int16_t)bn;
  }
}

}  // namespace

namespace nre {
template <typename T>
AmpView<T> metric_view(const nre_metric* m) {
  const nre_cf_plan* p = m->cf;
  if (!binned_model(p)) return amp_view<T>(p, nullptr, 0);
  AmpView<T> v = amp_view<T>(p, m->state.as<double>() + as_A(p->n_bins), 0);
  v.mode = AMPV_PIX;
  v.afull = m->apix.as<T>();
  v.bpix = m->bpix.as<int16_t>();
  return v;
}
template AmpView<float> metric_view<float>(const nre_metric*);
template AmpView<double> metric_view<double>(const nre_metric*);
}  // namespace nre

namespace {

template <typename T>
int cf_metric_setup(nre_metric* m, const void* xi_p_in, cudaStream_t st) {
  nre_cf_plan* p = m->cf;
  const int64_t N = p->N;
  if (!m->side && p->ndim >= 2 && m->max_batch >= 2) {
    // the second stream of split products (created here, outside any capture)
    // with the priority of the stream the metric is created on (serving gives
    // small requests higher priority)
    int prio = 0;
    if (cudaStreamGetPriority(st, &prio) != cudaSuccess) {
      cudaGetLastError();
      prio = 0;
    }
    NRE_TRY_CUDA(cudaStreamCreateWithPriority(&m->side, cudaStreamNonBlocking, prio));
    NRE_TRY_CUDA(cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming));
    NRE_TRY_CUDA(cudaEventCreateWithFlags(&m->ev_join, cudaEventDisableTiming));
  }
  NRE_TRY(ensure(m->xi_p, p->stride * sizeof(T)));
  NRE_TRY_CUDA(cudaMemcpyAsync(m->xi_p.p, xi_p_in, p->latent * sizeof(T), cudaMemcpyDeviceToDevice, st));
  NRE_TRY(ensure(m->w, N * sizeof(T)));
  if (!m->lik.mask.empty()) {
    if (!m->mask.p) {
      std::vector<T> mk(m->lik.mask.begin(), m->lik.mask.end());
      NRE_TRY(m->mask.upload(mk.data(), mk.size() * sizeof(T)));
    }
  }
  NRE_TRY(ensure(m->tmp0, (size_t)m->max_batch * N * sizeof(T)));
  NRE_TRY(ensure(m->tmp1, (size_t)m->max_batch * N * sizeof(T)));
  const T* xp = m->xi_p.as<T>();
  Pro<T> pro{};
  pro.mode = PRO_AMP;
  pro.x = xp;
  pro.xs = 0;
  Epi<T> epi{};
  epi.mode = EPI_WEIGHT;
  epi.y = m->w.as<T>();
  epi.ys = 0;
  epi.offset = p->offset_mean;
  epi.lik_kind = m->lik.kind;
  epi.response = m->lik.response;
  epi.sig_or_scale = m->lik.sig_or_scale;
  epi.mask = m->mask.p ? m->mask.as<T>() : nullptr;
  if (binned_model(p)) {
    const int nb = p->n_bins;
    NRE_TRY(ensure(m->state, amp_state_size(nb) * sizeof(double)));
    NRE_TRY(ensure(m->dA, (size_t)m->max_batch * nb * sizeof(double)));
    NRE_TRY(ensure(m->part, (size_t)m->max_batch * max_parts(p) * nb * sizeof(double)));
    NRE_TRY(amp_forward<T>(amp_prior_of(p), xp + N, 0, m->state.as<double>(), 1, st));
    if (sizeof(T) == 4 && p->n_hyper <= 1024) {
      // FP32 products: the amplitude JVP / VJP become products with the
      // Jacobian at xi_p, formed once here from FP64 JVPs
      const int nh = p->n_hyper;
      // rows padded to multiples of four floats
      NRE_TRY(ensure(m->amp_G, (size_t)nb * ((nh + 3) & ~3) * sizeof(float)));
      NRE_TRY(ensure(m->amp_Gt, (size_t)nh * ((nb + 3) & ~3) * sizeof(float)));
      NRE_TRY(ensure(m->amp_eye, (size_t)nh * nh * sizeof(T)));
      NRE_TRY(ensure(m->amp_Jt, (size_t)nh * nb * sizeof(double)));
      NRE_TRY(ensure(m->gsum, (size_t)m->max_batch * nb * sizeof(double)));
      const size_t cnt = (size_t)m->max_batch * kGcntStride * sizeof(unsigned);
      if (m->gcnt.bytes < cnt) {
        NRE_TRY(ensure(m->gcnt, cnt));
        NRE_TRY_CUDA(cudaMemsetAsync(m->gcnt.p, 0, cnt, st));  // the sweeps leave them zero
      }
      NRE_TRY(amp_jacobian<T>(amp_prior_of(p), m->state.as<double>(), nh, m->amp_eye.as<T>(),
                              m->amp_Jt.as<double>(), m->amp_G.as<float>(), m->amp_Gt.as<float>(), st));
      m->amp_lin = true;
    }
    pro.av = amp_view<T>(p, m->state.as<double>() + as_A(nb), 0);
    NRE_TRY(ensure(m->apix, N * sizeof(T)));
    NRE_TRY(ensure(m->bpix, N * sizeof(int16_t)));
    prof_begin("pix_tables", (double)N * (sizeof(T) + 2), st);
    k_pix_tables<T><<<304, 256, 0, st>>>(pro.av, m->apix.as<T>(), m->bpix.as<int16_t>(), N);
    prof_end(st);
    NRE_CHECK_LAUNCH();
  } else {
    pro.av = amp_view<T>(p, nullptr, 0);
  }
  int np = 0;
  return run_hartley<T>(p, 1, pro, epi, nullptr, m->tmp0.as<T>(), m->tmp1.as<T>(), nullptr, &np, st);
}

template <typename T>
int cf_metric_apply(nre_metric* m, const T* v, T* out, int B, cudaStream_t st, double* dot,
                    bool hyper_in_cg) {
  nre_cf_plan* p = m->cf;
  const int64_t N = p->N, S = p->stride;
  const T* xp = m->xi_p.as<T>();
  Pro<T> pro{};
  pro.mode = PRO_AMP;
  pro.x = v;
  pro.xs = S;
  Epi<T> epi{};
  epi.mode = EPI_AMP;
  epi.y = out;
  epi.ys = S;
  epi.base = v;
  epi.bs = S;
  epi.dot = dot;
  Mid<T> mid{m->w.as<T>()};
  const bool model = binned_model(p);
  const int nb = p->n_bins;
  const AmpPrior pr = model ? amp_prior_of(p) : AmpPrior{};
  hyper_in_cg = hyper_in_cg && model && m->amp_lin;
  if (model) {
    if (hyper_in_cg)
      ;  // dA of v formed and gsum zeroed by the CG kernels
    else if (m->amp_lin)  // also zeroes the in-place bin sums of the last sweep
      NRE_TRY(amp_jvp_lin<T>(m->amp_G.as<float>(), nb, p->n_hyper, v + N, S, m->dA.as<double>(), B, st,
                             m->gsum.as<double>()));
    else
      NRE_TRY(amp_jvp<T>(pr, m->state.as<double>(), 0, v + N, S, m->dA.as<double>(), B, st));
    pro.av = metric_view<T>(m);
    pro.dA = m->dA.as<double>();
    pro.nb = nb;
    pro.xi_p = xp;
    pro.ps = 0;
    epi.av = pro.av;
    epi.bins = 1;
    epi.xi_p = xp;
    epi.ps = 0;
    if (m->amp_lin) {
      epi.gsum = m->gsum.as<double>();
      epi.gcnt = m->gcnt.as<unsigned>();
    }
  } else {
    pro.av = amp_view<T>(p, nullptr, 0);
    epi.av = pro.av;
  }
  int np = 0;
  // Two half batches on two streams: the persistent sweeps of one half fill
  // the SMs that the other half's last rounds leave idle (a sweep's units
  // rarely divide evenly over its resident CTAs).  Grids and fused partials
  // are per sample, so each half is the same computation on its own samples.
  // Needs per-sample bin sums (gsum) or none; not while launches are traced.
  const bool split = m->side && B >= 2 && p->ndim >= 2 && (!model || m->amp_lin) && !prof_tracing();
  if (!split) {
    NRE_TRY(run_hartley<T>(p, B, pro, epi, &mid, m->tmp0.as<T>(), m->tmp1.as<T>(),
                           model ? m->part.as<double>() : nullptr, &np, st));
  } else {
    NRE_TRY_CUDA(cudaEventRecord(m->ev_fork, st));
    NRE_TRY_CUDA(cudaStreamWaitEvent(m->side, m->ev_fork, 0));
    const int B0 = (B + 1) / 2;
    for (int h = 0; h < 2; ++h) {
      const int b0 = h ? B0 : 0, Bh = h ? B - B0 : B0;
      Pro<T> ph = pro;
      Epi<T> eh = epi;
      ph.x += (int64_t)b0 * pro.xs;
      if (ph.dA) ph.dA += (int64_t)b0 * nb;
      if (ph.ps) ph.xi_p += (int64_t)b0 * ph.ps;
      eh.y += (int64_t)b0 * epi.ys;
      if (eh.base) eh.base += (int64_t)b0 * epi.bs;
      if (eh.ps) eh.xi_p += (int64_t)b0 * eh.ps;
      if (eh.gsum) {
        eh.gsum += (int64_t)b0 * nb;
        eh.gcnt += (int64_t)b0 * kGcntStride;
      }
      if (eh.dot) eh.dot += (int64_t)b0 * kDotStride;
      // each half's CTA partials in its own slab of the partials buffer
      double* hpart = model ? m->part.as<double>() + (int64_t)b0 * max_parts(p) * nb : nullptr;
      NRE_TRY(run_hartley<T>(p, Bh, ph, eh, &mid, m->tmp0.as<T>() + (int64_t)b0 * N,
                             m->tmp1.as<T>() + (int64_t)b0 * N, hpart, &np, h ? m->side : st));
    }
    NRE_TRY_CUDA(cudaEventRecord(m->ev_join, m->side));
    NRE_TRY_CUDA(cudaStreamWaitEvent(st, m->ev_join, 0));
  }
  if (model && !hyper_in_cg) {
    if (m->amp_lin)  // the bin sums are complete in gsum (one "partial")
      NRE_TRY(amp_vjp_lin<T>(m->amp_Gt.as<float>(), nb, p->n_hyper, m->gsum.as<double>(), v + N, S, out + N,
                             S, B, st, dot));
    else
      NRE_TRY(amp_vjp<T>(pr, m->state.as<double>(), 0, m->part.as<double>(), np, v + N, S, out + N, S,
                         B, st, dot));
  }
  return NRE_OK;
}

template <typename T>
int cf_mgvi_rhs(nre_metric* m, const T* xi_prime, const T* eta, T* b, int B, cudaStream_t st) {
  nre_cf_plan* p = m->cf;
  const int64_t N = p->N, S = p->stride;
  const T* xp = m->xi_p.as<T>();
  Pro<T> pro{};
  pro.mode = PRO_SQRTW;
  pro.x = eta;
  pro.xs = N;
  pro.w = m->w.as<T>();
  Epi<T> epi{};
  epi.mode = EPI_AMP;
  epi.y = b;
  epi.ys = S;
  epi.base = xi_prime;
  epi.bs = S;
  const bool model = binned_model(p);
  if (model) {
    epi.av = metric_view<T>(m);
    epi.bins = 1;
    epi.xi_p = xp;
    epi.ps = 0;
  } else {
    epi.av = amp_view<T>(p, nullptr, 0);
  }
  int np = 0;
  NRE_TRY(run_hartley<T>(p, B, pro, epi, nullptr, m->tmp0.as<T>(), m->tmp1.as<T>(),
                         model ? m->part.as<double>() : nullptr, &np, st));
  if (model)
    NRE_TRY(amp_vjp<T>(amp_prior_of(p), m->state.as<double>(), 0, m->part.as<double>(), np,
                       xi_prime + N, S, b + N, S, B, st));
  return NRE_OK;
}

}  // namespace

namespace nre {
int metric_relinearize(nre_metric* m, const void* xi_p, cudaStream_t st) {
  if (m->model_kind != NRE_MODEL_CF) return set_error(NRE_EINVAL, "relinearisation is implemented for the correlated field");
  return m->dtype == NRE_F64 ? cf_metric_setup<double>(m, xi_p, st) : cf_metric_setup<float>(m, xi_p, st);
}

int metric_apply_impl(nre_metric* m, const void* v, void* out, int batch, cudaStream_t st, double* dot,
                      bool hyper_in_cg) {
  if (m->model_kind == NRE_MODEL_ICR) return icr_metric_apply(m, v, out, batch, st);
  if (m->model_kind == NRE_MODEL_KL) return kl_metric_apply(m->kl, v, out, batch, st);
  if (m->dtype == NRE_F64)
    return cf_metric_apply<double>(m, (const double*)v, (double*)out, batch, st, dot, hyper_in_cg);
  return cf_metric_apply<float>(m, (const float*)v, (float*)out, batch, st, dot, hyper_in_cg);
}
}  // namespace nre

extern "C" {

int lik_create(nre_lik** lik, int kind, int response, const double* mask_host, int64_t n_data,
               double sigma_or_scale) {
  clear_error();
  if (!lik) return set_error(NRE_EINVAL, "lik must not be NULL");
  *lik = nullptr;
  if (kind != NRE_LIK_GAUSS && kind != NRE_LIK_POISSON) return set_error(NRE_EINVAL, "unknown likelihood kind %d", kind);
  if (response != NRE_RESP_EXP && response != NRE_RESP_IDENTITY) return set_error(NRE_EINVAL, "unknown response %d", response);
  if (kind == NRE_LIK_POISSON && response != NRE_RESP_EXP)
    return set_error(NRE_EINVAL, "the Poisson likelihood uses the exponential response");
  if (!(sigma_or_scale > 0) || !std::isfinite(sigma_or_scale))
    return set_error(NRE_EINVAL, "sigma / scale must be positive");
  if (n_data < 0) return set_error(NRE_EINVAL, "n_data must be >= 0");
  nre_lik* l = new nre_lik();
  l->kind = kind;
  l->response = response;
  l->sig_or_scale = sigma_or_scale;
  l->n_data = n_data;
  if (mask_host) {
    if (kind == NRE_LIK_POISSON) {
      delete l;
      return set_error(NRE_EINVAL, "the Poisson likelihood takes no mask");
    }
    l->mask.assign(mask_host, mask_host + n_data);
  }
  *lik = l;
  return NRE_OK;
}

int lik_destroy(nre_lik* lik) {
  delete lik;
  return NRE_OK;
}

int metric_create(nre_metric** out, int model_kind, void* model_plan, const nre_lik* lik,
                  const void* xi_p, int max_batch, nre_stream_t stream) {
  clear_error();
  if (!out || !model_plan || !lik || !xi_p) return set_error(NRE_EINVAL, "NULL argument");
  *out = nullptr;
  if (max_batch < 1 || max_batch > 65535) return set_error(NRE_EINVAL, "max_batch must be in [1, 65535]");
  cudaStream_t st = (cudaStream_t)stream;
  nre_metric* m = new nre_metric();
  m->model_kind = model_kind;
  m->max_batch = max_batch;
  m->lik = *lik;
  int s = NRE_OK;
  if (model_kind == NRE_MODEL_CF) {
    m->cf = (nre_cf_plan*)model_plan;
    m->dtype = m->cf->dtype;
    m->n_data = m->cf->N;
    m->latent = m->cf->latent;
    m->stride = m->cf->stride;
    if (!m->lik.mask.empty() && (int64_t)m->lik.mask.size() != m->n_data)
      s = set_error(NRE_EINVAL, "mask has %lld entries, the grid %lld", (long long)m->lik.mask.size(),
                    (long long)m->n_data);
    else
      s = m->dtype == NRE_F64 ? cf_metric_setup<double>(m, xi_p, st) : cf_metric_setup<float>(m, xi_p, st);
  } else if (model_kind == NRE_MODEL_ICR) {
    m->icr = (nre_icr_plan*)model_plan;
    int dt;
    s = icr_layout(m->icr, &m->n_data, &m->latent, &m->stride, &dt);
    m->dtype = dt;
    if (s == NRE_OK) {
      if (m->lik.kind != NRE_LIK_GAUSS || m->lik.response != NRE_RESP_IDENTITY)
        s = set_error(NRE_EINVAL, "the ICR metric takes a Gaussian likelihood with identity response");
      else if (!m->lik.mask.empty() && (int64_t)m->lik.mask.size() != m->n_data)
        s = set_error(NRE_EINVAL, "mask size does not match the ICR output");
      else {
        const size_t es = m->dtype == NRE_F64 ? 8 : 4;
        s = m->xi_p.alloc(m->stride * es);
        if (s == NRE_OK) {
          cudaError_t e = cudaMemcpyAsync(m->xi_p.p, xi_p, m->latent * es, cudaMemcpyDeviceToDevice, st);
          if (e != cudaSuccess) s = set_error(NRE_ECUDA, "cudaMemcpyAsync: %s", cudaGetErrorString(e));
        }
        if (s == NRE_OK) s = icr_metric_setup(m, st);
      }
    }
  } else {
    s = set_error(NRE_EINVAL, "unknown model kind %d", model_kind);
  }
  if (s != NRE_OK) {
    delete m;
    return s;
  }
  *out = m;
  return NRE_OK;
}

int metric_destroy(nre_metric* m) {
  clear_error();
  if (m && m->model_kind == NRE_MODEL_KL)
    return set_error(NRE_EINVAL, "this metric belongs to its KL object (kl_destroy releases it)");
  delete m;
  return NRE_OK;
}

int metric_apply(nre_metric* m, const void* v, void* out, int batch, nre_stream_t stream) {
  clear_error();
  if (!m) return set_error(NRE_EINVAL, "metric must not be NULL");
  if (batch < 0 || batch > m->max_batch) return set_error(NRE_EINVAL, "batch %d outside [0, max_batch=%d]", batch, m->max_batch);
  if (batch == 0) return NRE_OK;
  if (!v || !out) return set_error(NRE_EINVAL, "NULL array argument");
  if (v == out) return set_error(NRE_EINVAL, "out may not alias v");
  return metric_apply_impl(m, v, out, batch, (cudaStream_t)stream);
}

int mgvi_rhs(nre_metric* m, const void* xi_prime, const void* eta, void* b, int batch, nre_stream_t stream) {
  clear_error();
  if (!m) return set_error(NRE_EINVAL, "metric must not be NULL");
  if (batch < 0 || batch > m->max_batch) return set_error(NRE_EINVAL, "batch %d outside [0, max_batch=%d]", batch, m->max_batch);
  if (batch == 0) return NRE_OK;
  if (!xi_prime || !eta || !b) return set_error(NRE_EINVAL, "NULL array argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (m->model_kind == NRE_MODEL_KL) return set_error(NRE_EINVAL, "mgvi_rhs needs the metric of one expansion point");
  if (m->model_kind == NRE_MODEL_ICR) return icr_mgvi_rhs(m, xi_prime, eta, b, batch, st);
  if (m->dtype == NRE_F64)
    return cf_mgvi_rhs<double>(m, (const double*)xi_prime, (const double*)eta, (double*)b, batch, st);
  return cf_mgvi_rhs<float>(m, (const float*)xi_prime, (const float*)eta, (float*)b, batch, st);
}

}  // extern "C"
