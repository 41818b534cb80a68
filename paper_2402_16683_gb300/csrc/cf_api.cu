// C ABI of the correlated-field model: plan creation (host geometry, bins,
// twiddles, reflection orbits) and cf_forward / cf_jvp / cf_vjp.
#include <cmath>
#include <cstring>
#include <vector>

#include "cf_internal.cuh"
#include "tma.cuh"

namespace nre {

static thread_local std::string g_err;

int set_error(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}
void clear_error() { g_err.clear(); }

int ensure(DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return NRE_OK;
  return b.alloc(bytes);
}

template <typename T>
AmpView<T> amp_view(const nre_cf_plan* p, const double* abin, int64_t astride) {
  AmpView<T> v{};
  v.mode = binned_model(p) ? AMPV_MODEL : AMPV_FIXED;
  v.afull = p->afull.as<T>();
  v.abin = abin;
  v.astride = astride;
  v.a0 = p->offset_std;
  v.lut = p->lut.as<uint16_t>();
  v.bpix = nullptr;
  v.tab = nullptr;
  v.a0t = T(p->offset_std);
  v.geo.ndim = p->ndim;
  for (int d = 0; d < 3; ++d) v.geo.l2[d] = p->l2[d];
  return v;
}
template AmpView<float> amp_view<float>(const nre_cf_plan*, const double*, int64_t);
template AmpView<double> amp_view<double>(const nre_cf_plan*, const double*, int64_t);

namespace {

bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }
int ilog2(int64_t x) {
  int r = 0;
  while ((int64_t(1) << r) < x) ++r;
  return r;
}

// Geometry checks shared by cf_create and cf_bin_map.  Returns the total
// length L_box (identical on every axis).
int check_geometry(int ndim, const int64_t* shape, const double* spacing, double* lbox) {
  if (ndim < 1 || ndim > 3) return set_error(NRE_EINVAL, "ndim must be 1, 2 or 3 (got %d)", ndim);
  if (!shape || !spacing) return set_error(NRE_EINVAL, "shape / spacing must not be NULL");
  for (int d = 0; d < ndim; ++d) {
    if (!is_pow2(shape[d]) || shape[d] < 4 || shape[d] > 4096)
      return set_error(NRE_EINVAL, "shape[%d] = %lld must be a power of two in [4, 4096]", d,
                       (long long)shape[d]);
    if (!(spacing[d] > 0.0) || !std::isfinite(spacing[d]))
      return set_error(NRE_EINVAL, "spacing[%d] must be positive and finite", d);
  }
  const double L0 = shape[0] * spacing[0];
  for (int d = 1; d < ndim; ++d) {
    const double Ld = shape[d] * spacing[d];
    if (std::fabs(Ld - L0) > 1e-12 * L0)
      return set_error(NRE_EINVAL, "total length N_d * spacing_d must agree on every axis "
                       "(isotropic |k|): axis 0 has %g, axis %d has %g", L0, d, Ld);
  }
  *lbox = L0;
  return NRE_OK;
}

// Folded squared radius q = sum m_d^2 of every harmonic pixel (C order).
void q_map(int ndim, const int64_t* shape, std::vector<int>& q) {
  int64_t N = 1;
  for (int d = 0; d < ndim; ++d) N *= shape[d];
  q.assign(N, 0);
  for (int64_t f = 0; f < N; ++f) {
    int64_t r = f;
    int acc = 0;
    for (int d = ndim - 1; d >= 0; --d) {
      const int64_t n = shape[d];
      const int64_t i = r % n;
      r /= n;
      const int64_t m = i <= n / 2 ? i : i - n;
      acc += (int)(m * m);
    }
    q[f] = acc;
  }
}

// Log-|k| binning: n_bins equal-width bins on l = ln|k| between the smallest
// and largest non-zero |k|, |k| = sqrt(q) / L_box; bin(q) for every q <= qmax.
void log_bins(int qmax, double lbox, int nb, std::vector<int>& bin_of_q,
              double* lmin_out, double* dl_out) {
  const double kmin = 1.0 / lbox;  // q = 1 always exists (every axis has >= 4 pixels)
  const double kmax = std::sqrt((double)qmax) / lbox;
  const double lmin = std::log(kmin), lmax = std::log(kmax);
  double dl = (lmax - lmin) / nb;
  if (dl == 0.0) dl = 1.0;
  bin_of_q.assign(qmax + 1, -1);
  for (int q = 1; q <= qmax; ++q) {
    const double k = std::sqrt((double)q / (lbox * lbox));
    const double l = std::log(k);
    int b = (int)std::floor((l - lmin) / dl);
    if (b > nb - 1) b = nb - 1;
    if (b < 0) b = 0;
    bin_of_q[q] = b;
  }
  *lmin_out = lmin;
  *dl_out = dl;
}

void lognormal(double mean, double sd, double* mu, double* s) {
  *mu = std::log(mean * mean / std::sqrt(mean * mean + sd * sd));
  *s = std::sqrt(std::log(1.0 + sd * sd / (mean * mean)));
}

template <typename T>
void fill_twiddles(std::vector<T>& tw, int L) {
  tw.resize(2 * (size_t)L);
  for (int m = 0; m < L; ++m) {
    const double ang = 2.0 * M_PI * ((double)m / (double)L);
    tw[2 * m] = (T)std::cos(ang);
    tw[2 * m + 1] = (T)(-std::sin(ang));
  }
}

// Reflection orbits of the rows (all axes but the last), see sweeps.cu.
void row_groups(const nre_cf_plan* p, std::vector<int>& rows, std::vector<int>& flags) {
  rows.clear();
  flags.clear();
  if (p->ndim == 2) {
    const int N0 = p->n[0];
    rows.push_back(0);
    rows.push_back(N0 / 2);
    flags.push_back(0);
    for (int i = 1; i < N0 / 2; ++i) {
      rows.push_back(i);
      rows.push_back(N0 - i);
      flags.push_back(1);
    }
  } else if (p->ndim == 3) {
    const int N0 = p->n[0], N1 = p->n[1];
    auto r = [&](int i0, int i1) { return ((i0 % N0 + N0) % N0) * N1 + ((i1 % N1 + N1) % N1); };
    const int h0 = N0 / 2, h1 = N1 / 2;
    // both indices self-mirrored
    rows.insert(rows.end(), {r(0, 0), r(h0, 0), r(0, h1), r(h0, h1)});
    flags.push_back(0);
    for (int i1 = 1; i1 < h1; ++i1) {  // axis 0 self-mirrored
      rows.insert(rows.end(), {r(0, i1), r(h0, i1), r(0, -i1), r(h0, -i1)});
      flags.push_back(2);
    }
    for (int i0 = 1; i0 < h0; ++i0) {  // axis 1 self-mirrored
      rows.insert(rows.end(), {r(i0, 0), r(-i0, 0), r(i0, h1), r(-i0, h1)});
      flags.push_back(1);
    }
    for (int i0 = 1; i0 < h0; ++i0)
      for (int i1 = 1; i1 < h1; ++i1) {
        rows.insert(rows.end(), {r(i0, i1), r(-i0, i1), r(i0, -i1), r(-i0, -i1)});
        flags.push_back(3);
      }
  }
}

template <typename T>
int upload_plan_tables(nre_cf_plan* p, const std::vector<double>& afull_host) {
  std::vector<T> tw;
  fill_twiddles(tw, p->Lmax);
  NRE_TRY(p->tw.upload(tw.data(), tw.size() * sizeof(T)));
  if (!afull_host.empty()) {
    std::vector<T> a(afull_host.begin(), afull_host.end());
    NRE_TRY(p->afull.upload(a.data(), a.size() * sizeof(T)));
  }
  return NRE_OK;
}

template <typename T>
int cf_forward_t(nre_cf_plan* p, const T* xi, T* s, int B, cudaStream_t st) {
  const int64_t N = p->N;
  NRE_TRY(ensure(p->ws_tmp0, (size_t)B * N * sizeof(T)));
  NRE_TRY(ensure(p->ws_tmp1, (size_t)B * N * sizeof(T)));
  Pro<T> pro{};
  pro.mode = PRO_AMP;
  pro.x = xi;
  pro.xs = p->stride;
  Epi<T> epi{};
  epi.mode = EPI_OFFSET;
  epi.y = s;
  epi.ys = N;
  epi.offset = p->offset_mean;
  if (binned_model(p)) {
    const int SS = amp_state_size(p->n_bins);
    NRE_TRY(ensure(p->ws_state, (size_t)B * SS * sizeof(double)));
    double* state = p->ws_state.as<double>();
    NRE_TRY(amp_forward<T>(amp_prior_of(p), xi + N, p->stride, state, B, st));
    pro.av = amp_view<T>(p, state + as_A(p->n_bins), SS);
  } else {
    pro.av = amp_view<T>(p, nullptr, 0);
  }
  int np = 0;
  return run_hartley<T>(p, B, pro, epi, nullptr, p->ws_tmp0.as<T>(), p->ws_tmp1.as<T>(), nullptr,
                        &np, st);
}

template <typename T>
int cf_jvp_t(nre_cf_plan* p, const T* xi_p, const T* v, T* jv, int B, cudaStream_t st) {
  const int64_t N = p->N;
  NRE_TRY(ensure(p->ws_tmp0, (size_t)B * N * sizeof(T)));
  NRE_TRY(ensure(p->ws_tmp1, (size_t)B * N * sizeof(T)));
  Pro<T> pro{};
  pro.mode = PRO_AMP;
  pro.x = v;
  pro.xs = p->stride;
  Epi<T> epi{};
  epi.mode = EPI_BUF;
  epi.y = jv;
  epi.ys = N;
  if (binned_model(p)) {
    const int nb = p->n_bins, SS = amp_state_size(nb);
    NRE_TRY(ensure(p->ws_state, (size_t)B * SS * sizeof(double)));
    NRE_TRY(ensure(p->ws_dA, (size_t)B * nb * sizeof(double)));
    double* state = p->ws_state.as<double>();
    const AmpPrior pr = amp_prior_of(p);
    NRE_TRY(amp_forward<T>(pr, xi_p + N, p->stride, state, B, st));
    NRE_TRY(amp_jvp<T>(pr, state, SS, v + N, p->stride, p->ws_dA.as<double>(), B, st));
    pro.av = amp_view<T>(p, state + as_A(nb), SS);
    pro.dA = p->ws_dA.as<double>();
    pro.nb = nb;
    pro.xi_p = xi_p;
    pro.ps = p->stride;
  } else {
    pro.av = amp_view<T>(p, nullptr, 0);
  }
  int np = 0;
  return run_hartley<T>(p, B, pro, epi, nullptr, p->ws_tmp0.as<T>(), p->ws_tmp1.as<T>(), nullptr,
                        &np, st);
}

template <typename T>
int cf_vjp_t(nre_cf_plan* p, const T* xi_p, const T* ct, T* g, int B, cudaStream_t st) {
  const int64_t N = p->N;
  NRE_TRY(ensure(p->ws_tmp0, (size_t)B * N * sizeof(T)));
  NRE_TRY(ensure(p->ws_tmp1, (size_t)B * N * sizeof(T)));
  Pro<T> pro{};
  pro.mode = PRO_BUF;
  pro.x = ct;
  pro.xs = N;
  Epi<T> epi{};
  epi.mode = EPI_AMP;
  epi.y = g;
  epi.ys = p->stride;
  if (binned_model(p)) {
    const int nb = p->n_bins, SS = amp_state_size(nb);
    NRE_TRY(ensure(p->ws_state, (size_t)B * SS * sizeof(double)));
    NRE_TRY(ensure(p->ws_part, (size_t)B * max_parts(p) * nb * sizeof(double)));
    double* state = p->ws_state.as<double>();
    const AmpPrior pr = amp_prior_of(p);
    NRE_TRY(amp_forward<T>(pr, xi_p + N, p->stride, state, B, st));
    epi.av = amp_view<T>(p, state + as_A(nb), SS);
    epi.bins = 1;
    epi.xi_p = xi_p;
    epi.ps = p->stride;
    int np = 0;
    double* part = p->ws_part.as<double>();
    NRE_TRY(run_hartley<T>(p, B, pro, epi, nullptr, p->ws_tmp0.as<T>(), p->ws_tmp1.as<T>(), part,
                           &np, st));
    return amp_vjp<T>(pr, state, SS, part, np, nullptr, 0, g + N, p->stride, B, st);
  }
  epi.av = amp_view<T>(p, nullptr, 0);
  int np = 0;
  return run_hartley<T>(p, B, pro, epi, nullptr, p->ws_tmp0.as<T>(), p->ws_tmp1.as<T>(), nullptr,
                        &np, st);
}

}  // namespace
}  // namespace nre

using namespace nre;

extern "C" {

const char* nre_last_error(void) { return g_err.c_str(); }
int nre_version(void) { return 100; }

int cf_bin_map(int ndim, const int64_t* shape, const double* spacing, int n_bins, int32_t* out) {
  clear_error();
  double lbox;
  NRE_TRY(check_geometry(ndim, shape, spacing, &lbox));
  if (n_bins < 2 || n_bins > 1024) return set_error(NRE_EINVAL, "n_bins must be in [2, 1024]");
  if (!out) return set_error(NRE_EINVAL, "out must not be NULL");
  std::vector<int> q;
  q_map(ndim, shape, q);
  int qmax = 0;
  for (int v : q) qmax = v > qmax ? v : qmax;
  std::vector<int> boq;
  double lmin, dl;
  log_bins(qmax, lbox, n_bins, boq, &lmin, &dl);
  for (size_t f = 0; f < q.size(); ++f) out[f] = q[f] == 0 ? -1 : boq[q[f]];
  return NRE_OK;
}

int cf_create(nre_cf_plan** plan, int ndim, const int64_t* shape, const double* spacing,
              const nre_cf_amp_params* amp, int dtype) {
  clear_error();
  if (!plan || !amp) return set_error(NRE_EINVAL, "plan / amp must not be NULL");
  *plan = nullptr;
  double lbox;
  NRE_TRY(check_geometry(ndim, shape, spacing, &lbox));
  if (dtype != NRE_F32 && dtype != NRE_F64) return set_error(NRE_EINVAL, "dtype must be NRE_F32 or NRE_F64");
  if (amp->kind < NRE_AMP_ARRAY || amp->kind > NRE_AMP_MATERN_MODEL)
    return set_error(NRE_EINVAL, "unknown amplitude kind %d", amp->kind);
  // the device's count of bounded waits that ran out, allocated here (outside
  // any stream capture) before the first sweep takes it
  (void)timeout_word();
  nre_cf_plan* p = new nre_cf_plan();
  p->ndim = ndim;
  p->dtype = dtype;
  p->N = 1;
  for (int d = 0; d < ndim; ++d) {
    p->n[d] = (int)shape[d];
    p->l2[d] = ilog2(shape[d]);
    p->N *= shape[d];
    if (p->n[d] > p->Lmax) p->Lmax = p->n[d];
  }
  p->log2Lmax = ilog2(p->Lmax);
  p->nrows = p->N / p->n[ndim - 1];
  p->amp_kind = amp->kind;
  p->offset_mean = amp->offset_mean;
  p->offset_std = amp->offset_std;
  auto fail = [&](int code) {
    delete p;
    return code;
  };

  std::vector<int> q;
  q_map(ndim, shape, q);
  int qmax = 0;
  for (int v : q) qmax = v > qmax ? v : qmax;
  std::vector<double> afull;
  if (amp->kind == NRE_AMP_ARRAY) {
    if (!amp->amp_array) return fail(set_error(NRE_EINVAL, "NRE_AMP_ARRAY needs amp_array"));
    afull.assign(amp->amp_array, amp->amp_array + p->N);
  } else if (amp->kind == NRE_AMP_MATERN_FIXED) {
    if (!(amp->k0 > 0) || !(amp->variance >= 0))
      return fail(set_error(NRE_EINVAL, "MATERN_FIXED needs k0 > 0 and variance >= 0"));
    afull.resize(p->N);
    double s2 = 0.0;
    for (int64_t f = 0; f < p->N; ++f) {
      const double k = std::sqrt((double)q[f] / (lbox * lbox));
      const double a = std::pow(1.0 + (k / amp->k0) * (k / amp->k0), -amp->gamma);
      afull[f] = a;
      if (q[f] != 0) s2 += a * a;
    }
    const double sc = s2 > 0 ? std::sqrt(amp->variance / s2) : 0.0;
    for (int64_t f = 0; f < p->N; ++f) afull[f] = q[f] == 0 ? amp->zero_mode : afull[f] * sc;
  } else {
    const int nb = amp->n_bins;
    if (nb < 2 || nb > 1024) return fail(set_error(NRE_EINVAL, "n_bins must be in [2, 1024]"));
    if (amp->kind == NRE_AMP_POWER_MODEL) {
      if (!(amp->fluct_mean > 0 && amp->fluct_std > 0 && amp->flex_mean > 0 && amp->flex_std > 0 &&
            amp->asp_mean > 0 && amp->asp_std > 0 && amp->slope_std >= 0))
        return fail(set_error(NRE_EINVAL, "log-normal hyper-parameters need positive mean and std"));
    } else if (!(amp->scale_mean > 0 && amp->scale_std > 0 && amp->cutoff_mean > 0 && amp->cutoff_std > 0 &&
                 amp->lls_std >= 0)) {
      return fail(set_error(NRE_EINVAL, "Matern scale / cutoff need positive mean and std, slope std >= 0"));
    }
    if (qmax > 65535 * 4096)  // unreachable for shapes <= 4096^2 but keeps the LUT bounded
      return fail(set_error(NRE_EINVAL, "grid too large for the bin table"));
    p->n_bins = nb;
    if (amp->kind == NRE_AMP_POWER_MODEL) {
      p->n_hyper = 4 + 2 * (nb - 1);
      lognormal(amp->fluct_mean, amp->fluct_std, &p->mu_fl, &p->s_fl);
      lognormal(amp->flex_mean, amp->flex_std, &p->mu_fx, &p->s_fx);
      lognormal(amp->asp_mean, amp->asp_std, &p->mu_as, &p->s_as);
      p->sl_m = amp->slope_mean;
      p->sl_s = amp->slope_std;
    } else {
      p->n_hyper = 3;  // xi_scale, xi_cutoff, xi_slope
      lognormal(amp->scale_mean, amp->scale_std, &p->mu_sc, &p->s_sc);
      lognormal(amp->cutoff_mean, amp->cutoff_std, &p->mu_ct, &p->s_ct);
      p->al_m = amp->lls_mean;
      p->al_s = amp->lls_std;
    }
    std::vector<int> boq;
    double lmin, dl;
    log_bins(qmax, lbox, nb, boq, &lmin, &dl);
    std::vector<uint16_t> lut(qmax + 1, 0xFFFF);
    for (int v = 1; v <= qmax; ++v) lut[v] = (uint16_t)boq[v];
    std::vector<double> counts(nb, 0.0), centres(nb);
    for (int64_t f = 0; f < p->N; ++f)
      if (q[f] != 0) counts[boq[q[f]]] += 1.0;
    for (int i = 0; i < nb; ++i) centres[i] = lmin + (i + 0.5) * dl;
    int s;
    if ((s = p->lut.upload(lut.data(), lut.size() * sizeof(uint16_t))) != NRE_OK) return fail(s);
    if ((s = p->counts.upload(counts.data(), nb * sizeof(double))) != NRE_OK) return fail(s);
    if ((s = p->centres.upload(centres.data(), nb * sizeof(double))) != NRE_OK) return fail(s);
  }
  p->latent = p->N + p->n_hyper;
  p->stride = round_up(p->latent, 64);

  std::vector<int> rows, flags;
  row_groups(p, rows, flags);
  p->n_groups = (int)flags.size();
  p->G = ndim == 3 ? 4 : 2;
  int s;
  if (!rows.empty()) {
    if ((s = p->grows.upload(rows.data(), rows.size() * sizeof(int))) != NRE_OK) return fail(s);
    if ((s = p->gflags.upload(flags.data(), flags.size() * sizeof(int))) != NRE_OK) return fail(s);
  }
  s = dtype == NRE_F64 ? upload_plan_tables<double>(p, afull) : upload_plan_tables<float>(p, afull);
  if (s != NRE_OK) return fail(s);
  *plan = p;
  return NRE_OK;
}

int cf_destroy(nre_cf_plan* plan) {
  delete plan;
  return NRE_OK;
}

int cf_latent_layout(const nre_cf_plan* p, int64_t* n_field, int64_t* n_hyper, int64_t* latent_size,
                     int64_t* stride) {
  clear_error();
  if (!p) return set_error(NRE_EINVAL, "plan must not be NULL");
  if (n_field) *n_field = p->N;
  if (n_hyper) *n_hyper = p->n_hyper;
  if (latent_size) *latent_size = p->latent;
  if (stride) *stride = p->stride;
  return NRE_OK;
}

int cf_latent_size(const nre_cf_plan* p, int64_t* latent_size) {
  return cf_latent_layout(p, nullptr, nullptr, latent_size, nullptr);
}

#define NRE_CF_CHECK(ptrs)                                                    \
  clear_error();                                                              \
  if (!plan) return set_error(NRE_EINVAL, "plan must not be NULL");           \
  if (batch < 0 || batch > 65535) return set_error(NRE_EINVAL, "batch must be in [0, 65535]"); \
  if (batch == 0) return NRE_OK;                                              \
  if (!(ptrs)) return set_error(NRE_EINVAL, "NULL array argument");

int cf_forward(nre_cf_plan* plan, const void* xi, void* s, int batch, nre_stream_t stream) {
  NRE_CF_CHECK(xi && s);
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->dtype == NRE_F64) return cf_forward_t<double>(plan, (const double*)xi, (double*)s, batch, st);
  return cf_forward_t<float>(plan, (const float*)xi, (float*)s, batch, st);
}

int cf_jvp(nre_cf_plan* plan, const void* xi_p, const void* v, void* jv, int batch, nre_stream_t stream) {
  NRE_CF_CHECK(xi_p && v && jv);
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->dtype == NRE_F64)
    return cf_jvp_t<double>(plan, (const double*)xi_p, (const double*)v, (double*)jv, batch, st);
  return cf_jvp_t<float>(plan, (const float*)xi_p, (const float*)v, (float*)jv, batch, st);
}

int cf_vjp(nre_cf_plan* plan, const void* xi_p, const void* ct, void* g, int batch, nre_stream_t stream) {
  NRE_CF_CHECK(xi_p && ct && g);
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->dtype == NRE_F64)
    return cf_vjp_t<double>(plan, (const double*)xi_p, (const double*)ct, (double*)g, batch, st);
  return cf_vjp_t<float>(plan, (const float*)xi_p, (const float*)ct, (float*)g, batch, st);
}

}  // extern "C"
