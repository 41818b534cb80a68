// Non-parametric amplitude model sqrt(P) of the correlated field, FP64 for both
// plan dtypes: forward, JVP and VJP.  One CTA per sample, one thread per log-|k|
// bin; the integrated Wiener process is two prefix sums, its adjoint two suffix
// sums.
//
// Sec. "Gaussian Processes" (add_fluctuations with fluctuations,
// loglogavgslope, flexibility, asperity; non_parametric_kind = "power").  The
// paper defers the equations to its citations; the reading implemented here:
//   theta_fl, theta_flex, theta_asp log-normal with the given (mean, std) of the
//   variable itself, theta_slope normal;  D_i = l_i - l_{i-1};
//   x_i = x_{i-1} + theta_flex sqrt(D_i) xi1_i,
//   y_i = y_{i-1} + D_i (x_{i-1} + x_i)/2 + theta_flex sqrt(D_i^3/12 + theta_asp D_i) xi2_i,
//   tau_i = theta_slope (l_i - l_0) + y_i,  a_i = exp(tau_i / 2),
//   A_i = theta_fl a_i / sqrt(sum_b n_b a_b^2)   (n_b: non-zero modes in bin b).
//
// The parametric Matern kernel the same section names beside it, on the same
// bins at the bin-centre wavenumbers k_i = exp(l_i) (reading of this library):
//   theta_scale, theta_cutoff log-normal, theta_slope normal;
//   a_i = (1 + (k_i / theta_cutoff)^2)^(theta_slope / 4),
//   A_i = theta_scale a_i / sqrt(sum_b n_b a_b^2).
// Its JVP and VJP are per-bin maps plus one block reduction each.
#include "cf_internal.cuh"

namespace nre {

namespace {

// Block-wide inclusive prefix / suffix sums of one double per thread
// (blockDim.x a multiple of 32): shuffle scans within each warp, then a scan of
// the warp totals.  The result is also left in buf[threadIdx.x] for the
// neighbour reads of the callers.
__device__ __forceinline__ double warp_prefix(double v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

__device__ __forceinline__ double warp_suffix(double v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_down_sync(0xffffffffu, v, o);
    if (lane + o < 32) v += t;
  }
  return v;
}

__device__ double scan_incl(double v, double* buf) {
  __shared__ double wt[32];
  const int i = threadIdx.x, lane = i & 31, w = i >> 5, nw = blockDim.x >> 5;
  double x = warp_prefix(v);
  __syncthreads();  // earlier readers of buf / wt are done
  if (lane == 31) wt[w] = x;
  __syncthreads();
  if (w == 0) wt[lane] = warp_prefix(lane < nw ? wt[lane] : 0.0);
  __syncthreads();
  if (w > 0) x += wt[w - 1];
  buf[i] = x;
  __syncthreads();
  return x;
}

__device__ double scan_suffix(double v, double* buf) {
  __shared__ double wt[32];
  const int i = threadIdx.x, lane = i & 31, w = i >> 5, nw = blockDim.x >> 5;
  double x = warp_suffix(v);
  __syncthreads();
  if (lane == 0) wt[w] = x;
  __syncthreads();
  if (w == 0) wt[lane] = warp_suffix(lane < nw ? wt[lane] : 0.0);
  __syncthreads();
  if (w + 1 < nw) x += wt[w + 1];
  buf[i] = x;
  __syncthreads();
  return x;
}

struct Th {
  double fl, sl, fx, as;
};

template <typename T>
__device__ Th thetas(const AmpPrior& pr, const T* h) {
  Th t;
  t.fl = exp(pr.mu_fl + pr.s_fl * double(h[0]));
  t.sl = pr.sl_m + pr.sl_s * double(h[1]);
  t.fx = exp(pr.mu_fx + pr.s_fx * double(h[2]));
  t.as = exp(pr.mu_as + pr.s_as * double(h[3]));
  return t;
}

template <typename T>
__global__ void k_amp_forward(AmpPrior pr, const T* h, int64_t hs, double* state) {
  __shared__ double buf[1024];
  __shared__ double red[32];
  const int b = blockIdx.x, i = threadIdx.x, nb = pr.nb;
  const T* hb = h + b * hs;
  double* st = state + (int64_t)b * amp_state_size(nb);
  const Th th = thetas(pr, hb);
  const bool act = i < nb;
  const double l = act ? pr.centres[i] : 0.0;
  const double l0 = pr.centres[0];
  const double d = (act && i > 0) ? l - pr.centres[i - 1] : 0.0;
  const double xi1 = (act && i > 0) ? double(hb[4 + i - 1]) : 0.0;
  const double xi2 = (act && i > 0) ? double(hb[4 + nb - 1 + i - 1]) : 0.0;
  const double x = scan_incl(th.fx * sqrt(d) * xi1, buf);
  const double xprev = i > 0 ? buf[i - 1] : 0.0;
  const double c = (act && i > 0) ? sqrt(d * d * d / 12.0 + th.as * d) : 0.0;
  const double incy = (act && i > 0) ? d * (xprev + x) / 2.0 + th.fx * c * xi2 : 0.0;
  const double y = scan_incl(incy, buf);
  const double tau = th.sl * (l - l0) + y;
  const double a = act ? exp(tau / 2.0) : 0.0;
  const double S = block_sum(act ? pr.counts[i] * a * a : 0.0, red);
  if (act) {
    st[as_a(nb) + i] = a;
    st[as_c(nb) + i] = c;
    st[as_A(nb) + i] = th.fl * a / sqrt(S);
    st[as_xi1(nb) + i] = xi1;
    st[as_xi2(nb) + i] = xi2;
  }
  if (i == 0) {
    st[AS_THFL] = th.fl;
    st[AS_THSL] = th.sl;
    st[AS_THFX] = th.fx;
    st[AS_THAS] = th.as;
    st[AS_S] = S;
  }
}

template <typename T>
__global__ void k_amp_jvp(AmpPrior pr, const double* state, int64_t ss, const T* dh, int64_t dhs,
                          double* dA) {
  __shared__ double buf[1024];
  __shared__ double red[32];
  const int b = blockIdx.x, i = threadIdx.x, nb = pr.nb;
  const double* st = state + b * ss;
  const T* g = dh + b * dhs;
  const double th_fl = st[AS_THFL], th_fx = st[AS_THFX], th_as = st[AS_THAS], S = st[AS_S];
  const double dth_fl = th_fl * pr.s_fl * double(g[0]);
  const double dth_sl = pr.sl_s * double(g[1]);
  const double dth_fx = th_fx * pr.s_fx * double(g[2]);
  const double dth_as = th_as * pr.s_as * double(g[3]);
  const bool act = i < nb;
  const double l = act ? pr.centres[i] : 0.0;
  const double l0 = pr.centres[0];
  const double d = (act && i > 0) ? l - pr.centres[i - 1] : 0.0;
  const double xi1 = act ? st[as_xi1(nb) + i] : 0.0;
  const double xi2 = act ? st[as_xi2(nb) + i] : 0.0;
  const double c = act ? st[as_c(nb) + i] : 0.0;
  const double a = act ? st[as_a(nb) + i] : 0.0;
  const double dxi1 = (act && i > 0) ? double(g[4 + i - 1]) : 0.0;
  const double dxi2 = (act && i > 0) ? double(g[4 + nb - 1 + i - 1]) : 0.0;
  const double sd = sqrt(d);
  const double dx = scan_incl((act && i > 0) ? dth_fx * sd * xi1 + th_fx * sd * dxi1 : 0.0, buf);
  const double dxprev = i > 0 ? buf[i - 1] : 0.0;
  double incy = 0.0;
  if (act && i > 0) {
    const double dc = d * dth_as / (2.0 * c);
    incy = d * (dxprev + dx) / 2.0 + (dth_fx * c + th_fx * dc) * xi2 + th_fx * c * dxi2;
  }
  const double dy = scan_incl(incy, buf);
  const double dtau = dth_sl * (l - l0) + dy;
  const double da = a * dtau / 2.0;
  const double dS = block_sum(act ? pr.counts[i] * 2.0 * a * da : 0.0, red);
  const double rs = 1.0 / sqrt(S);
  if (act) dA[(int64_t)b * nb + i] = dth_fl * a * rs + th_fl * da * rs - th_fl * a * dS * rs * rs * rs / 2.0;
}

template <typename T>
__global__ void k_amp_vjp(AmpPrior pr, const double* state, int64_t ss, const double* partials,
                          int nparts, const T* base, int64_t bhs, T* out, int64_t ohs, double* dot) {
  __shared__ double buf[1024];
  __shared__ double red[32];
  const int b = blockIdx.x, i = threadIdx.x, nb = pr.nb;
  const double* st = state + b * ss;
  const bool act = i < nb;
  const double gA = act ? sum_strided(partials + (int64_t)b * nparts * nb + i, nparts, nb) : 0.0;
  const double th_fl = st[AS_THFL], th_fx = st[AS_THFX], th_as = st[AS_THAS], S = st[AS_S];
  const double rs = 1.0 / sqrt(S);
  const double a = act ? st[as_a(nb) + i] : 0.0;
  const double c = act ? st[as_c(nb) + i] : 0.0;
  const double xi1 = act ? st[as_xi1(nb) + i] : 0.0;
  const double xi2 = act ? st[as_xi2(nb) + i] : 0.0;
  const double n = act ? pr.counts[i] : 0.0;
  const double l = act ? pr.centres[i] : 0.0;
  const double l0 = pr.centres[0];
  const double d = (act && i > 0) ? l - pr.centres[i - 1] : 0.0;
  const double d_next = (i + 1 < nb) ? pr.centres[i + 1] - l : 0.0;

  const double ga_dot = block_sum(gA * a, red);
  const double g_thfl = ga_dot * rs;
  const double g_a = th_fl * rs * gA - th_fl * rs * rs * rs * n * a * ga_dot;
  const double g_tau = g_a * a / 2.0;
  const double g_thsl = block_sum(g_tau * (l - l0), red);
  const double y_hat = scan_suffix(g_tau, buf);
  const double y_hat_next = (i + 1 < (int)blockDim.x) ? buf[i + 1] : 0.0;
  double x_dir = 0.0, g_xi2 = 0.0, p_fx = 0.0, p_as = 0.0;
  if (act && i >= 1) {
    x_dir += y_hat * d / 2.0;
    g_xi2 = y_hat * th_fx * c;
    p_fx += y_hat * c * xi2;
    p_as += y_hat * th_fx * xi2 * d / (2.0 * c);
  }
  if (act && i + 1 < nb) x_dir += y_hat_next * d_next / 2.0;
  const double x_hat = scan_suffix(x_dir, buf);
  double g_xi1 = 0.0;
  if (act && i >= 1) {
    g_xi1 = x_hat * th_fx * sqrt(d);
    p_fx += x_hat * sqrt(d) * xi1;
  }
  const double g_thfx = block_sum(p_fx, red);
  const double g_thas = block_sum(p_as, red);
  T* o = out + b * ohs;
  const T* bb = base ? base + b * bhs : nullptr;
  double dsum = 0.0;  // sum(base * out) over the hyper entries (fused inner product)
  if (act && i >= 1) {
    const int j1 = 4 + i - 1, j2 = 4 + nb - 1 + i - 1;
    const T o1 = T((bb ? double(bb[j1]) : 0.0) + g_xi1), o2 = T((bb ? double(bb[j2]) : 0.0) + g_xi2);
    o[j1] = o1;
    o[j2] = o2;
    if (bb) dsum += double(bb[j1] * o1) + double(bb[j2] * o2);
  }
  if (i == 0) {
    const double g4[4] = {g_thfl * th_fl * pr.s_fl, g_thsl * pr.sl_s, g_thfx * th_fx * pr.s_fx,
                          g_thas * th_as * pr.s_as};
    for (int j = 0; j < 4; ++j) {
      const T oj = T((bb ? double(bb[j]) : 0.0) + g4[j]);
      o[j] = oj;
      if (bb) dsum += double(bb[j] * oj);
    }
  }
  if (dot != nullptr) {
    const double t = block_sum(dsum, red);
    if (i == 0) dot[(int64_t)b * kDotStride + kDotHyper] = t;
  }
}

// ---------------------------------------------------------------- Matern
// State of a sample (amp_state_size layout): header theta_scale (AS_THFL),
// theta_slope (AS_THSL), theta_cutoff (AS_THFX), S; per bin a_i (as_a),
// L_i = ln(1 + r_i) (as_c), A_i (as_A), r_i / (1 + r_i) (as_xi1) with
// r_i = (k_i / theta_cutoff)^2.
template <typename T>
__global__ void k_amp_forward_matern(AmpPrior pr, const T* h, int64_t hs, double* state) {
  __shared__ double red[32];
  const int b = blockIdx.x, i = threadIdx.x, nb = pr.nb;
  const T* hb = h + b * hs;
  double* st = state + (int64_t)b * amp_state_size(nb);
  const double th_sc = exp(pr.mu_sc + pr.s_sc * double(hb[0]));
  const double th_ct = exp(pr.mu_ct + pr.s_ct * double(hb[1]));
  const double th_al = pr.al_m + pr.al_s * double(hb[2]);
  const bool act = i < nb;
  const double k = act ? exp(pr.centres[i]) : 0.0;
  const double r = (k / th_ct) * (k / th_ct);
  const double L = log1p(r);
  const double a = act ? exp(th_al * L / 4.0) : 0.0;
  const double S = block_sum(act ? pr.counts[i] * a * a : 0.0, red);
  if (act) {
    st[as_a(nb) + i] = a;
    st[as_c(nb) + i] = L;
    st[as_A(nb) + i] = th_sc * a / sqrt(S);
    st[as_xi1(nb) + i] = r / (1.0 + r);
    st[as_xi2(nb) + i] = 0.0;
  }
  if (i == 0) {
    st[AS_THFL] = th_sc;
    st[AS_THSL] = th_al;
    st[AS_THFX] = th_ct;
    st[AS_THAS] = 0.0;
    st[AS_S] = S;
  }
}

// dA_i: d ln a_i = d theta_slope L_i / 4 - (theta_slope / 2) q_i d theta_cutoff / theta_cutoff
// (q_i = r_i / (1 + r_i)), then the normalisation as in the power model.
template <typename T>
__global__ void k_amp_jvp_matern(AmpPrior pr, const double* state, int64_t ss, const T* dh, int64_t dhs,
                                 double* dA) {
  __shared__ double red[32];
  const int b = blockIdx.x, i = threadIdx.x, nb = pr.nb;
  const double* st = state + b * ss;
  const T* g = dh + b * dhs;
  const double th_sc = st[AS_THFL], th_al = st[AS_THSL], th_ct = st[AS_THFX], S = st[AS_S];
  const double dsc = th_sc * pr.s_sc * double(g[0]);
  const double dct = th_ct * pr.s_ct * double(g[1]);
  const double dal = pr.al_s * double(g[2]);
  const bool act = i < nb;
  const double a = act ? st[as_a(nb) + i] : 0.0;
  const double L = act ? st[as_c(nb) + i] : 0.0;
  const double q = act ? st[as_xi1(nb) + i] : 0.0;
  const double da = a * (dal * L / 4.0 - (th_al / 2.0) * q * dct / th_ct);
  const double dS = block_sum(act ? pr.counts[i] * 2.0 * a * da : 0.0, red);
  const double rs = 1.0 / sqrt(S);
  if (act) dA[(int64_t)b * nb + i] = dsc * a * rs + th_sc * da * rs - th_sc * a * dS * rs * rs * rs / 2.0;
}

template <typename T>
__global__ void k_amp_vjp_matern(AmpPrior pr, const double* state, int64_t ss, const double* partials,
                                 int nparts, const T* base, int64_t bhs, T* out, int64_t ohs, double* dot) {
  __shared__ double red[32];
  const int b = blockIdx.x, i = threadIdx.x, nb = pr.nb;
  const double* st = state + b * ss;
  const bool act = i < nb;
  const double gA = act ? sum_strided(partials + (int64_t)b * nparts * nb + i, nparts, nb) : 0.0;
  const double th_sc = st[AS_THFL], th_al = st[AS_THSL], th_ct = st[AS_THFX], S = st[AS_S];
  const double rs = 1.0 / sqrt(S);
  const double a = act ? st[as_a(nb) + i] : 0.0;
  const double L = act ? st[as_c(nb) + i] : 0.0;
  const double q = act ? st[as_xi1(nb) + i] : 0.0;
  const double n = act ? pr.counts[i] : 0.0;
  const double ga_dot = block_sum(gA * a, red);
  const double g_a = th_sc * rs * gA - th_sc * rs * rs * rs * n * a * ga_dot;
  const double g_lna = g_a * a;
  const double g_al = block_sum(g_lna * L / 4.0, red);
  const double g_ct = block_sum(g_lna * (-(th_al / 2.0) * q / th_ct), red);
  if (i == 0) {
    T* o = out + b * ohs;
    const T* bb = base ? base + b * bhs : nullptr;
    const double g3[3] = {ga_dot * rs * th_sc * pr.s_sc, g_ct * th_ct * pr.s_ct, g_al * pr.al_s};
    double dsum = 0.0;
    for (int j = 0; j < 3; ++j) {
      const T oj = T((bb ? double(bb[j]) : 0.0) + g3[j]);
      o[j] = oj;
      if (bb) dsum += double(bb[j] * oj);
    }
    if (dot != nullptr) dot[(int64_t)b * kDotStride + kDotHyper] = dsum;
  }
}

// Linearised amplitude model: the Jacobian at the expansion point,
// Jt[h][i] = dA_i / dh (FP64, from the JVP along the unit vectors, so the
// cumulative integration stays FP64), stored in FP32 both ways for the FP32
// path:  dA = J dh  and  g_h = J^T gA, in FP32 (a warp per output: lane runs
// of at most 17 products, then a shuffle tree).
template <typename T>
__global__ void k_eye(T* e, int n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < (int64_t)n * n;
       k += (int64_t)gridDim.x * blockDim.x)
    e[k] = (k / n == k % n) ? T(1) : T(0);
}

// Jacobian copies in FP32 with rows padded to a multiple of four floats
// (zeros), so that the products below read them as 16-byte vectors:
// G [nb][nhp] and Gt [nh][nbp], nhp / nbp = nh / nb rounded up to 4.
__global__ void k_jac_store(const double* Jt, int nh, int nb, float* G, float* Gt) {
  const int nhp = (nh + 3) & ~3, nbp = (nb + 3) & ~3;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < (int64_t)nb * nhp; k += stride) {
    const int i = (int)(k / nhp), h = (int)(k % nhp);
    G[k] = h < nh ? float(Jt[(int64_t)h * nb + i]) : 0.f;
  }
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < (int64_t)nh * nbp; k += stride) {
    const int h = (int)(k / nbp), i = (int)(k % nbp);
    Gt[k] = i < nb ? float(Jt[(int64_t)h * nb + i]) : 0.f;
  }
}

// dA[b][i] = sum_h G[i][h] dh[b][h] (G rows padded to nhp floats); one warp
// per output, each lane with eight loads of G and eight of dh in flight per
// round, FP32 arithmetic (the FP64 units of this part are a small fraction of
// its FP32 rate).  Staging dh in shared memory measured slower: the barrier
// puts a second round trip on the path of this latency-bound kernel.
template <typename T>
__global__ void __launch_bounds__(256) k_amp_jvp_lin(const float* G, int64_t gs, int nb, int nh, const T* dh,
                                                    int64_t dhs, double* dA, double* gzero) {
  const int b = blockIdx.y, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= nb) return;
  if (gzero != nullptr && lane == 0) gzero[(int64_t)b * nb + i] = 0.0;
  const float* g = G + b * gs + (int64_t)i * ((nh + 3) & ~3);
  const T* d = dh + b * dhs;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int h0 = 0; h0 < nh; h0 += 256) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int h = h0 + lane + 32 * k;
      if (h < nh) acc[k] += __ldg(&g[h]) * float(d[h]);
    }
  }
  const float t = warp_sum_f(((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7])));
  if (lane == 0) dA[(int64_t)b * nb + i] = double(t);
}

// out_h[b] = base_h[b] + G^T g[b] with the per-bin sums g[b] complete in
// gsum[b][nb] (nb <= 1024); CTAs of 32 outputs, 8 warps of 4 rows of Gt,
// g[b] staged in shared memory as FP32.  With `dot`, also the CTA's share of
// sum(base_h * out_h) at dot[b][kDotHyper + cta].  FP32 arithmetic; FP64 only
// for the one conversion of each staged sum and of the CTA's share.
template <typename T>
__global__ void __launch_bounds__(256) k_amp_vjp_lin(const float* Gt, int64_t gs, int nb, int nh,
                                                    const double* gsum, const T* base, int64_t bhs, T* out,
                                                    int64_t ohs, double* dot) {
  __shared__ float4 sg[256];
  __shared__ float red[8];
  const int b = blockIdx.y, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nb4 = (nb + 3) >> 2;
  const int h0 = blockIdx.x * 32 + w * 4;
  const int hq = h0 + (lane & 3);  // lanes 0-3: the warp's four outputs
  const T* bb = base ? base + b * bhs : nullptr;
  float bval = 0.f;
  if (bb != nullptr && lane < 4 && hq < nh) bval = float(bb[hq]);
  // first 64 vectors of the warp's rows, in flight across the staging barrier
  float4 gv[4][2];
  const float4* g4 = reinterpret_cast<const float4*>(Gt + b * gs);
  auto load = [&](int j0) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int j = j0 + lane + 32 * k;
        gv[q][k] = (h0 + q < nh && j < nb4) ? __ldg(g4 + (int64_t)(h0 + q) * nb4 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
  };
  load(0);
  float* sgf = reinterpret_cast<float*>(sg);
  const double* gb = gsum + (int64_t)b * nb;
  for (int i = threadIdx.x; i < 4 * nb4; i += blockDim.x) sgf[i] = i < nb ? float(gb[i]) : 0.f;
  __syncthreads();
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int j0 = 0; j0 < nb4; j0 += 64) {
    if (j0 > 0) load(j0);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int j = j0 + lane + 32 * k;
      if (j < nb4) {
        const float4 a = sg[j];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += dot4(gv[q][k], a);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = warp_sum_f(acc[q]);
  const int ql = lane & 3;
  const float t = ql == 0 ? acc[0] : ql == 1 ? acc[1] : ql == 2 ? acc[2] : acc[3];
  float dsum = 0.f;
  if (lane < 4 && hq < nh) {
    const T v = T(bval + t);
    out[b * ohs + hq] = v;
    dsum = bval * float(v);
  }
  if (dot != nullptr) {
    dsum = warp_sum_f(dsum);
    if (lane == 0) red[w] = dsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      float tot = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) tot += red[k];
      dot[(int64_t)b * kDotStride + kDotHyper + blockIdx.x] = double(tot);
    }
  }
}

int amp_threads(int nb) { return (nb + 31) / 32 * 32; }

}  // namespace

AmpPrior amp_prior_of(const nre_cf_plan* p) {
  AmpPrior a;
  a.kind = p->amp_kind;
  a.mu_sc = p->mu_sc;
  a.s_sc = p->s_sc;
  a.mu_ct = p->mu_ct;
  a.s_ct = p->s_ct;
  a.al_m = p->al_m;
  a.al_s = p->al_s;
  a.mu_fl = p->mu_fl;
  a.s_fl = p->s_fl;
  a.mu_fx = p->mu_fx;
  a.s_fx = p->s_fx;
  a.mu_as = p->mu_as;
  a.s_as = p->s_as;
  a.sl_m = p->sl_m;
  a.sl_s = p->sl_s;
  a.centres = p->centres.as<double>();
  a.counts = p->counts.as<double>();
  a.nb = p->n_bins;
  return a;
}

template <typename T>
int amp_forward(const AmpPrior& pr, const T* h, int64_t hs, double* state, int B, cudaStream_t st) {
  prof_begin("amp_forward", (double)B * pr.nb * (2 * sizeof(T) + 5 * 8), st);
  if (pr.kind == NRE_AMP_MATERN_MODEL) k_amp_forward_matern<T><<<B, amp_threads(pr.nb), 0, st>>>(pr, h, hs, state);
  else k_amp_forward<T><<<B, amp_threads(pr.nb), 0, st>>>(pr, h, hs, state);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  return NRE_OK;
}

template <typename T>
int amp_jvp(const AmpPrior& pr, const double* state, int64_t ss, const T* dh, int64_t dhs,
            double* dA, int B, cudaStream_t st) {
  prof_begin("amp_jvp", (double)B * pr.nb * (2 * sizeof(T) + 8) + (ss ? B : 1) * pr.nb * 40.0, st);
  if (pr.kind == NRE_AMP_MATERN_MODEL) k_amp_jvp_matern<T><<<B, amp_threads(pr.nb), 0, st>>>(pr, state, ss, dh, dhs, dA);
  else k_amp_jvp<T><<<B, amp_threads(pr.nb), 0, st>>>(pr, state, ss, dh, dhs, dA);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  return NRE_OK;
}

template <typename T>
int amp_vjp(const AmpPrior& pr, const double* state, int64_t ss, const double* partials,
            int nparts, const T* base_h, int64_t bhs, T* out_h, int64_t ohs, int B,
            cudaStream_t st, double* dot) {
  prof_begin("amp_vjp", (double)B * pr.nb * (8.0 * nparts + (base_h ? 4 : 2) * sizeof(T)) +
                            (ss ? B : 1) * pr.nb * 40.0, st);
  if (pr.kind == NRE_AMP_MATERN_MODEL)
    k_amp_vjp_matern<T><<<B, amp_threads(pr.nb), 0, st>>>(pr, state, ss, partials, nparts, base_h, bhs, out_h, ohs,
                                                         dot);
  else
    k_amp_vjp<T><<<B, amp_threads(pr.nb), 0, st>>>(pr, state, ss, partials, nparts, base_h, bhs, out_h, ohs, dot);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  return NRE_OK;
}

template <typename T>
int amp_jacobian(const AmpPrior& pr, const double* state, int nh, T* eye, double* Jt, float* G, float* Gt,
                 cudaStream_t st) {
  prof_begin("amp_jacobian", (double)nh * nh * sizeof(T), st);
  k_eye<T><<<304, 256, 0, st>>>(eye, nh);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  NRE_TRY(amp_jvp<T>(pr, state, 0, eye, nh, Jt, nh, st));
  prof_begin("amp_jacobian", (double)nh * pr.nb * 16.0, st);
  k_jac_store<<<304, 256, 0, st>>>(Jt, nh, pr.nb, G, Gt);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  return NRE_OK;
}

template <typename T>
int amp_jvp_lin(const float* G, int nb, int nh, const T* dh, int64_t dhs, double* dA, int B, cudaStream_t st,
                double* gzero, int64_t gs) {
  prof_begin("amp_jvp", (double)nb * nh * 4 * (gs ? B : 1) + (double)B * (nh * sizeof(T) + nb * 8), st);
  k_amp_jvp_lin<T><<<dim3((nb + 7) / 8, B), 256, 0, st>>>(G, gs, nb, nh, dh, dhs, dA, gzero);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  return NRE_OK;
}

template <typename T>
int amp_vjp_lin(const float* Gt, int nb, int nh, const double* gsum, const T* base_h, int64_t bhs, T* out_h,
                int64_t ohs, int B, cudaStream_t st, double* dot, int64_t gs) {
  prof_begin("amp_vjp", (double)nb * nh * 4 * (gs ? B : 1) + (double)B * (8.0 * nb + (base_h ? 2 : 1) * nh * sizeof(T)),
             st);
  k_amp_vjp_lin<T><<<dim3((nh + 31) / 32, B), 256, 0, st>>>(Gt, gs, nb, nh, gsum, base_h, bhs, out_h, ohs, dot);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  return NRE_OK;
}

#define NRE_INST(T)                                                                              \
  template int amp_forward<T>(const AmpPrior&, const T*, int64_t, double*, int, cudaStream_t);   \
  template int amp_jvp<T>(const AmpPrior&, const double*, int64_t, const T*, int64_t, double*,   \
                          int, cudaStream_t);                                                    \
  template int amp_vjp<T>(const AmpPrior&, const double*, int64_t, const double*, int, const T*, \
                          int64_t, T*, int64_t, int, cudaStream_t, double*);                      \
  template int amp_jacobian<T>(const AmpPrior&, const double*, int, T*, double*, float*, float*,       \
                               cudaStream_t);                                                          \
  template int amp_jvp_lin<T>(const float*, int, int, const T*, int64_t, double*, int, cudaStream_t,    \
                              double*, int64_t);                                                      \
  template int amp_vjp_lin<T>(const float*, int, int, const double*, const T*, int64_t, T*, int64_t, int, \
                              cudaStream_t, double*, int64_t);
NRE_INST(float)
NRE_INST(double)
#undef NRE_INST

}  // namespace nre
