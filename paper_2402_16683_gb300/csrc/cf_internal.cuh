// Correlated-field plan internals: geometry, amplitude lookup and the fused
// prologue / middle / epilogue operations applied around the Hartley sweeps.
//
// The unnormalised multi-dimensional Hartley transform (Sec. "Gaussian
// Processes", FT of s = FT o sqrt(P) o xi, read as a DHT) is computed as
//     H = P o H_0 o ... o H_{D-1},
// one 1-D DHT per axis plus the reflection combination
//     D = 2:  P = (I + R_0 + R_1 - R_0 R_1) / 2
//     D = 3:  P = (R_0 + R_1 + R_2 - R_0 R_1 R_2) / 2
// (R_d negates the index on axis d), which follows from
// cas(sum_d a_d) = Re[(1 - i) prod_d exp(i a_d)] and
// exp(i a) = [(1 + i) cas(a) + (1 - i) cas(-a)] / 2.  P commutes with every H_d,
// so it is applied in a row sweep (last axis), where a CTA holds every row of a
// reflection orbit.  Each 1-D DHT of two real lines a, b is one complex FFT of
// a + i b followed by the Hartley unpack.
#pragma once

#include "common.cuh"
#include "fft.cuh"

namespace nre {

enum { AMPV_FIXED = 0, AMPV_MODEL = 1, AMPV_PIX = 2, AMPV_TAB = 3 };

// Per-sample amplitude model state (doubles), see amp.cu.
enum { AS_THFL = 0, AS_THSL = 1, AS_THFX = 2, AS_THAS = 3, AS_S = 4, AS_HDR = 8 };
inline __host__ __device__ int amp_state_size(int nb) { return AS_HDR + 5 * nb; }
inline __host__ __device__ int as_a(int nb) { return AS_HDR; }
inline __host__ __device__ int as_c(int nb) { return AS_HDR + nb; }
inline __host__ __device__ int as_A(int nb) { return AS_HDR + 2 * nb; }
inline __host__ __device__ int as_xi1(int nb) { return AS_HDR + 3 * nb; }
inline __host__ __device__ int as_xi2(int nb) { return AS_HDR + 4 * nb; }

struct Geo {
  int ndim;
  int l2[3];  // log2 of the axis lengths, last axis fastest
  // squared folded harmonic radius q = sum_d m_d^2 of pixel `flat`
  __device__ __forceinline__ int q_of(int64_t flat) const {
    int q = 0;
    for (int d = ndim - 1; d >= 0; --d) {
      const int n = 1 << l2[d];
      const int i = (int)(flat & (n - 1));
      flat >>= l2[d];
      const int m = i <= (n >> 1) ? i : i - n;
      q += m * m;
    }
    return q;
  }
};

// Amplitude A_full at a harmonic pixel.
template <typename T>
struct AmpView {
  int mode;                // AMPV_FIXED, AMPV_MODEL or AMPV_PIX
  const T* afull;          // FIXED and PIX: A per pixel [N]
  const double* abin;      // MODEL: A per bin of sample b at abin + b * astride
  int64_t astride;         // 0: shared by all samples
  double a0;               // MODEL: amplitude of the zero mode
  const uint16_t* lut;     // MODEL: bin of q (0xFFFF: zero mode)
  const int16_t* bpix;     // PIX (and TAB when set): bin per pixel (-1: zero mode)
  const T* tab;            // TAB: A per bin of this CTA's sample, in shared memory
  T a0t;                   // TAB: a0 in T
  Geo geo;
  __device__ __forceinline__ int bin(int64_t flat) const {
    if (bpix != nullptr && mode != AMPV_MODEL) return (int)__ldg(&bpix[flat]);
    const int q = geo.q_of(flat);
    return q == 0 ? -1 : (int)__ldg(&lut[q]);
  }
  // With `stab` (this CTA's per-bin table in shared memory) the per-bin modes
  // read A from it.
  __device__ __forceinline__ T amp_t(int b, int64_t flat, int bn, const T* stab) const {
    if (stab != nullptr && mode != AMPV_FIXED) return bn < 0 ? a0t : stab[bn];
    return amp(b, flat, bn);
  }
  // PIX without a per-pixel array (the KL's per-point views) reads the
  // per-bin table of sample b through the per-pixel bins.
  __device__ __forceinline__ T amp(int b, int64_t flat, int bn) const {
    if (mode == AMPV_TAB) return bn < 0 ? a0t : tab[bn];
    if (mode == AMPV_FIXED || (mode == AMPV_PIX && afull != nullptr)) return __ldg(&afull[flat]);
    return bn < 0 ? T(a0) : T(__ldg(&abin[b * astride + bn]));
  }
  __device__ __forceinline__ bool binned() const { return mode != AMPV_FIXED; }
};

enum { PRO_BUF = 0, PRO_AMP = 1, PRO_SQRTW = 2 };

// Value entering the first transform at (sample b, pixel flat).
template <typename T>
struct Pro {
  int mode;
  const T* x;         // input, sample b at x + b * xs
  int64_t xs;
  const T* xi_p;      // PRO_AMP with dA: expansion point field, sample b at xi_p + b * ps
  int64_t ps;
  const double* dA;   // PRO_AMP: per-sample dA bins (nullptr: none)
  int nb;
  const T* w;         // PRO_SQRTW: weights [N]
  const T* sdA;       // dA of this CTA's sample in shared memory (set by the kernel)
  AmpView<T> av;
  __device__ __forceinline__ T load(int b, int64_t flat) const { return apply(b, flat, x[b * xs + flat]); }
  // The prologue of the input value v = x[b][flat] (already loaded); stab /
  // stdA: per-bin A and dA of this CTA's sample in shared memory, or nullptr.
  __device__ __forceinline__ T apply(int b, int64_t flat, T v, const T* stab = nullptr,
                                     const T* stdA = nullptr) const {
    if (mode == PRO_BUF) return v;
    if (mode == PRO_SQRTW) return sqrt(__ldg(&w[flat])) * v;
    const int bn = av.binned() ? av.bin(flat) : -1;
    const T xv = dA != nullptr ? xi_p[b * ps + flat] : T(0);  // loaded alongside the bin, not after it
    T u = av.amp_t(b, flat, bn, stab) * v;
    if (dA != nullptr && bn >= 0) u += (stdA ? stdA[bn] : T(__ldg(&dA[b * nb + bn]))) * xv;
    return u;
  }
  // Values at flat and flat + 1 (flat even) as one complex pair.
  __device__ __forceinline__ typename CplxT<T>::type load2(int b, int64_t flat) const {
    typedef typename CplxT<T>::type C;
    if (mode == PRO_BUF) return *reinterpret_cast<const C*>(x + b * xs + flat);
    return cmake<C>(load(b, flat), load(b, flat + 1));
  }
};

enum { EPI_BUF = 0, EPI_OFFSET = 1, EPI_WEIGHT = 2, EPI_AMP = 3 };

// Consumer of the last transform's output at (sample b, pixel flat).
// Partials of the fused metric-product inner product per sample: one per CTA
// of the last sweep (at most 128) at [0, 128), the hyper-parameter part at
// [128, 160) (one per CTA of the amplitude VJP; unused entries are zero).
constexpr int kDotStride = 160;
constexpr int kDotHyper = 128;

template <typename T>
struct Epi {
  int mode;
  T* y;               // output, sample b at y + b * ys
  int64_t ys;
  double offset;      // EPI_OFFSET / EPI_WEIGHT: offset_mean
  // EPI_WEIGHT: Fisher weight from cf = offset + value
  int lik_kind, response;
  double sig_or_scale;
  const T* mask;      // [N] or nullptr
  // EPI_AMP: y = base + A * value; hist[bin] += xi_p * value
  const T* base;
  int64_t bs;
  const T* xi_p;
  int64_t ps;
  int bins;           // accumulate the per-bin sums
  AmpView<T> av;
  // EPI_AMP with bins: when set, the complete per-bin sums go into gsum[b][nb]
  // (so that the reader sums nothing): every CTA writes its partial; the last
  // CTA of each group of kBinGroup consecutive CTAs to finish adds its group's
  // partials, and the last group to finish adds the group sums, each in a
  // fixed order (counters gcnt[b * kGcntStride + ...], zero on entry and left
  // zero)
  double* gsum;
  unsigned* gcnt;
  // EPI_AMP with base, last sweep of a metric product: per-CTA partials of
  // sum(base * y) at dot[b * kDotStride + cta] (row sweeps of 2-D / 3-D grids;
  // other sweeps leave them to a separate reduction)
  double* dot;

  // Writes the output of pixel `flat` of sample b.  EPI_AMP with bins also
  // returns the pixel's contribution xi_p * value to its log-|k| bin (bn = -1:
  // none); the caller reduces the contributions.
  __device__ __forceinline__ void store(int b, int64_t flat, T val, int& bn_out, T& contrib) const {
    store_b(b, flat, val, (mode == EPI_AMP && base != nullptr) ? base[b * bs + flat] : T(0), bn_out, contrib);
  }
  // As store, with the EPI_AMP base value already loaded.
  // Returns the value written.
  __device__ __forceinline__ T store_b(int b, int64_t flat, T val, T bval, int& bn_out, T& contrib,
                                       const T* stab = nullptr) const {
    bn_out = -1;
    contrib = T(0);
    if (mode == EPI_BUF) {
      y[b * ys + flat] = val;
      return val;
    } else if (mode == EPI_OFFSET) {
      y[b * ys + flat] = T(offset) + val;
      return T(offset) + val;
    } else if (mode == EPI_WEIGHT) {
      const T cf = T(offset) + val;
      T w;
      if (lik_kind == NRE_LIK_POISSON) {
        w = T(sig_or_scale) * exp(cf);
      } else {
        const T inv = T(1.0 / (sig_or_scale * sig_or_scale));
        if (response == NRE_RESP_EXP) {
          const T s = exp(cf);
          w = s * s * inv;
        } else {
          w = inv;
        }
        if (mask != nullptr) w *= __ldg(&mask[flat]);
      }
      y[b * ys + flat] = w;
      return w;
    } else {
      const int bn = av.binned() ? av.bin(flat) : -1;
      const T xv = bins ? xi_p[b * ps + flat] : T(0);  // loaded alongside the bin, not after it
      const T o = av.amp_t(b, flat, bn, stab) * val + bval;
      y[b * ys + flat] = o;
      if (bins && bn >= 0) {
        bn_out = bn;
        contrib = xv * val;
      }
      return o;
    }
  }
  // Outputs at flat and flat + 1 (flat even).
  __device__ __forceinline__ void store2(int b, int64_t flat, T v0, T v1, int (&bn)[2], T (&c)[2]) const {
    if (mode == EPI_BUF) {
      *reinterpret_cast<typename CplxT<T>::type*>(y + b * ys + flat) = cmake<typename CplxT<T>::type>(v0, v1);
      bn[0] = bn[1] = -1;
      c[0] = c[1] = T(0);
      return;
    }
    store(b, flat, v0, bn[0], c[0]);
    store(b, flat + 1, v1, bn[1], c[1]);
  }
};

// Middle operation between the two transforms of the metric: t = w * y, the
// weights of sample b at w + b * ws (ws = 0: one weight array for the batch;
// ws = N: a linearisation point per sample, as in the KL's averaged metric).
template <typename T>
struct Mid {
  const T* w;  // [N] or [B][N]
  int64_t ws;
  __device__ __forceinline__ T at(int b, int64_t flat) const { return __ldg(&w[b * ws + flat]); }
  __device__ __forceinline__ T apply(int b, int64_t flat, T y) const { return at(b, flat) * y; }
  __device__ __forceinline__ typename CplxT<T>::type apply2(int b, int64_t flat, T y0, T y1) const {
    typedef typename CplxT<T>::type C;
    const C ww = __ldg(reinterpret_cast<const C*>(w + b * ws + flat));
    return cmake<C>(ww.x * y0, ww.y * y1);
  }
};

// A CTA's per-bin sums, from nreg warp-private histograms (region r at
// hist + r * rstride, folded in region order in the histograms' type H), as
// partial `part` of nparts for sample b at partials[(b * nparts + part) * nb]
// (FP64); with e.gsum the partials are kept as pairs (sum, error) of H in the
// same slots (the buffer read as H) and added in two fixed-order levels (the
// CTAs of a group of kBinGroup, then the groups) into e.gsum[b * nb] (see
// Epi::gsum).  All additions are compensated, so FP32 histograms fold to about
// FP64 accuracy.  Called by all threads of the CTA after
// its last histogram update, with a __syncthreads() before.
// CTAs per group of the in-place bin sums, and the arrival counters per sample
// (one for the groups, one per group; up to 128 CTAs per sample).
constexpr int kBinGroup = 8;
constexpr int kGcntStride = 1 + 128 / kBinGroup;

// Compensated (Neumaier) addition of x into s with the rounding errors
// collected in c: s + c carries the sum to about twice the working precision.
template <typename H>
__device__ __forceinline__ void comp_add(H& s, H& c, H x) {
  const H t = s + x;
  c += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
  s = t;
}

// The two reduction levels of fold_bins for the in-place sums, out of line so
// that the sweeps' main loops keep their registers.  hp: the partial pairs.
template <typename H>
__device__ __noinline__ void bins_complete(H* hp, double* gsum, unsigned* gcnt, int b, int nparts, int part,
                                           int nb) {
  // the last CTA of the group adds the group's partials into the slot of
  // its first CTA; the last group then adds the group sums
  const int g = part / kBinGroup, ng = (nparts + kBinGroup - 1) / kBinGroup;
  const int g0 = g * kBinGroup, gn = min(kBinGroup, nparts - g0);
  unsigned* cnt = gcnt + (int64_t)b * kGcntStride;
  const H* src = hp + 2 * ((int64_t)b * nparts * nb);
  H* gdst = hp + 2 * (((int64_t)b * nparts + g0) * nb);
  // Arrival: the CTA's partial (written by all its threads, ordered before
  // thread 0 by the barrier) is released by thread 0's fence before its
  // counter add; only thread 0 fences, so the other warps do not wait for
  // their own outstanding output stores.
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&cnt[1 + g], 1u) == (unsigned)(gn - 1);
    if (s_last) __threadfence();  // acquire the other CTAs' partials
  }
  __syncthreads();
  if (!s_last) return;
  // the group's partials from L2 (ld.global.cg: not through this SM's L1), all
  // in flight at once, added in CTA order
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    H ps[kBinGroup], pc[kBinGroup];
#pragma unroll
    for (int u = 0; u < kBinGroup; ++u) {
      const int64_t o = 2 * ((int64_t)(g0 + u) * nb + i);
      ps[u] = u < gn ? __ldcg(&src[o]) : H(0);
      pc[u] = u < gn ? __ldcg(&src[o + 1]) : H(0);
    }
    H s = H(0), c = H(0);
#pragma unroll
    for (int u = 0; u < kBinGroup; ++u) {
      comp_add(s, c, ps[u]);
      c += pc[u];
    }
    gdst[2 * i] = s;
    gdst[2 * i + 1] = c;
  }
  __syncthreads();  // the group sum, then the group's arrival (released as above)
  if (threadIdx.x == 0) {
    cnt[1 + g] = 0u;
    __threadfence();
    s_last = atomicAdd(&cnt[0], 1u) == (unsigned)(ng - 1);
    if (s_last) __threadfence();
  }
  __syncthreads();
  if (!s_last) return;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    H s = H(0), c = H(0);
    for (int q0 = 0; q0 < ng; q0 += kBinGroup) {
      H ps[kBinGroup], pc[kBinGroup];
#pragma unroll
      for (int u = 0; u < kBinGroup; ++u) {
        const int64_t o = 2 * ((int64_t)(q0 + u) * kBinGroup * nb + i);
        ps[u] = q0 + u < ng ? __ldcg(&src[o]) : H(0);
        pc[u] = q0 + u < ng ? __ldcg(&src[o + 1]) : H(0);
      }
#pragma unroll
      for (int u = 0; u < kBinGroup; ++u) {
        comp_add(s, c, ps[u]);
        c += pc[u];
      }
    }
    gsum[(int64_t)b * nb + i] = double(s) + double(c);
  }
  if (threadIdx.x == 0) cnt[0] = 0u;
}

template <typename T, typename H>
__device__ __forceinline__ void fold_bins(const Epi<T>& e, double* partials, int b, int nparts, int part,
                                          const H* hist, int nreg, int rstride, int nb) {
  // the warps' histograms in warp order, in the histograms' type with the
  // rounding errors carried along (the FP64 units of this part run at a small
  // fraction of the FP32 rate)
  if (e.gsum == nullptr) {
    double* dst = partials + ((int64_t)b * nparts + part) * nb;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
      H s = H(0), c = H(0);
      for (int r = 0; r < nreg; ++r) comp_add(s, c, hist[r * rstride + i]);
      dst[i] = double(s) + double(c);
    }
    return;
  }
  // complete sums in place: each CTA's partial as a pair (sum, error) of H in
  // the buffer's slot, the last CTA adds them
  H* hp = reinterpret_cast<H*>(partials);
  H* dst = hp + 2 * (((int64_t)b * nparts + part) * nb);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    H s = H(0), c = H(0);
    for (int r = 0; r < nreg; ++r) comp_add(s, c, hist[r * rstride + i]);
    dst[2 * i] = s;
    dst[2 * i + 1] = c;
  }
  bins_complete<H>(hp, e.gsum, e.gcnt, b, nparts, part, nb);
}

// Arguments of one row sweep (last axis, length L).
template <typename T>
struct RowArgs {
  int L, log2L, log2Lmax;
  const typename CplxT<T>::type* tw;
  int pm;              // 1, 2 or 3: grid dimensionality (P combination)
  int n_units;         // PM >= 2: row groups per sample; PM == 1: sample pairs
  int nU;              // units per CTA iteration
  int B;               // batch
  const int* grows;    // PM >= 2: rows of group g at grows[g * G + s]
  const int* gflags;   // PM >= 2: bit0 = R_0 swaps slots in a line, bit1 = R_1 swaps lines
  Pro<T> pro;
  Epi<T> epi;
  Mid<T> mid;
  int nb;              // bins of the histogram (epi.bins)
  double* partials;    // [B][gridDim.x][nb] (PM >= 2) or [B][1][nb] (PM == 1)
  unsigned* status;    // count of bounded waits that ran out (may be null)
};

// Arguments of one sweep along a non-contiguous axis.
template <typename T>
struct ColArgs {
  int L, log2L, log2Lmax;
  const typename CplxT<T>::type* tw;
  int64_t inner;       // product of the axis lengths after this axis
  int W;               // grid columns per unit (even, divides inner)
  int64_t nblk;        // inner / W
  int64_t n_units;     // outer * nblk
  Pro<T> pro;
  Epi<T> epi;
  Mid<T> mid;
  int nb;
  double* partials;    // [B][gridDim.x][nb]
};

}  // namespace nre

// The opaque plan of the C ABI.
struct nre_cf_plan {
  int ndim = 0, dtype = NRE_F32;
  int n[3] = {1, 1, 1}, l2[3] = {0, 0, 0};
  int64_t N = 0, nrows = 0;
  int Lmax = 0, log2Lmax = 0;
  int amp_kind = 0;
  double offset_mean = 0.0, offset_std = 1.0;
  int n_bins = 0, n_hyper = 0;
  int64_t latent = 0, stride = 0;
  // prior of the power model: log-normal (mu, s) and slope (mean, std)
  double mu_fl = 0, s_fl = 0, mu_fx = 0, s_fx = 0, mu_as = 0, s_as = 0, sl_m = 0, sl_s = 0;
  // prior of the Matern model: scale and cutoff log-normal, slope (mean, std)
  double mu_sc = 0, s_sc = 0, mu_ct = 0, s_ct = 0, al_m = 0, al_s = 0;
  int n_groups = 0, G = 1;
  nre::DevBuf tw;        // complex twiddles, Lmax entries, plan dtype
  nre::DevBuf afull;     // fixed kinds: A_full [N], plan dtype
  nre::DevBuf lut;       // model: uint16 bin of q
  nre::DevBuf centres;   // model: double[n_bins]
  nre::DevBuf counts;    // model: double[n_bins]
  nre::DevBuf grows;     // int[n_groups * G]
  nre::DevBuf gflags;    // int[n_groups]
  // workspaces grown on demand by the cf_* calls
  nre::DevBuf ws_tmp0, ws_tmp1, ws_state, ws_dA, ws_part;
};

namespace nre {

// Amplitude models with hyper-parameters on log-|k| bins (the power model and
// the Matern model): every per-bin table, bin sum and Jacobian path serves both.
inline bool binned_model(const nre_cf_plan* p) {
  return p->amp_kind == NRE_AMP_POWER_MODEL || p->amp_kind == NRE_AMP_MATERN_MODEL;
}

// Amplitude-model kernels (amp.cu)
struct AmpPrior {
  int kind;  // NRE_AMP_POWER_MODEL or NRE_AMP_MATERN_MODEL
  double mu_fl, s_fl, mu_fx, s_fx, mu_as, s_as, sl_m, sl_s;  // power model
  double mu_sc, s_sc, mu_ct, s_ct, al_m, al_s;               // Matern model
  const double* centres;
  const double* counts;
  int nb;
};
AmpPrior amp_prior_of(const nre_cf_plan* p);
// state[b] from the hyper-latents at h + b * hs (n_hyper doubles or floats).
template <typename T>
int amp_forward(const AmpPrior& pr, const T* h, int64_t hs, double* state, int B, cudaStream_t st);
// dA[b] = JVP at state (sample b at state + b * ss) in direction dh[b].
template <typename T>
int amp_jvp(const AmpPrior& pr, const double* state, int64_t ss, const T* dh, int64_t dhs,
            double* dA, int B, cudaStream_t st);
// out_h[b] = base_h[b] (optional) + VJP at state of gA[b] = sum_c partials[b][c][:].
// With `dot` (and a base): dot[b * kDotStride + kDotHyper] = sum(base_h * out_h).
template <typename T>
int amp_vjp(const AmpPrior& pr, const double* state, int64_t ss, const double* partials,
            int nparts, const T* base_h, int64_t bhs, T* out_h, int64_t ohs, int B,
            cudaStream_t st, double* dot = nullptr);

// Linearised amplitude model at an expansion point (FP32 path): the Jacobian
// from nh JVPs along the unit vectors (eye: [nh][nh] scratch, Jt: [nh][nb] FP64
// scratch), stored as G [nb][nhp] and Gt [nh][nbp] floats (rows zero-padded to
// multiples of 4); then dA = G dh and out_h = base_h + Gt-contractions of the
// complete per-bin sums gsum [B][nb] (as amp_jvp / amp_vjp; nb, nh <= 1024).
template <typename T>
int amp_jacobian(const AmpPrior& pr, const double* state, int nh, T* eye, double* Jt, float* G, float* Gt,
                 cudaStream_t st);
// gs: float stride of the matrix between batch entries (0: one matrix for the
// batch; the KL metric's samples each have their own expansion point).
template <typename T>
int amp_jvp_lin(const float* G, int nb, int nh, const T* dh, int64_t dhs, double* dA, int B, cudaStream_t st,
                double* gzero = nullptr,  // gzero: [B][nb] set to 0 (the next sweep's in-place bin sums)
                int64_t gs = 0);
template <typename T>
int amp_vjp_lin(const float* Gt, int nb, int nh, const double* gsum, const T* base_h, int64_t bhs, T* out_h,
                int64_t ohs, int B, cudaStream_t st, double* dot = nullptr, int64_t gs = 0);

// Sweep chains (sweeps.cu).  Runs one Hartley transform (mid == nullptr) or the
// metric's transform pair with t = w * y between them (mid != nullptr) over a
// batch, fusing the prologue into the first sweep and the epilogue into the
// last.  tmp0/tmp1 hold B * N elements each.  *nparts receives the number of
// histogram partials per sample written by the last sweep.
template <typename T>
int run_hartley(const nre_cf_plan* p, int B, const Pro<T>& pro, const Epi<T>& epi,
                const Mid<T>* mid, T* tmp0, T* tmp1, double* partials, int* nparts,
                cudaStream_t st);
// Maximum number of histogram partials per sample of any sweep of the plan.
int max_parts(const nre_cf_plan* p);
// Workspace growth helper.
int ensure(DevBuf& b, size_t bytes);

template <typename T>
AmpView<T> amp_view(const nre_cf_plan* p, const double* abin, int64_t astride);

}  // namespace nre
