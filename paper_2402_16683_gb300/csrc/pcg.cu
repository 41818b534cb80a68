// Preconditioned CG on the correlated-field metric (metric_set_precond).
//
// With the weight w replaced by its mean w_bar and H H = N I, the metric in
// harmonic coordinates is "diagonal + low rank":
//     M~ = [[D, B], [B^T, C]],  D = I + c A^2 (c = N w_bar),
//     B = c diag(A xi_p) G_full,  C = I + c G_full^T diag(xi_p^2) G_full,
// with G_full[k][h] = dA_{bin(k)}/dh.  Its exact inverse by the Schur
// complement on the hyper block, S = C - B^T D^-1 B = I + c G^T diag(U) G with
// U_b = sum_{k in b} xi_p[k]^2 / D_k (G = dA/dh per bin), is applied as
//     y = r_f / D,  t_b = sum_{k in b} A_k xi_p[k] y_k,
//     z_h = S^-1 (r_h - c G^T t),   g = G z_h,
//     z_f = (r_f - c A xi_p g_bin) / D.
// The constant-weight approximation is exact for w = const and spectrally close
// when w varies smoothly; for a sparse observation mask it is not (see the
// design notes).  Preconditioned CG (x_0 = 0, r_0 = b, z = P r, p = z,
// alpha = r.z / p.Mp, beta = r'.z' / r.z) stops on the unpreconditioned
// recursive residual ||r|| <= rtol ||b||; inner products are FP64, the small
// dense preconditioner products FP32.
#include <cmath>
#include <vector>

#include "metric_internal.cuh"
#include "regfft.cuh"

using namespace nre;

namespace {

constexpr int PC_THREADS = 256;
// SC_XALPHA: the update kernel's alpha, whose step x += alpha p the p-update
// kernel applies (it reads p anyway: one vector read less per iteration).
enum { SC_RR = CG_SC_RR, SC_BB = CG_SC_BB, SC_RZ = 2, SC_BETA = 3, SC_ACTIVE = CG_SC_ACTIVE,
       SC_ITERS = CG_SC_ITERS, SC_XALPHA = 6, SC_N = CG_SC_N };

// Blocks per system of the vector kernels: about four waves of the device's SMs
// over the whole batch (enough loads in flight, few partials to fold), at
// least 4 vectors per thread and at most 64 blocks.
// Dynamic shared memory beyond the 48 KB default with the static (warp-private
// histograms of up to 1024 bins).
template <typename K>
int pc_smem(K k, size_t bytes) {
  return raise_smem(k, bytes);
}

int pc_blocks(int64_t n, int B) {
  int64_t nb = (4 * (int64_t)sm_count() + B - 1) / B;
  const int64_t cap = (n + PC_THREADS * 16 - 1) / (PC_THREADS * 16);
  if (nb > cap) nb = cap;
  if (nb > 64) nb = 64;
  if (nb < 1) nb = 1;
  return (int)nb;
}

template <typename T>
struct PCArgs {
  int64_t N;            // field entries (the rest of the latent vector is hyper)
  const double* cdev;   // N * mean(w) on the device (read at run time, so that
                        // captured launches follow a re-linearised metric)
  AmpView<T> av;        // amplitude at the expansion point (set-up only)
  const T* xi_p;        // expansion point (set-up only)
  const T* invD;        // [N] 1 / D_k = 1 / (1 + c A_k^2)
  const T* e;           // [N] A_k xi_p[k] / D_k (nb > 0)
  const int16_t* bpix;  // [N] log-|k| bin (nb > 0)
  int nb;               // bins (0: fixed amplitude, no hyper block)
  double* bin_part;     // [B][gridDim.x][nb] partial sums t_b
  const double* gz;     // [B][nb]
};

template <typename T>
__device__ void partial_out(const RunSum<T>& acc, double* part) {
  const double t = acc.block_sum();
  if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// 16-byte vector of T.
template <typename T>
struct alignas(16) PV {
  static constexpr int W = 16 / sizeof(T);
  T e[W];
};
template <typename T>
__device__ __forceinline__ PV<T> ldp(const T* p) { return *reinterpret_cast<const PV<T>*>(p); }
template <typename T>
__device__ __forceinline__ void stp(T* p, const PV<T>& v) { *reinterpret_cast<PV<T>*>(p) = v; }

// Grid-stride loop of the CTAs of system blockIdx.y over the n entries in
// vectors of W = 16 / sizeof(T); the trip count is uniform over the block
// (the warp reductions of the bins need whole warps).  f(i, full) handles
// entries i .. i+W-1 (full) or the entries i.. below n (tail; i may be >= n).
template <typename T, class F>
__device__ __forceinline__ void for_pv(int64_t n, F f) {
  constexpr int W = PV<T>::W;
  const int64_t step = (int64_t)gridDim.x * blockDim.x * W;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x * W; base < n; base += step) {
    const int64_t i = base + (int64_t)threadIdx.x * W;
    f(i, i + W <= n);
  }
}

// t_b += e_k v_k for the W entries from i (field entries only: N is a multiple
// of W, so a vector is all field or all hyper).  Called by every lane.
template <typename T>
__device__ __forceinline__ void bins_add(const PCArgs<T>& pc, int64_t i, const T (&v)[PV<T>::W], double* hist) {
  constexpr int W = PV<T>::W;
  int key[W];
  T val[W];
  const bool in = i + W <= pc.N;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    key[k] = in ? (int)__ldg(&pc.bpix[i + k]) : -1;
    val[k] = in ? __ldg(&pc.e[i + k]) * v[k] : T(0);
  }
  add_slots<W, T>(key, val, hist);
}

// The block's bin sums from its warps' private histograms (hist + w nb),
// folded in warp order, as partial blockIdx.x of system b.
template <typename T>
__device__ __forceinline__ void bins_out(const PCArgs<T>& pc, int b, const double* hist) {
  __syncthreads();
  double* dst = pc.bin_part + ((int64_t)b * gridDim.x + blockIdx.x) * pc.nb;
  const int nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < pc.nb; i += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += hist[w * pc.nb + i];
    dst[i] = t;
  }
}

// x = 0, r = b; partials of r.r and of the bins of r.
template <typename T>
__global__ void __launch_bounds__(PC_THREADS) k_pcg_init(const T* bsrc, T* x, T* r, int64_t n, int64_t S,
                                                        double* rr_part, PCArgs<T> pc) {
  extern __shared__ double hist[];
  constexpr int W = PV<T>::W;
  const int b = blockIdx.y;
  // warp-private bin histograms of nb entries (see warp_run_add)
  for (int i = threadIdx.x; i < (PC_THREADS / 32) * pc.nb; i += blockDim.x) hist[i] = 0.0;
  double* whist = hist + (threadIdx.x >> 5) * pc.nb;
  __syncthreads();
  const int64_t off = (int64_t)b * S;
  RunSum<T> acc;
  for_pv<T>(n, [&](int64_t i, bool full) {
    T v[W];
    T run = T(0);
    if (full) {
      const PV<T> bv = ldp(bsrc + off + i);
      PV<T> z;
#pragma unroll
      for (int k = 0; k < W; ++k) {
        v[k] = bv.e[k];
        z.e[k] = T(0);
        run += v[k] * v[k];
      }
      stp(x + off + i, z);
      stp(r + off + i, bv);
    } else {
#pragma unroll
      for (int k = 0; k < W; ++k) {
        v[k] = T(0);
        if (i + k < n) {
          v[k] = bsrc[off + i + k];
          x[off + i + k] = T(0);
          r[off + i + k] = v[k];
          run += v[k] * v[k];
        }
      }
    }
    acc.add(run);
    if (pc.nb > 0) bins_add(pc, i, v, whist);
  });
  partial_out(acc, rr_part);
  if (pc.nb > 0) bins_out(pc, b, hist);
}

// alpha = r.z / p.q (p.q from npq partials per system), kept in SC_XALPHA
// for the p-update kernel's x += alpha p; r -= alpha q; partials of r.r and
// of the bins of r.
template <typename T>
__global__ void __launch_bounds__(PC_THREADS) k_pcg_update(T* r, const T* q, int64_t n, int64_t S, double* sc,
                                                          const double* pq_part,
                                                          int npq, double* rr_part, PCArgs<T> pc) {
  extern __shared__ double hist[];
  constexpr int W = PV<T>::W;
  const int b = blockIdx.y;
  // warp-private bin histograms of nb entries (see warp_run_add)
  for (int i = threadIdx.x; i < (PC_THREADS / 32) * pc.nb; i += blockDim.x) hist[i] = 0.0;
  double* whist = hist + (threadIdx.x >> 5) * pc.nb;
  __syncthreads();
  double* c = sc + b * SC_N;
  const bool active = c[SC_ACTIVE] != 0.0;
  __shared__ T s_alpha;  // one FP64 division per block, not per thread
  const double pq = block_sum_array(pq_part + (int64_t)b * npq, npq);
  if (threadIdx.x == 0) {
    const T al = T(active && pq != 0.0 ? c[SC_RZ] / pq : 0.0);
    s_alpha = al;
    if (blockIdx.x == 0) c[SC_XALPHA] = double(al);
  }
  __syncthreads();
  const T alpha = s_alpha;
  const int64_t off = (int64_t)b * S;
  RunSum<T> acc;
  for_pv<T>(n, [&](int64_t i, bool full) {
    T v[W];
    T run = T(0);
    if (full) {
      PV<T> ri = ldp(r + off + i);
      if (active) {
        const PV<T> qi = ldp(q + off + i);
#pragma unroll
        for (int k = 0; k < W; ++k) ri.e[k] -= alpha * qi.e[k];
        stp(r + off + i, ri);
      }
#pragma unroll
      for (int k = 0; k < W; ++k) {
        v[k] = ri.e[k];
        run += v[k] * v[k];
      }
    } else {
#pragma unroll
      for (int k = 0; k < W; ++k) {
        v[k] = T(0);
        if (i + k < n) {
          T ri = r[off + i + k];
          if (active) {
            ri -= alpha * q[off + i + k];
            r[off + i + k] = ri;
          }
          v[k] = ri;
          run += ri * ri;
        }
      }
    }
    acc.add(run);
    if (pc.nb > 0) bins_add(pc, i, v, whist);
  });
  partial_out(acc, rr_part);
  if (pc.nb > 0) bins_out(pc, b, hist);
}

// Hyper block of the preconditioner, one CTA per system:
// z_h = S^-1 (r_h - c G t), gz = G^T z_h  (G [nh][nb], Gt = G^T [nb][nh]).
template <typename T>
__global__ void k_pcg_hyper(const T* r, T* z, int64_t S, int64_t N, int nh, int nb, const double* cdev,
                            const float* G, const float* Gt, const float* Sinv, const double* bin_part,
                            int nparts, double* gz) {
  extern __shared__ float sh[];
  float* t = sh;        // [nb]
  float* u = t + nb;    // [nh]
  float* zh = u + nh;   // [nh]
  const int b = blockIdx.x;
  for (int i = threadIdx.x; i < nb; i += blockDim.x)
    t[i] = float(sum_strided(bin_part + (int64_t)b * nparts * nb + i, nparts, nb));
  __syncthreads();
  const T* rh = r + (int64_t)b * S + N;
  const double c = *cdev;
  for (int h = threadIdx.x; h < nh; h += blockDim.x) {
    float s0 = 0.f, s1 = 0.f;
    int i = 0;
    for (; i + 1 < nb; i += 2) {
      s0 += __ldg(&Gt[(int64_t)i * nh + h]) * t[i];
      s1 += __ldg(&Gt[(int64_t)(i + 1) * nh + h]) * t[i + 1];
    }
    if (i < nb) s0 += __ldg(&Gt[(int64_t)i * nh + h]) * t[i];
    u[h] = float(rh[h]) - float(c) * (s0 + s1);
  }
  __syncthreads();
  T* zo = z + (int64_t)b * S + N;
  for (int h = threadIdx.x; h < nh; h += blockDim.x) {
    float s0 = 0.f, s1 = 0.f;
    int k = 0;
    for (; k + 1 < nh; k += 2) {  // S^-1 symmetric: column h read as row h
      s0 += __ldg(&Sinv[(int64_t)k * nh + h]) * u[k];
      s1 += __ldg(&Sinv[(int64_t)(k + 1) * nh + h]) * u[k + 1];
    }
    if (k < nh) s0 += __ldg(&Sinv[(int64_t)k * nh + h]) * u[k];
    zh[h] = s0 + s1;
    zo[h] = T(s0 + s1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    float s0 = 0.f, s1 = 0.f;
    int h = 0;
    for (; h + 1 < nh; h += 2) {
      s0 += __ldg(&G[(int64_t)h * nb + i]) * zh[h];
      s1 += __ldg(&G[(int64_t)(h + 1) * nb + i]) * zh[h + 1];
    }
    if (h < nh) s0 += __ldg(&G[(int64_t)h * nb + i]) * zh[h];
    gz[(int64_t)b * nb + i] = s0 + s1;
  }
}

// Field block z_f = r_f / D - c e gz[bin] ; partials of r.z over the whole
// latent vector (the hyper part of z was written by k_pcg_hyper).  With
// `init`, also p = z.
template <typename T>
__global__ void __launch_bounds__(PC_THREADS) k_pcg_z(const T* r, T* z, T* p, int64_t n, int64_t S,
                                                     double* rz_part, PCArgs<T> pc, int init) {
  __shared__ float sgz[1024];
  constexpr int W = PV<T>::W;
  const int b = blockIdx.y;
  const double cc = *pc.cdev;
  for (int i = threadIdx.x; i < pc.nb; i += blockDim.x) sgz[i] = float(cc * pc.gz[(int64_t)b * pc.nb + i]);
  __syncthreads();
  const int64_t off = (int64_t)b * S;
  RunSum<T> acc;
  for_pv<T>(n, [&](int64_t i, bool full) {
    T run = T(0);
    if (full && i + W <= pc.N) {
      const PV<T> ri = ldp(r + off + i), id = ldp(pc.invD + i);
      PV<T> zi;
      if (pc.nb > 0) {
        const PV<T> ei = ldp(pc.e + i);
#pragma unroll
        for (int k = 0; k < W; ++k) {
          const int bn = __ldg(&pc.bpix[i + k]);
          zi.e[k] = ri.e[k] * id.e[k] - (bn >= 0 ? ei.e[k] * T(sgz[bn]) : T(0));
        }
      } else {
#pragma unroll
        for (int k = 0; k < W; ++k) zi.e[k] = ri.e[k] * id.e[k];
      }
      stp(z + off + i, zi);
      if (init) stp(p + off + i, zi);
#pragma unroll
      for (int k = 0; k < W; ++k) run += ri.e[k] * zi.e[k];
    } else {
#pragma unroll
      for (int k = 0; k < W; ++k) {
        const int64_t j = i + k;
        if (j >= n) continue;
        const T ri = r[off + j];
        T zi;
        if (j < pc.N) {
          zi = ri * pc.invD[j];
          if (pc.nb > 0) {
            const int bn = pc.bpix[j];
            if (bn >= 0) zi -= pc.e[j] * T(sgz[bn]);
          }
          z[off + j] = zi;
        } else {
          zi = z[off + j];
        }
        if (init) p[off + j] = zi;
        run += ri * zi;
      }
    }
    acc.add(run);
  });
  partial_out(acc, rz_part);
}

__global__ void k_pcg_start(double* sc, const double* rr_part, const double* rz_part, int nblk, double rtol) {
  const int b = blockIdx.x;
  if (threadIdx.x != 0) return;
  double rr = 0.0, rz = 0.0;
  for (int i = 0; i < nblk; ++i) {
    rr += rr_part[b * nblk + i];
    rz += rz_part[b * nblk + i];
  }
  double* c = sc + b * SC_N;
  c[SC_RR] = rr;
  c[SC_BB] = rr;
  c[SC_RZ] = rz;
  c[SC_BETA] = 0.0;
  c[SC_XALPHA] = 0.0;
  c[SC_ITERS] = 0.0;
  c[SC_ACTIVE] = (rr > 0.0 && rtol < 1.0) ? 1.0 : 0.0;
}

// x += alpha p (the update kernel's step), then beta = r'.z' / r.z and
// p = z + beta p (every block reads the old r.z; the scalars, the activity
// flag included, are updated by k_pcg_finish afterwards, so a system active
// in the update kernel is active here).
template <typename T>
__global__ void __launch_bounds__(PC_THREADS) k_pcg_pupdate(T* x, T* p, const T* z, int64_t n, int64_t S,
                                                           const double* sc, const double* rz_part, int nblk) {
  constexpr int W = PV<T>::W;
  const int b = blockIdx.y;
  const double* c = sc + b * SC_N;
  if (c[SC_ACTIVE] == 0.0) return;
  __shared__ T s_beta;  // one FP64 division per block, not per thread
  const double rz = block_sum_array(rz_part + (int64_t)b * nblk, nblk);
  if (threadIdx.x == 0) s_beta = T(rz / c[SC_RZ]);
  __syncthreads();
  const T beta = s_beta, xa = T(c[SC_XALPHA]);
  const int64_t off = (int64_t)b * S;
  for_pv<T>(n, [&](int64_t i, bool full) {
    if (full) {
      const PV<T> zi = ldp(z + off + i);
      PV<T> pi = ldp(p + off + i), xi = ldp(x + off + i);
#pragma unroll
      for (int k = 0; k < W; ++k) {
        xi.e[k] += xa * pi.e[k];
        pi.e[k] = zi.e[k] + beta * pi.e[k];
      }
      stp(x + off + i, xi);
      stp(p + off + i, pi);
    } else {
      for (int k = 0; k < W; ++k)
        if (i + k < n) {
          const T pv = p[off + i + k];
          x[off + i + k] += xa * pv;
          p[off + i + k] = z[off + i + k] + beta * pv;
        }
    }
  });
}

__global__ void k_pcg_finish(double* sc, const double* rr_part, const double* rz_part, int nblk, double rtol) {
  const int b = blockIdx.x;
  if (threadIdx.x != 0) return;
  double* c = sc + b * SC_N;
  if (c[SC_ACTIVE] == 0.0) return;
  double rr = 0.0, rz = 0.0;
  for (int i = 0; i < nblk; ++i) {
    rr += rr_part[b * nblk + i];
    rz += rz_part[b * nblk + i];
  }
  c[SC_BETA] = c[SC_RZ] != 0.0 ? rz / c[SC_RZ] : 0.0;
  c[SC_RR] = rr;
  c[SC_RZ] = rz;
  c[SC_ITERS] += 1.0;
  // an exact zero residual ends the system at any rtol (beta would be 0/0 next)
  if (rr == 0.0 || rz == 0.0 || (rtol > 0.0 && sqrt(rr) <= rtol * sqrt(c[SC_BB]))) {
    c[SC_ACTIVE] = 0.0;
    c[SC_BETA] = 0.0;
  }
}

// Partials of p.q.
template <typename T>
__global__ void __launch_bounds__(PC_THREADS) k_dot_p(const T* a, const T* q, int64_t n, int64_t S, double* part) {
  constexpr int W = PV<T>::W;
  const int64_t off = (int64_t)blockIdx.y * S;
  RunSum<T> acc;
  for_pv<T>(n, [&](int64_t i, bool full) {
    T run = T(0);
    if (full) {
      const PV<T> u = ldp(a + off + i), v = ldp(q + off + i);
#pragma unroll
      for (int k = 0; k < W; ++k) run += u.e[k] * v.e[k];
    } else {
      for (int k = 0; k < W; ++k)
        if (i + k < n) run += a[off + i + k] * q[off + i + k];
    }
    acc.add(run);
  });
  partial_out(acc, part);
}

// Per-pixel preconditioner coefficients at the expansion point.
template <typename T>
__global__ void k_pc_pix(PCArgs<T> pc, T* invD, T* e) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < pc.N; i += (int64_t)gridDim.x * blockDim.x) {
    const int bn = pc.av.binned() ? pc.av.bin(i) : -1;
    const double A = double(pc.av.amp(0, i, bn));
    const double D = 1.0 + *pc.cdev * A * A;
    invD[i] = T(1.0 / D);
    if (e) e[i] = (bn >= 0 && pc.nb > 0) ? T(A * double(pc.xi_p[i]) / D) : T(0);
  }
}

// U_b = sum_{k in b} xi_p[k]^2 / D_k (bins of the expansion point), and
// sum w for c = N mean(w): per block into part[blockIdx.x][1 + nb] (entry 0 the
// weight sum), from warp-private histograms folded in warp order; the trip
// count is uniform over the block (warp reductions of the bins).
template <typename T>
__global__ void __launch_bounds__(PC_THREADS) k_pc_setup(const T* w, int64_t N, PCArgs<T> pc, double* part,
                                                        int with_bins) {
  extern __shared__ double hist[];
  const int nbh = (pc.nb > 0 && with_bins) ? pc.nb : 0;
  const double cc = with_bins ? *pc.cdev : 0.0;
  double* whist = hist + (threadIdx.x >> 5) * nbh;
  for (int i = threadIdx.x; i < (PC_THREADS / 32) * nbh; i += blockDim.x) hist[i] = 0.0;
  __syncthreads();
  double acc = 0.0;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < N; i0 += step) {
    const int64_t i = i0 + threadIdx.x;
    const bool act = i < N;
    if (act) acc += double(w[i]);
    if (nbh > 0) {
      const int bn = act ? pc.av.bin(i) : -1;
      double c = 0.0;
      if (bn >= 0) {
        const double A = double(pc.av.amp(0, i, bn));
        const double xp = double(pc.xi_p[i]);
        c = xp * xp / (1.0 + cc * A * A);
      }
      warp_run_add(bn, c, whist);
    }
  }
  __shared__ double red[PC_THREADS / 32];
  const double t = block_sum(acc, red);
  double* dst = part + (int64_t)blockIdx.x * (1 + pc.nb);
  if (threadIdx.x == 0) dst[0] = t;
  __syncthreads();
  for (int i = threadIdx.x; i < pc.nb; i += blockDim.x) {
    double u = 0.0;
    for (int wi = 0; wi < (nbh > 0 ? PC_THREADS / 32 : 0); ++wi) u += hist[wi * nbh + i];
    dst[1 + i] = u;
  }
}

// out[j] = sum over blocks (in block order) of part[blk][j], j < nj.
__global__ void k_pc_setup_sum(const double* part, int nblk, int nj, double* out) {
  for (int j = threadIdx.x; j < nj; j += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * nj + j];
    out[j] = s;
  }
}

// ---------------------------------------------------------------- Schur block
// The preconditioner's hyper block S = I + c G diag(U) G^T (G [nh][nb]) is
// formed and inverted on the device in FP64, so that a set-up never waits for
// the host (serving re-linearises a metric per request).

template <typename T>
__global__ void k_schur_eye(T* e, int nh) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nh * nh) e[t] = (t / nh == t % nh) ? T(1) : T(0);
}

// wb == 0: A = S (nh x nh).  wb == 1: A = K = I + F^T F (nb x nb),
// F[h][b] = G[h][b] sqrt(c U_b).  One entry per thread, sums in index order.
__global__ void k_schur_assemble(const double* G, const double* U, const double* cdev, int nh, int nb, int wb,
                                 double* A) {
  const int n = wb ? nb : nh;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int i = t / n, j = t % n;
  const double c = *cdev;
  double s = 0.0;
  if (wb) {
    for (int h = 0; h < nh; ++h) s += G[(int64_t)h * nb + i] * G[(int64_t)h * nb + j];
    s *= c * sqrt(fmax(U[i], 0.0) * fmax(U[j], 0.0));
  } else {
    for (int b = 0; b < nb; ++b) s += G[(int64_t)i * nb + b] * U[b] * G[(int64_t)j * nb + b];
    s *= c;
  }
  A[t] = s + (i == j ? 1.0 : 0.0);
}

// Inverse of the SPD n x n matrix A (row-major) in three launches:
// k_chol factors A = L L^T in place (lower triangle; one CTA), k_trinv forms
// X = L^-1 (one warp per column), k_gram A^-1 = X^T X.  A pivot that is not
// positive makes k_chol write the identity and flag[0] = 1 (the later kernels
// then copy it through).
__global__ void __launch_bounds__(1024) k_chol(double* A, int n, int* flag) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double d = A[(int64_t)j * n + j];
      if (!(d > 0.0)) bad = 1;
      A[(int64_t)j * n + j] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    if (bad) break;
    const double dj = A[(int64_t)j * n + j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[(int64_t)i * n + j] /= dj;
    __syncthreads();
    // trailing lower triangle: A[i][k] -= L[i][j] L[k][j], j < k <= i
    const int m = n - j - 1;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int i = j + 1 + t / m, k = j + 1 + t % m;
      if (k <= i) A[(int64_t)i * n + k] -= A[(int64_t)i * n + j] * A[(int64_t)k * n + j];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) flag[0] = bad;
  if (bad)
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) A[t] = (t / n == t % n) ? 1.0 : 0.0;
}

// X = L^-1: warp c solves L x = e_c by forward substitution (x_k = 0 for
// k < c); each dot product is split over the lanes and reduced in lane order.
__global__ void k_trinv(const double* L, int n, const int* flag, double* X) {
  const int c = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (c >= n || flag[0]) return;
  for (int i = 0; i < c; ++i)
    if (lane == 0) X[(int64_t)i * n + c] = 0.0;
  for (int i = c; i < n; ++i) {
    double s = 0.0;
    for (int k = c + lane; k < i; k += 32) s += L[(int64_t)i * n + k] * X[(int64_t)k * n + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) X[(int64_t)i * n + c] = ((i == c ? 1.0 : 0.0) - s) / L[(int64_t)i * n + i];
    __syncwarp();
  }
}

// A^-1[a][b] = sum_{i >= max(a, b)} X[i][a] X[i][b] (A keeps the identity
// written by k_chol on a failed factorisation).
__global__ void k_gram(const double* X, int n, const int* flag, double* A) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n || flag[0]) return;
  const int a = t / n, b = t % n;
  double s = 0.0;
  for (int i = a > b ? a : b; i < n; ++i) s += X[(int64_t)i * n + a] * X[(int64_t)i * n + b];
  A[t] = s;
}

// T1 = F K^-1 (nh x nb), F[h][a] = G[h][a] sqrt(c U_a).
__global__ void k_wb_t1(const double* G, const double* U, const double* cdev, const double* Kinv, int nh, int nb,
                        double* T1) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nh * nb) return;
  const int h = t / nb, b = t % nb;
  const double c = *cdev;
  double s = 0.0;
  for (int a = 0; a < nb; ++a) s += G[(int64_t)h * nb + a] * sqrt(c * fmax(U[a], 0.0)) * Kinv[(int64_t)a * nb + b];
  T1[t] = s;
}

// S^-1 = I - T1 F^T (nh x nh).
__global__ void k_wb_s(const double* G, const double* U, const double* cdev, const double* T1, int nh, int nb,
                       double* Sinv) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nh * nh) return;
  const int i = t / nh, j = t % nh;
  const double c = *cdev;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += T1[(int64_t)i * nb + b] * G[(int64_t)j * nb + b] * sqrt(c * fmax(U[b], 0.0));
  Sinv[t] = (i == j ? 1.0 : 0.0) - s;
}

// FP32 copies for the iteration kernels: G [nh][nb], G^T [nb][nh], S^-1.
__global__ void k_schur_f32(const double* G, const double* Sinv, int nh, int nb, float* Gf, float* Gtf, float* Sf) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nh * nb) {
    const int h = t / nb, b = t % nb;
    Gf[t] = float(G[t]);
    Gtf[(int64_t)b * nh + h] = float(G[t]);
  }
  if (t < nh * nh) Sf[t] = float(Sinv[t]);
}

template <typename T>
PCArgs<T> pc_args(nre_metric* m) {
  nre_cf_plan* p = m->cf;
  PCArgs<T> a{};
  a.N = p->N;
  a.cdev = m->pc_cdev.as<double>();
  a.xi_p = m->xi_p.as<T>();
  const bool model = binned_model(p);
  a.av = metric_view<T>(m);
  a.nb = model ? p->n_bins : 0;
  a.invD = m->pc_invD.as<T>();
  a.e = model ? m->pc_e.as<T>() : nullptr;
  a.bpix = model ? m->bpix.as<int16_t>() : nullptr;
  return a;
}


template <typename T>
int setup_t(nre_metric* m, cudaStream_t st) {
  nre_cf_plan* p = m->cf;
  const int64_t N = p->N;
  const bool model = binned_model(p);
  const int nb = model ? p->n_bins : 0, nh = model ? p->n_hyper : 0;
  DevBuf& dbuf = m->pc_tmp;  // metric-owned, so a re-setup allocates nothing
  // [0, 1 + nb): the sums; then one row of 1 + nb per block of k_pc_setup
  const int sblk = sm_count();
  NRE_TRY(ensure(dbuf, (size_t)(1 + sblk) * (1 + nb) * sizeof(double)));
  double* spart = dbuf.as<double>() + (1 + nb);
  NRE_TRY(ensure(m->pc_cdev, sizeof(double)));
  NRE_TRY(ensure(m->pc_invD, (size_t)N * sizeof(T)));
  if (model) NRE_TRY(ensure(m->pc_e, (size_t)N * sizeof(T)));
  PCArgs<T> a = pc_args<T>(m);
  // pass 1: c = sum(w) = N mean(w), kept on the device
  prof_begin("pc_setup", (double)N * sizeof(T), st);
  NRE_TRY(pc_smem(k_pc_setup<T>, (size_t)(PC_THREADS / 32) * (nb > 0 ? nb : 1) * sizeof(double)));
  k_pc_setup<T><<<sblk, PC_THREADS, (size_t)(PC_THREADS / 32) * (nb > 0 ? nb : 1) * sizeof(double), st>>>(
      m->w.as<T>(), N, a, spart, 0);
  k_pc_setup_sum<<<1, 256, 0, st>>>(spart, sblk, 1, m->pc_cdev.as<double>());
  prof_end(st);
  NRE_CHECK_LAUNCH();
  m->pc_nh = nh;
  // per-pixel coefficients 1 / D and A xi_p / D
  prof_begin("pc_setup", (double)N * 3 * sizeof(T), st);
  k_pc_pix<T><<<304, PC_THREADS, 0, st>>>(a, m->pc_invD.as<T>(), model ? m->pc_e.as<T>() : nullptr);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  if (!model) return NRE_OK;
  // pass 2: U_b with the final c (dbuf[1 .. nb])
  prof_begin("pc_setup", (double)N * 2 * sizeof(T), st);
  k_pc_setup<T><<<sblk, PC_THREADS, (size_t)(PC_THREADS / 32) * nb * sizeof(double), st>>>(m->w.as<T>(), N, a,
                                                                                          spart, 1);
  k_pc_setup_sum<<<1, 256, 0, st>>>(spart, sblk, 1 + nb, dbuf.as<double>());
  prof_end(st);
  NRE_CHECK_LAUNCH();
  // amplitude Jacobian G[h][b] = dA_b / dh: JVPs along the unit vectors
  DevBuf& deye = m->pc_eye;
  DevBuf& dG = m->pc_dG;
  NRE_TRY(ensure(deye, (size_t)nh * nh * sizeof(T)));
  NRE_TRY(ensure(dG, (size_t)nh * nb * sizeof(double)));
  k_schur_eye<T><<<(nh * nh + 255) / 256, 256, 0, st>>>(deye.as<T>(), nh);
  NRE_CHECK_LAUNCH();
  NRE_TRY(amp_jvp<T>(amp_prior_of(p), m->state.as<double>(), 0, deye.as<T>(), nh, dG.as<double>(), nh, st));
  // S^-1 of S = I + c G diag(U) G^T on the device, in FP64: directly when
  // nh <= nb, else by the Woodbury identity through the nb x nb matrix
  // K = I + F^T F, F = G diag(sqrt(c U)):  S^-1 = I - F K^-1 F^T
  const bool wb = nh > nb;
  const int n = wb ? nb : nh;
  NRE_TRY(ensure(m->pc_A, (size_t)n * n * sizeof(double)));
  NRE_TRY(ensure(m->pc_W, (size_t)n * n * sizeof(double) + 16));  // X = L^-1 and a flag
  NRE_TRY(ensure(m->pc_Sd, (size_t)nh * nh * sizeof(double)));
  if (wb) NRE_TRY(ensure(m->pc_T1, (size_t)nh * nb * sizeof(double)));
  const double* c = m->pc_cdev.as<double>();
  const double* U = dbuf.as<double>() + 1;
  const double* G = dG.as<double>();
  double* A = m->pc_A.as<double>();
  prof_begin("pc_schur", (double)(nh * nb + 2 * n * n) * sizeof(double), st);
  k_schur_assemble<<<(n * n + 255) / 256, 256, 0, st>>>(G, U, c, nh, nb, wb ? 1 : 0, A);
  int* flag = reinterpret_cast<int*>(m->pc_W.as<double>() + (size_t)n * n);
  k_chol<<<1, 1024, 0, st>>>(A, n, flag);
  k_trinv<<<(n + 7) / 8, 256, 0, st>>>(A, n, flag, m->pc_W.as<double>());
  k_gram<<<(n * n + 255) / 256, 256, 0, st>>>(m->pc_W.as<double>(), n, flag, A);
  if (wb) {
    k_wb_t1<<<(nh * nb + 255) / 256, 256, 0, st>>>(G, U, c, A, nh, nb, m->pc_T1.as<double>());
    k_wb_s<<<(nh * nh + 255) / 256, 256, 0, st>>>(G, U, c, m->pc_T1.as<double>(), nh, nb, m->pc_Sd.as<double>());
  }
  NRE_TRY(ensure(m->pc_G, (size_t)nh * nb * sizeof(float)));
  NRE_TRY(ensure(m->pc_Gt, (size_t)nb * nh * sizeof(float)));
  NRE_TRY(ensure(m->pc_Sinv, (size_t)nh * nh * sizeof(float)));
  k_schur_f32<<<(nh * (nh > nb ? nh : nb) + 255) / 256, 256, 0, st>>>(G, wb ? m->pc_Sd.as<double>() : A, nh, nb,
                                                                      m->pc_G.as<float>(), m->pc_Gt.as<float>(),
                                                                      m->pc_Sinv.as<float>());
  prof_end(st);
  NRE_CHECK_LAUNCH();
  return NRE_OK;
}

// Workspace pointers and launch shapes of a preconditioned solve of B systems.
template <typename T>
struct PCGWork {
  T *r, *p, *q, *z;
  double *sc, *part_pq, *part_rr, *part_rz;
  PCArgs<T> pc;
  int nb, nh, nblk;
  size_t hsm, hyp_sm;
};

template <typename T>
PCGWork<T> pcg_work(nre_metric* m, int B) {
  PCGWork<T> w;
  nre_cf_plan* p = m->cf;
  w.nb = m->pc_nh > 0 ? p->n_bins : 0;
  w.nh = m->pc_nh;
  w.nblk = pc_blocks(m->latent, B);
  w.r = m->cg_r.as<T>();
  w.p = m->cg_p.as<T>();
  w.q = m->cg_q.as<T>();
  w.z = m->cg_z.as<T>();
  w.sc = m->cg_sc.as<double>();
  w.part_pq = m->cg_part.as<double>();
  w.part_rr = w.part_pq + (size_t)B * w.nblk;
  w.part_rz = w.part_rr + (size_t)B * w.nblk;
  w.pc = pc_args<T>(m);
  w.pc.nb = w.nb;
  w.pc.bin_part = w.nb > 0 ? m->pc_part.as<double>() : nullptr;
  w.pc.gz = w.nb > 0 ? m->pc_gz.as<double>() : nullptr;
  w.hsm = (size_t)(PC_THREADS / 32) * (w.nb > 0 ? w.nb : 1) * sizeof(double);  // warp-private histograms
  w.hyp_sm = (size_t)(w.nb + 2 * w.nh) * sizeof(float);
  return w;
}

// z = P r (and p = z on the first call).
template <typename T>
int pcg_precondition(nre_metric* m, const PCGWork<T>& w, int B, int init, cudaStream_t st) {
  const int64_t n = m->latent, S = m->stride, N = m->cf->N;
  const double vb = (double)B * n * sizeof(T);
  if (w.nb > 0) {
    prof_begin("pcg_hyper", (double)B * w.nh * sizeof(T) * 2, st);
    k_pcg_hyper<T><<<B, 512, w.hyp_sm, st>>>(w.r, w.z, S, N, w.nh, w.nb, m->pc_cdev.as<double>(), m->pc_G.as<float>(),
                                              m->pc_Gt.as<float>(), m->pc_Sinv.as<float>(), w.pc.bin_part,
                                              w.nblk, m->pc_gz.as<double>());
    prof_end(st);
  }
  prof_begin("pcg_z", (init ? 3.0 : 2.0) * vb + (double)N * sizeof(T), st);
  k_pcg_z<T><<<dim3(w.nblk, B), PC_THREADS, 0, st>>>(w.r, w.z, w.p, n, S, w.part_rz, w.pc, init);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  return NRE_OK;
}

template <typename T>
int pcg_begin_t(nre_metric* m, const T* b, T* x, int B, double rtol, cudaStream_t st) {
  const int64_t n = m->latent, S = m->stride;
  nre_cf_plan* p = m->cf;
  const int nb = m->pc_nh > 0 ? p->n_bins : 0;
  NRE_TRY(ensure(m->cg_r, (size_t)B * S * sizeof(T)));
  NRE_TRY(ensure(m->cg_p, (size_t)B * S * sizeof(T)));
  NRE_TRY(ensure(m->cg_q, (size_t)B * S * sizeof(T)));
  NRE_TRY(ensure(m->cg_z, (size_t)B * S * sizeof(T)));
  NRE_TRY(ensure(m->cg_sc, (size_t)B * SC_N * sizeof(double)));
  const int nblk = pc_blocks(n, B);
  NRE_TRY(ensure(m->cg_part, (size_t)3 * B * nblk * sizeof(double)));
  NRE_TRY(ensure(m->cg_dot, (size_t)B * kDotStride * sizeof(double)));
  if (nb > 0) {
    NRE_TRY(ensure(m->pc_part, (size_t)B * nblk * nb * sizeof(double)));
    NRE_TRY(ensure(m->pc_gz, (size_t)B * nb * sizeof(double)));
  }
  const PCGWork<T> w = pcg_work<T>(m, B);
  const double vb = (double)B * n * sizeof(T);
  prof_begin("pcg_init", 3.0 * vb, st);
  NRE_TRY(pc_smem(k_pcg_init<T>, w.hsm));
  k_pcg_init<T><<<dim3(nblk, B), PC_THREADS, w.hsm, st>>>(b, x, w.r, n, S, w.part_rr, w.pc);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  NRE_TRY(pcg_precondition<T>(m, w, B, 1, st));
  prof_begin("cg_scalars", 0.0, st);
  k_pcg_start<<<B, 32, 0, st>>>(w.sc, w.part_rr, w.part_rz, nblk, rtol);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  return NRE_OK;
}

template <typename T>
int pcg_iter_t(nre_metric* m, T* x, int B, int iters, double rtol, cudaStream_t st) {
  const int64_t n = m->latent, S = m->stride;
  const PCGWork<T> w = pcg_work<T>(m, B);
  const dim3 grid(w.nblk, B);
  const double vb = (double)B * n * sizeof(T);
  for (int it = 0; it < iters; ++it) {
    // p.q comes fused with the metric product (kDotStride partials per system)
    NRE_TRY(metric_apply_impl(m, w.p, w.q, B, st, m->cg_dot.as<double>()));
    prof_begin("pcg_update", 3 * vb, st);
    NRE_TRY(pc_smem(k_pcg_update<T>, w.hsm));
    k_pcg_update<T><<<grid, PC_THREADS, w.hsm, st>>>(w.r, w.q, n, S, w.sc, m->cg_dot.as<double>(), kDotStride,
                                                      w.part_rr, w.pc);
    prof_end(st);
    NRE_CHECK_LAUNCH();
    NRE_TRY(pcg_precondition<T>(m, w, B, 0, st));
    prof_begin("cg_pupdate", 5 * vb, st);
    k_pcg_pupdate<T><<<grid, PC_THREADS, 0, st>>>(x, w.p, w.z, n, S, w.sc, w.part_rz, w.nblk);
    prof_end(st);
    prof_begin("cg_scalars", 0.0, st);
    k_pcg_finish<<<B, 32, 0, st>>>(w.sc, w.part_rr, w.part_rz, w.nblk, rtol);
    prof_end(st);
    NRE_CHECK_LAUNCH();
  }
  return NRE_OK;
}

template <typename T>
int pcg_t(nre_metric* m, const T* b, T* x, int B, double rtol, int maxiter, int* iters_out,
          double* relres_out, cudaStream_t st) {
  NRE_TRY(pcg_begin_t<T>(m, b, x, B, rtol, st));
  const int check_every = 8;
  for (int it = 0; it < maxiter; it += check_every) {
    const int k = maxiter - it < check_every ? maxiter - it : check_every;
    NRE_TRY(pcg_iter_t<T>(m, x, B, k, rtol, st));
    if (rtol > 0.0 && it + k < maxiter) {
      NRE_TRY(cg_read_scalars(m, B, st));
      if (!cg_any_active(m, B)) break;
    }
  }
  NRE_TRY(cg_read_scalars(m, B, st));
  return cg_report(m, B, rtol, maxiter, iters_out, relres_out, "PCG");
}

}  // namespace

namespace nre {
int pcg_begin(nre_metric* m, const void* b, void* x, int B, double rtol, cudaStream_t st) {
  if (m->dtype == NRE_F64) return pcg_begin_t<double>(m, (const double*)b, (double*)x, B, rtol, st);
  return pcg_begin_t<float>(m, (const float*)b, (float*)x, B, rtol, st);
}

int pcg_iterate(nre_metric* m, void* x, int B, int iters, double rtol, cudaStream_t st) {
  if (m->dtype == NRE_F64) return pcg_iter_t<double>(m, (double*)x, B, iters, rtol, st);
  return pcg_iter_t<float>(m, (float*)x, B, iters, rtol, st);
}

int pcg_solve_impl(nre_metric* m, const void* b, void* x, int batch, double rtol, int maxiter,
                   int* iters_out, double* relres_out, cudaStream_t st) {
  if (m->dtype == NRE_F64)
    return pcg_t<double>(m, (const double*)b, (double*)x, batch, rtol, maxiter, iters_out, relres_out, st);
  return pcg_t<float>(m, (const float*)b, (float*)x, batch, rtol, maxiter, iters_out, relres_out, st);
}
}  // namespace nre

extern "C" int metric_set_precond(nre_metric* m, int kind, nre_stream_t stream) {
  clear_error();
  if (!m) return set_error(NRE_EINVAL, "metric must not be NULL");
  if (kind == NRE_PRECOND_NONE) {
    m->precond = kind;
    return NRE_OK;
  }
  if (kind != NRE_PRECOND_HARMONIC) return set_error(NRE_EINVAL, "unknown preconditioner %d", kind);
  if (m->model_kind != NRE_MODEL_CF)
    return set_error(NRE_EINVAL, "the harmonic preconditioner needs a correlated-field metric");
  cudaStream_t st = (cudaStream_t)stream;
  const int s = m->dtype == NRE_F64 ? setup_t<double>(m, st) : setup_t<float>(m, st);
  if (s != NRE_OK) return s;
  m->precond = kind;
  return NRE_OK;
}
