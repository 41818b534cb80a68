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

using namespace nre;

namespace {

constexpr int PC_THREADS = 256;
enum { SC_RR = 0, SC_BB = 1, SC_RZ = 2, SC_BETA = 3, SC_ACTIVE = 4, SC_ITERS = 5, SC_N = 8 };

int pc_blocks(int64_t n) {
  int64_t nb = (n + PC_THREADS * 8 - 1) / (PC_THREADS * 8);
  if (nb > 64) nb = 64;
  if (nb < 1) nb = 1;
  return (int)nb;
}

template <typename T>
struct PCArgs {
  int64_t N;          // field entries (the rest of the latent vector is hyper)
  double c;           // N * mean(w)
  AmpView<T> av;      // amplitude at the expansion point
  const T* xi_p;      // expansion point (field)
  int nb;             // bins (0: fixed amplitude, no hyper block)
  double* bin_part;   // [B][gridDim.x][nb] partial sums t_b
  const double* gz;   // [B][nb]
};

__device__ void partial_out(double acc, double* part) {
  __shared__ double red[PC_THREADS / 32];
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// Bins t_b += A_k xi_p[k] r_k / D_k of the field entries of r (per-CTA
// histogram in shared memory, one partial per CTA).
template <typename T>
__device__ void bins_of(const PCArgs<T>& pc, int b, const T* r, int64_t S, double* hist) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < pc.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int bn = pc.av.bin(i);
    if (bn < 0) continue;
    const T A = pc.av.amp(0, i, bn);
    const T D = T(1) + T(pc.c) * A * A;
    atomicAdd(&hist[bn], double(A * pc.xi_p[i] * r[b * S + i] / D));
  }
}

template <typename T>
__global__ void __launch_bounds__(PC_THREADS) k_pcg_init(const T* bsrc, T* x, T* r, int64_t n, int64_t S,
                                                        double* rr_part, PCArgs<T> pc) {
  extern __shared__ double hist[];
  const int b = blockIdx.y;
  for (int i = threadIdx.x; i < pc.nb; i += blockDim.x) hist[i] = 0.0;
  __syncthreads();
  const int64_t off = (int64_t)b * S;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T v = bsrc[off + i];
    x[off + i] = T(0);
    r[off + i] = v;
    acc += double(v * v);
  }
  if (pc.nb > 0) bins_of(pc, b, bsrc, S, hist);
  partial_out(acc, rr_part);
  __syncthreads();
  if (pc.nb > 0) {
    double* dst = pc.bin_part + ((int64_t)b * gridDim.x + blockIdx.x) * pc.nb;
    for (int i = threadIdx.x; i < pc.nb; i += blockDim.x) dst[i] = hist[i];
  }
}

// alpha = r.z / p.q; x += alpha p; r -= alpha q; partials of r.r and of the bins.
template <typename T>
__global__ void __launch_bounds__(PC_THREADS) k_pcg_update(T* x, T* r, const T* p, const T* q, int64_t n,
                                                          int64_t S, const double* sc, const double* pq_part,
                                                          double* rr_part, PCArgs<T> pc) {
  extern __shared__ double hist[];
  const int b = blockIdx.y, nblk = gridDim.x;
  for (int i = threadIdx.x; i < pc.nb; i += blockDim.x) hist[i] = 0.0;
  __syncthreads();
  const double* c = sc + b * SC_N;
  const bool active = c[SC_ACTIVE] != 0.0;
  double pq = 0.0;
  for (int i = 0; i < nblk; ++i) pq += pq_part[b * nblk + i];
  const T alpha = T(active && pq != 0.0 ? c[SC_RZ] / pq : 0.0);
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
  __syncthreads();
  if (pc.nb > 0) bins_of(pc, b, r, S, hist);
  partial_out(acc, rr_part);
  __syncthreads();
  if (pc.nb > 0) {
    double* dst = pc.bin_part + ((int64_t)b * gridDim.x + blockIdx.x) * pc.nb;
    for (int i = threadIdx.x; i < pc.nb; i += blockDim.x) dst[i] = hist[i];
  }
}

// Hyper block of the preconditioner, one CTA per system:
// z_h = S^-1 (r_h - c G^T t), g = G z_h.
template <typename T>
__global__ void k_pcg_hyper(const T* r, T* z, int64_t S, int64_t N, int nh, int nb, double c,
                            const float* G, const float* Sinv, const double* bin_part, int nparts,
                            double* gz) {
  extern __shared__ float sh[];
  float* t = sh;        // [nb]
  float* u = t + nb;    // [nh]
  float* zh = u + nh;   // [nh]
  const int b = blockIdx.x;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    double s = 0.0;
    const double* pp = bin_part + (int64_t)b * nparts * nb + i;
    for (int k = 0; k < nparts; ++k) s += pp[(int64_t)k * nb];
    t[i] = float(s);
  }
  __syncthreads();
  const T* rh = r + (int64_t)b * S + N;
  for (int h = threadIdx.x; h < nh; h += blockDim.x) {
    float s = 0.f;
    const float* g = G + (int64_t)h * nb;
    for (int i = 0; i < nb; ++i) s += g[i] * t[i];
    u[h] = float(rh[h]) - float(c) * s;
  }
  __syncthreads();
  T* zo = z + (int64_t)b * S + N;
  for (int h = threadIdx.x; h < nh; h += blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < nh; ++k) s += Sinv[(int64_t)k * nh + h] * u[k];  // S^-1 symmetric
    zh[h] = s;
    zo[h] = T(s);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    float s = 0.f;
    for (int h = 0; h < nh; ++h) s += G[(int64_t)h * nb + i] * zh[h];
    gz[(int64_t)b * nb + i] = s;
  }
}

// Field block z_f = (r_f - c A xi_p g_bin) / D; partials of r.z over the whole
// latent vector (the hyper part of z was written by k_pcg_hyper).  With
// `init`, also p = z.
template <typename T>
__global__ void __launch_bounds__(PC_THREADS) k_pcg_z(const T* r, T* z, T* p, int64_t n, int64_t S,
                                                     double* rz_part, PCArgs<T> pc, int init) {
  const int b = blockIdx.y;
  const int64_t off = (int64_t)b * S;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T ri = r[off + i];
    T zi;
    if (i < pc.N) {
      const int bn = pc.av.binned() ? pc.av.bin(i) : -1;
      const T A = pc.av.amp(0, i, bn);
      const T D = T(1) + T(pc.c) * A * A;
      T num = ri;
      if (bn >= 0 && pc.nb > 0) num -= T(pc.c) * A * pc.xi_p[i] * T(pc.gz[(int64_t)b * pc.nb + bn]);
      zi = num / D;
      z[off + i] = zi;
    } else {
      zi = z[off + i];
    }
    if (init) p[off + i] = zi;
    acc += double(ri * zi);
  }
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
  c[SC_ITERS] = 0.0;
  c[SC_ACTIVE] = (rr > 0.0 && rtol < 1.0) ? 1.0 : 0.0;
}

// beta = r'.z' / r.z and p = z + beta p (every block reads the old r.z; the
// scalars are updated by k_pcg_finish afterwards).
template <typename T>
__global__ void __launch_bounds__(PC_THREADS) k_pcg_pupdate(T* p, const T* z, int64_t n, int64_t S,
                                                           const double* sc, const double* rz_part, int nblk) {
  const int b = blockIdx.y;
  const double* c = sc + b * SC_N;
  if (c[SC_ACTIVE] == 0.0) return;
  double rz = 0.0;
  for (int i = 0; i < nblk; ++i) rz += rz_part[b * nblk + i];
  const T beta = T(rz / c[SC_RZ]);
  const int64_t off = (int64_t)b * S;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[off + i] = z[off + i] + beta * p[off + i];
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
  c[SC_BETA] = rz / c[SC_RZ];
  c[SC_RR] = rr;
  c[SC_RZ] = rz;
  c[SC_ITERS] += 1.0;
  if (rtol > 0.0 && sqrt(rr) <= rtol * sqrt(c[SC_BB])) c[SC_ACTIVE] = 0.0;
}

template <typename T>
__global__ void k_dot_p(const T* a, const T* q, int64_t n, int64_t S, double* part) {
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
  partial_out(acc, part);
}

// U_b = sum_{k in b} xi_p[k]^2 / D_k (bins of the expansion point), and
// sum w for c = N mean(w).
template <typename T>
__global__ void k_pc_setup(const T* w, int64_t N, PCArgs<T> pc, double* U, double* wsum) {
  extern __shared__ double hist[];
  for (int i = threadIdx.x; i < pc.nb; i += blockDim.x) hist[i] = 0.0;
  __syncthreads();
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    acc += double(w[i]);
    if (pc.nb > 0 && pc.c > 0.0) {
      const int bn = pc.av.bin(i);
      if (bn >= 0) {
        const double A = double(pc.av.amp(0, i, bn));
        const double xp = double(pc.xi_p[i]);
        atomicAdd(&hist[bn], xp * xp / (1.0 + pc.c * A * A));
      }
    }
  }
  __shared__ double red[PC_THREADS / 32];
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) atomicAdd(wsum, t);
  __syncthreads();
  if (pc.nb > 0 && pc.c > 0.0)
    for (int i = threadIdx.x; i < pc.nb; i += blockDim.x) atomicAdd(&U[i], hist[i]);
}

template <typename T>
PCArgs<T> pc_args(nre_metric* m) {
  nre_cf_plan* p = m->cf;
  PCArgs<T> a{};
  a.N = p->N;
  a.c = m->pc_c;
  a.xi_p = m->xi_p.as<T>();
  const bool model = p->amp_kind == NRE_AMP_POWER_MODEL;
  a.av = metric_view<T>(m);
  a.nb = model ? p->n_bins : 0;
  return a;
}

// In-place Cholesky and inverse of an SPD n x n matrix (host, FP64).
bool spd_inverse(std::vector<double>& A, int n, std::vector<double>& inv) {
  std::vector<double> L = A;
  for (int j = 0; j < n; ++j) {
    double s = L[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(s > 0.0)) return false;
    const double d = std::sqrt(s);
    L[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = L[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = t / d;
    }
  }
  inv.assign((size_t)n * n, 0.0);
  std::vector<double> col(n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * col[k];
      col[i] = s / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = col[i];
      for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * col[k];
      col[i] = s / L[(size_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + c] = col[i];
  }
  return true;
}

template <typename T>
int setup_t(nre_metric* m, cudaStream_t st) {
  nre_cf_plan* p = m->cf;
  const int64_t N = p->N;
  const bool model = p->amp_kind == NRE_AMP_POWER_MODEL;
  const int nb = model ? p->n_bins : 0, nh = model ? p->n_hyper : 0;
  DevBuf dbuf;
  NRE_TRY(dbuf.alloc((size_t)(1 + nb) * sizeof(double)));
  NRE_TRY_CUDA(cudaMemsetAsync(dbuf.p, 0, (size_t)(1 + nb) * sizeof(double), st));
  // pass 1: mean weight
  PCArgs<T> a = pc_args<T>(m);
  a.c = 0.0;
  prof_begin("pc_setup", (double)N * sizeof(T), st);
  k_pc_setup<T><<<152, PC_THREADS, (size_t)(nb > 0 ? nb : 1) * sizeof(double), st>>>(
      m->w.as<T>(), N, a, dbuf.as<double>() + 1, dbuf.as<double>());
  prof_end(st);
  NRE_CHECK_LAUNCH();
  double wsum = 0.0;
  NRE_TRY_CUDA(cudaMemcpyAsync(&wsum, dbuf.p, sizeof(double), cudaMemcpyDeviceToHost, st));
  NRE_TRY_CUDA(cudaStreamSynchronize(st));
  m->pc_c = wsum;  // N * mean(w) = sum(w)
  m->pc_nh = nh;
  if (!model) return NRE_OK;
  // pass 2: U_b with the final c
  NRE_TRY_CUDA(cudaMemsetAsync(dbuf.p, 0, (size_t)(1 + nb) * sizeof(double), st));
  a.c = m->pc_c;
  prof_begin("pc_setup", (double)N * 2 * sizeof(T), st);
  k_pc_setup<T><<<152, PC_THREADS, (size_t)nb * sizeof(double), st>>>(m->w.as<T>(), N, a,
                                                                     dbuf.as<double>() + 1, dbuf.as<double>());
  prof_end(st);
  NRE_CHECK_LAUNCH();
  // amplitude Jacobian G[h][b] = dA_b / dh: JVPs along the unit vectors
  std::vector<T> eye((size_t)nh * nh, T(0));
  for (int h = 0; h < nh; ++h) eye[(size_t)h * nh + h] = T(1);
  DevBuf deye, dG;
  NRE_TRY(deye.upload(eye.data(), eye.size() * sizeof(T)));
  NRE_TRY(dG.alloc((size_t)nh * nb * sizeof(double)));
  NRE_TRY(amp_jvp<T>(amp_prior_of(p), m->state.as<double>(), 0, deye.as<T>(), nh, dG.as<double>(), nh, st));
  std::vector<double> G((size_t)nh * nb), U(nb);
  NRE_TRY_CUDA(cudaMemcpyAsync(G.data(), dG.p, G.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  NRE_TRY_CUDA(cudaMemcpyAsync(U.data(), dbuf.as<double>() + 1, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  NRE_TRY_CUDA(cudaStreamSynchronize(st));
  // S = I + c G diag(U) G^T (G stored [h][b])
  std::vector<double> S((size_t)nh * nh), Sinv;
  const double c = m->pc_c;
  for (int i = 0; i < nh; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = 0.0;
      for (int k = 0; k < nb; ++k) s += G[(size_t)i * nb + k] * U[k] * G[(size_t)j * nb + k];
      S[(size_t)i * nh + j] = S[(size_t)j * nh + i] = c * s + (i == j ? 1.0 : 0.0);
    }
  if (!spd_inverse(S, nh, Sinv)) return set_error(NRE_EINVAL, "preconditioner Schur block is not positive definite");
  std::vector<float> Gf(G.begin(), G.end()), Sf(Sinv.begin(), Sinv.end());
  NRE_TRY(m->pc_G.upload(Gf.data(), Gf.size() * sizeof(float)));
  NRE_TRY(m->pc_Sinv.upload(Sf.data(), Sf.size() * sizeof(float)));
  return NRE_OK;
}

template <typename T>
int pcg_t(nre_metric* m, const T* b, T* x, int B, double rtol, int maxiter, int* iters_out,
          double* relres_out, cudaStream_t st) {
  const int64_t n = m->latent, S = m->stride;
  nre_cf_plan* p = m->cf;
  const int nb = m->pc_nh > 0 ? p->n_bins : 0, nh = m->pc_nh;
  NRE_TRY(ensure(m->cg_r, (size_t)B * S * sizeof(T)));
  NRE_TRY(ensure(m->cg_p, (size_t)B * S * sizeof(T)));
  NRE_TRY(ensure(m->cg_q, (size_t)B * S * sizeof(T)));
  NRE_TRY(ensure(m->cg_z, (size_t)B * S * sizeof(T)));
  NRE_TRY(ensure(m->cg_sc, (size_t)B * SC_N * sizeof(double)));
  const int nblk = pc_blocks(n);
  NRE_TRY(ensure(m->cg_part, (size_t)3 * B * nblk * sizeof(double)));
  if (nb > 0) {
    NRE_TRY(ensure(m->pc_part, (size_t)B * nblk * nb * sizeof(double)));
    NRE_TRY(ensure(m->pc_gz, (size_t)B * nb * sizeof(double)));
  }
  T* r = m->cg_r.as<T>();
  T* pp = m->cg_p.as<T>();
  T* q = m->cg_q.as<T>();
  T* z = m->cg_z.as<T>();
  double* sc = m->cg_sc.as<double>();
  double* part_pq = m->cg_part.as<double>();
  double* part_rr = part_pq + (size_t)B * nblk;
  double* part_rz = part_rr + (size_t)B * nblk;
  PCArgs<T> pc = pc_args<T>(m);
  pc.nb = nb;
  pc.bin_part = nb > 0 ? m->pc_part.as<double>() : nullptr;
  pc.gz = nb > 0 ? m->pc_gz.as<double>() : nullptr;
  const dim3 grid(nblk, B);
  const size_t hsm = (size_t)(nb > 0 ? nb : 1) * sizeof(double);
  const size_t hyp_sm = (size_t)(nb + 2 * nh) * sizeof(float);
  const double vb = (double)B * n * sizeof(T);
  auto precondition = [&](int init) -> int {
    if (nb > 0) {
      prof_begin("pcg_hyper", (double)B * nh * sizeof(T) * 2, st);
      k_pcg_hyper<T><<<B, 256, hyp_sm, st>>>(r, z, S, p->N, nh, nb, m->pc_c, m->pc_G.as<float>(),
                                             m->pc_Sinv.as<float>(), pc.bin_part, nblk, m->pc_gz.as<double>());
      prof_end(st);
    }
    prof_begin("pcg_z", (init ? 3.0 : 2.0) * vb + (double)p->N * sizeof(T), st);
    k_pcg_z<T><<<grid, PC_THREADS, 0, st>>>(r, z, pp, n, S, part_rz, pc, init);
    prof_end(st);
    NRE_CHECK_LAUNCH();
    return NRE_OK;
  };
  prof_begin("pcg_init", 3.0 * vb, st);
  k_pcg_init<T><<<grid, PC_THREADS, hsm, st>>>(b, x, r, n, S, part_rr, pc);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  NRE_TRY(precondition(1));
  prof_begin("cg_scalars", 0.0, st);
  k_pcg_start<<<B, 32, 0, st>>>(sc, part_rr, part_rz, nblk, rtol);
  prof_end(st);
  m->cg_host.resize((size_t)B * SC_N);
  const int check_every = 8;
  for (int it = 0; it < maxiter; ++it) {
    NRE_TRY(metric_apply_impl(m, pp, q, B, st));
    prof_begin("cg_dot", 2 * vb, st);
    k_dot_p<T><<<grid, PC_THREADS, 0, st>>>(pp, q, n, S, part_pq);
    prof_end(st);
    prof_begin("pcg_update", 6 * vb, st);
    k_pcg_update<T><<<grid, PC_THREADS, hsm, st>>>(x, r, pp, q, n, S, sc, part_pq, part_rr, pc);
    prof_end(st);
    NRE_CHECK_LAUNCH();
    NRE_TRY(precondition(0));
    prof_begin("cg_pupdate", 3 * vb, st);
    k_pcg_pupdate<T><<<grid, PC_THREADS, 0, st>>>(pp, z, n, S, sc, part_rz, nblk);
    prof_end(st);
    prof_begin("cg_scalars", 0.0, st);
    k_pcg_finish<<<B, 32, 0, st>>>(sc, part_rr, part_rz, nblk, rtol);
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
  if (!conv) return set_error(NRE_ENOTCONV, "PCG: some system missed rtol=%g within maxiter=%d", rtol, maxiter);
  return NRE_OK;
}

}  // namespace

namespace nre {
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
