// Batched conjugate gradients on the metric (the linear MGVI sample draw).
//
// Sec. "Variational Inference": draw_linear_kwargs / cg_kwargs - samples are
// drawn by CG on M_p (maxiter = 100 in the example).  Textbook Hestenes-Stiefel
// per system b: x_0 = 0, r_0 = b, p_0 = r_0; alpha = r.r / p.Mp;
// x += alpha p; r -= alpha Mp; beta = r'.r' / r.r; p = r' + beta p.  A system
// stops (x frozen) once ||r|| <= rtol ||b|| on the recursive residual; rtol = 0
// runs exactly maxiter iterations.  Inner products and alpha / beta are FP64
// across threads and blocks; within a thread, FP32 products are summed in
// compensated FP32 (RunSum), FP64 products in FP64.
#include <cmath>

#include "metric_internal.cuh"

using namespace nre;

namespace {

constexpr int CG_THREADS = 256;
// SC_XALPHA: the step alpha of the last update kernel whose x += alpha p the
// next p-update kernel applies (0: none).
enum { SC_RR = CG_SC_RR, SC_BB = CG_SC_BB, SC_ALPHA = 2, SC_BETA = 3, SC_ACTIVE = CG_SC_ACTIVE,
       SC_ITERS = CG_SC_ITERS, SC_XALPHA = 6, SC_N = CG_SC_N };

// Blocks per system of the vector kernels: four per SM over the whole batch,
// one wave (each block forms alpha and its share of the hyper rows before and
// after its vector loop; 8, 12 and 16 per SM measured 36, 54 and 65 % slower
// update kernels at 512^2, batch 32, and 2 or 3 per SM 14 and 7 % slower), at
// least 4 vectors per thread and at most 64 blocks.
int cg_blocks(int64_t n, int B) {
  int64_t nb = (4 * (int64_t)sm_count() + B - 1) / B;
  const int64_t cap = (n + CG_THREADS * 16 - 1) / (CG_THREADS * 16);
  if (nb > cap) nb = cap;
  if (nb > 64) nb = 64;
  if (nb < 1) nb = 1;
  return (int)nb;
}

// Sum over the block, then one partial per (system, block).
template <typename T>
__device__ void write_partial(const RunSum<T>& acc, double* part) {
  const double t = acc.block_sum();
  if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// As write_partial; the last block of system blockIdx.y to finish then sums
// the partials in block order (deterministic) and calls fin(total) from
// thread 0.  counter[system] must be 0 on entry and is reset.
template <typename T, class F>
__device__ void finish_partial(const RunSum<T>& acc, double* part, unsigned* counter, F fin) {
  __shared__ bool last;
  const double t = acc.block_sum();
  const int b = blockIdx.y, nblk = gridDim.x;
  if (threadIdx.x == 0) {
    part[b * nblk + blockIdx.x] = t;
    __threadfence();
    last = atomicAdd(&counter[b], 1u) == (unsigned)(nblk - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double s = 0.0;
    const volatile double* vp = part + b * nblk;
    for (int i = 0; i < nblk; ++i) s += vp[i];
    fin(s);
    counter[b] = 0;
  }
}

// 16-byte vector of T (4 floats or 2 doubles).
template <typename T>
struct alignas(16) V16 {
  static constexpr int W = 16 / sizeof(T);
  T e[W];
};

// Grid-stride loop over the n entries of system blockIdx.y, 16-byte vectors
// first (the system offset is a multiple of 64 elements), then the scalar
// tail.  f(i, w) handles W consecutive entries starting at i (w = W) or one
// entry (w = 1).
template <typename T, class F>
__device__ __forceinline__ void for_vec(int64_t n, F f) {
  constexpr int W = V16<T>::W;
  const int64_t nv = n / W;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += stride) f(v * W, W);
  for (int64_t i = nv * W + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) f(i, 1);
}

// As for_vec, U vectors per thread and step: fv(idx, ok) gets the element
// indices of U vectors (ok: in range) so that it can issue all their loads
// before using any; fs(i) handles one tail entry.  The vectors a thread visits
// come in the same order as in for_vec.
// The loop runs over the CTAs cta = 0 .. ncta-1 of the system.
template <typename T, int U, class FV, class FS>
__device__ __forceinline__ void for_vec_u(int64_t n, int cta, int ncta, FV fv, FS fs) {
  constexpr int W = V16<T>::W;
  const int64_t nv = n / W;
  const int64_t stride = (int64_t)ncta * blockDim.x;
  for (int64_t v = cta * (int64_t)blockDim.x + threadIdx.x; v < nv; v += U * stride) {
    int64_t idx[U];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      idx[u] = (v + u * stride) * W;
      ok[u] = v + u * stride < nv;
    }
    fv(idx, ok);
  }
  for (int64_t i = nv * W + cta * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) fs(i);
}

// The FP32 power-spectrum model's hyper-parameter block, handled inside the
// CG vector kernels (G == nullptr: not fused; the metric product then forms
// dA and the hyper part of q itself).  Latent layout: field entries [0, N),
// hyper-parameters [N, N + nh).  With the Jacobian G of the amplitude model
// at the expansion point (G [nb][nhp], Gt [nh][nbp], rows zero-padded to
// multiples of 4 floats), the metric product's hyper part is
// q_h = p_h + G^T g with g = gsum, the log-|k| bin sums of its last sweep,
// and the product's tangent amplitude is dA = G p_h; so
// p_h . q_h = p_h . p_h + dA . g needs no G^T product.  The update kernel
// forms q_h row by row (each block a share of the rows), the p-update kernel's
// last block forms the next p_h, its dA and zeroes gsum for the next product.
struct CGHyper {
  const float* G;
  const float* Gt;
  double* dA;    // [B][nb]: G p_h of the current p
  double* gsum;  // [B][nb]
  int nb, nh;
  int64_t N;
};

template <typename T>
__device__ __forceinline__ V16<T> ldv(const T* p) { return *reinterpret_cast<const V16<T>*>(p); }
template <typename T>
__device__ __forceinline__ void stv(T* p, const V16<T>& v) { *reinterpret_cast<V16<T>*>(p) = v; }

template <typename T>
__global__ void __launch_bounds__(CG_THREADS) k_cg_init(const T* b, T* x, T* r, T* p, int64_t n,
                                                       int64_t S, double* part) {
  const int64_t off = (int64_t)blockIdx.y * S;
  RunSum<T> acc;
  for_vec<T>(n, [&](int64_t i, int w) {
    if (w > 1) {
      const V16<T> v = ldv(b + off + i);
      V16<T> z;
      T run = T(0);  // one vector
#pragma unroll
      for (int k = 0; k < V16<T>::W; ++k) {
        z.e[k] = T(0);
        run += v.e[k] * v.e[k];
      }
      stv(x + off + i, z);
      stv(r + off + i, v);
      stv(p + off + i, v);
      acc.add(run);
    } else {
      const T v = b[off + i];
      x[off + i] = T(0);
      r[off + i] = v;
      p[off + i] = v;
      acc.add(v * v);
    }
  });
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
  c[SC_XALPHA] = 0.0;
  c[SC_ITERS] = 0.0;
  c[SC_ACTIVE] = (s > 0.0 && rtol < 1.0) ? 1.0 : 0.0;
}

// p.q, then alpha = r.r / p.q for the system (last block).
template <typename T>
__global__ void __launch_bounds__(CG_THREADS) k_cg_dot(const T* a, const T* q, int64_t n, int64_t S,
                                                      double* part, unsigned* counter, double* sc) {
  const int64_t off = (int64_t)blockIdx.y * S;
  RunSum<T> acc;
  for_vec<T>(n, [&](int64_t i, int w) {
    T run = T(0);  // one vector's products in T, folded into FP64
    if (w > 1) {
      const V16<T> u = ldv(a + off + i), v = ldv(q + off + i);
#pragma unroll
      for (int k = 0; k < V16<T>::W; ++k) run += u.e[k] * v.e[k];
    } else {
      run = a[off + i] * q[off + i];
    }
    acc.add(run);
  });
  double* c = sc + blockIdx.y * SC_N;
  finish_partial(acc, part, counter, [&](double pq) {
    c[SC_ALPHA] = (c[SC_ACTIVE] != 0.0 && pq != 0.0) ? c[SC_RR] / pq : 0.0;
  });
}

// r -= alpha q; then (last block) beta = r'.r' / r.r, the iteration count and
// the convergence test.  A system that has converged keeps beta = 0 and its
// x, r frozen.  The step x += alpha p is left to the p-update kernel, which
// reads p anyway (alpha in SC_XALPHA): one vector read less per iteration,
// and x is complete after every p-update, the same values in the same
// arithmetic as when the update kernel applied it.
// With pq (the fused p.q partials of the metric product, kDotStride per
// system) every block forms alpha = r.r / p.q itself; the last block of the
// system, which alone rewrites r.r, starts only after every block has read it.
// With hy.G (CGHyper): the vector loop covers the field entries; p.q gains the
// hyper part p_h . p_h + dA . g (one warp per block, read from pn = the
// current p_h), and each block takes a share of the hyper rows: q_h = p_h +
// Gt[h] . g, r_h -= alpha q_h, p_h copied from pn into p.
template <typename T>
__global__ void __launch_bounds__(CG_THREADS, 4) k_cg_update(T* r, T* p, const T* q, int64_t n,
                                                         int64_t S, double* sc, double* rr_part,
                                                         unsigned* counter, double rtol, const double* pq,
                                                         CGHyper hy, const T* pn) {
  const int b = blockIdx.y;
  double* c = sc + b * SC_N;
  const bool active = c[SC_ACTIVE] != 0.0;
  const bool fused = hy.G != nullptr;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t off = (int64_t)b * S;
  T alpha;
  if (pq != nullptr) {
    // one FP64 division per block, not per thread
    __shared__ T s_alpha;
    __shared__ double s_hd;
    if (fused && wid == 1) {
      float pp = 0.f;
      for (int h = lane; h < hy.nh; h += 32) {
        const float v = float(pn[(int64_t)b * hy.nh + h]);
        pp += v * v;
      }
      double dg = 0.0;
      for (int i = lane; i < hy.nb; i += 32) dg += hy.dA[(int64_t)b * hy.nb + i] * hy.gsum[(int64_t)b * hy.nb + i];
      pp = warp_sum_f(pp);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dg += __shfl_xor_sync(0xffffffffu, dg, o);
      if (lane == 0) s_hd = dg + double(pp);
    }
    const double s0 = block_sum_array(pq + (int64_t)b * kDotStride, kDotStride);
    if (threadIdx.x == 0) {
      const double s = s0 + (fused ? s_hd : 0.0);
      s_alpha = T(active && s != 0.0 ? c[SC_RR] / s : 0.0);
    }
    __syncthreads();
    alpha = s_alpha;
  } else {
    alpha = T(c[SC_ALPHA]);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) c[SC_XALPHA] = active ? double(alpha) : 0.0;
  RunSum<T> acc;
  constexpr int U = 4;
  for_vec_u<T, U>(
      fused ? hy.N : n, blockIdx.x, gridDim.x,
      [&](const int64_t (&idx)[U], const bool (&ok)[U]) {
        V16<T> ri[U], qi[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (ok[u]) {
            ri[u] = ldv(r + off + idx[u]);
            if (active) qi[u] = ldv(q + off + idx[u]);
          }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (ok[u]) {
            if (active) {
#pragma unroll
              for (int k = 0; k < V16<T>::W; ++k) ri[u].e[k] -= alpha * qi[u].e[k];
              stv(r + off + idx[u], ri[u]);
            }
            T run = T(0);  // one vector
#pragma unroll
            for (int k = 0; k < V16<T>::W; ++k) run += ri[u].e[k] * ri[u].e[k];
            acc.add(run);
          }
      },
      [&](int64_t i) {
        T ri = r[off + i];
        if (active) {
          ri -= alpha * q[off + i];
          r[off + i] = ri;
        }
        acc.add(ri * ri);
      });
  if (fused) {
    // g = gsum[b] in FP32 (zero-padded), then four rows of Gt per warp and
    // round, all their 16-byte loads in flight
    __shared__ float4 sg4[256];
    float* sg = reinterpret_cast<float*>(sg4);
    const int nb4 = (hy.nb + 3) >> 2;
    for (int i = threadIdx.x; i < 4 * nb4; i += blockDim.x)
      sg[i] = i < hy.nb ? float(hy.gsum[(int64_t)b * hy.nb + i]) : 0.f;
    __syncthreads();
    const int rows = (hy.nh + gridDim.x - 1) / gridDim.x;
    const int h0 = blockIdx.x * rows, h1 = min(hy.nh, h0 + rows);
    const float4* G4 = reinterpret_cast<const float4*>(hy.Gt);
    for (int hb = h0 + 4 * wid; hb < h1; hb += 32) {
      float t[4] = {0.f, 0.f, 0.f, 0.f};
      for (int j0 = 0; j0 < nb4; j0 += 64) {
        float4 gv[4][2];
#pragma unroll
        for (int qr = 0; qr < 4; ++qr)
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const int j = j0 + lane + 32 * k;
            gv[qr][k] = (hb + qr < h1 && j < nb4) ? __ldg(G4 + (int64_t)(hb + qr) * nb4 + j)
                                                   : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int j = j0 + lane + 32 * k;
          if (j < nb4) {
            const float4 a4 = sg4[j];
#pragma unroll
            for (int qr = 0; qr < 4; ++qr) t[qr] += dot4(gv[qr][k], a4);
          }
        }
      }
#pragma unroll
      for (int qr = 0; qr < 4; ++qr) t[qr] = warp_sum_f(t[qr]);
      const int ql = lane & 3, h = hb + ql;
      if (lane < 4 && h < h1) {
        const int64_t e = off + hy.N + h;
        const T ph = pn[(int64_t)b * hy.nh + h];
        const T tq = T(ql == 0 ? t[0] : ql == 1 ? t[1] : ql == 2 ? t[2] : t[3]);
        T rh = r[e];
        p[e] = ph;
        if (active) {
          rh -= alpha * (ph + tq);
          r[e] = rh;
        }
        acc.add(rh * rh);
      }
    }
  }
  finish_partial(acc, rr_part, counter, [&](double rr_new) {
    if (c[SC_ACTIVE] == 0.0) {
      c[SC_BETA] = 0.0;
      return;
    }
    c[SC_BETA] = c[SC_RR] != 0.0 ? rr_new / c[SC_RR] : 0.0;
    c[SC_RR] = rr_new;
    c[SC_ITERS] += 1.0;
    // an exact zero residual ends the system at any rtol (beta would be 0/0 next)
    if (rr_new == 0.0 || (rtol > 0.0 && sqrt(rr_new) <= rtol * sqrt(c[SC_BB]))) {
      c[SC_ACTIVE] = 0.0;
      c[SC_BETA] = 0.0;
    }
  });
}

// x += alpha p (the update kernel's step, SC_XALPHA; also for a system that
// converged in that update), then p = r + beta p with beta from the update
// kernel (0 for a frozen system).  With hy.G: the vector loop covers the
// field entries; block 0 applies the step to x_h (p_h of the step is in p,
// where the update kernel copied it); every block forms the next p_h = r_h +
// beta p_h in shared memory (p_h itself is not written here: every block
// reads it), block 0 stores it to pn, and each block takes a share of the
// bins: dA = G p_h, gsum = 0 (the next product's bin sums).
template <typename T>
__global__ void __launch_bounds__(CG_THREADS, 4) k_cg_pupdate(T* x, T* p, const T* r, int64_t n, int64_t S,
                                                          const double* sc, CGHyper hy, T* pn) {
  const int b = blockIdx.y;
  const double* c = sc + b * SC_N;
  const bool fused = hy.G != nullptr;
  const int rows = fused ? (hy.nb + gridDim.x - 1) / gridDim.x : 0;
  const int i0 = blockIdx.x * rows, i1 = fused ? min(hy.nb, i0 + rows) : 0;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) hy.gsum[(int64_t)b * hy.nb + i] = 0.0;
  const bool active = c[SC_ACTIVE] != 0.0;
  const T xa = T(c[SC_XALPHA]);
  const bool step = xa != T(0);
  if (!active && !step) return;
  const T beta = T(c[SC_BETA]);
  const int64_t off = (int64_t)b * S;
  constexpr int U = 2;
  for_vec_u<T, U>(
      fused ? hy.N : n, blockIdx.x, gridDim.x,
      [&](const int64_t (&idx)[U], const bool (&ok)[U]) {
        V16<T> ri[U], pi[U], xi[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (ok[u]) {
            pi[u] = ldv(p + off + idx[u]);
            if (active) ri[u] = ldv(r + off + idx[u]);
            if (step) xi[u] = ldv(x + off + idx[u]);
          }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (ok[u]) {
            if (step) {
#pragma unroll
              for (int k = 0; k < V16<T>::W; ++k) xi[u].e[k] += xa * pi[u].e[k];
              stv(x + off + idx[u], xi[u]);
            }
            if (active) {
#pragma unroll
              for (int k = 0; k < V16<T>::W; ++k) pi[u].e[k] = ri[u].e[k] + beta * pi[u].e[k];
              stv(p + off + idx[u], pi[u]);
            }
          }
      },
      [&](int64_t i) {
        const T pv = p[off + i];
        if (step) x[off + i] += xa * pv;
        if (active) p[off + i] = r[off + i] + beta * pv;
      });
  if (fused && step && blockIdx.x == 0)
    for (int h = threadIdx.x; h < hy.nh; h += blockDim.x) {
      const int64_t e = off + hy.N + h;
      x[e] += xa * p[e];
    }
  if (!fused || !active || i0 >= i1) return;
  __shared__ float4 sp4[256];
  float* sp = reinterpret_cast<float*>(sp4);
  const int nh4 = (hy.nh + 3) >> 2;
  for (int h = threadIdx.x; h < 4 * nh4; h += blockDim.x) {
    float v = 0.f;
    if (h < hy.nh) {
      const int64_t e = off + hy.N + h;
      const T ph = r[e] + beta * p[e];
      if (blockIdx.x == 0) pn[(int64_t)b * hy.nh + h] = ph;
      v = float(ph);
    }
    sp[h] = v;
  }
  __syncthreads();
  // two rows of G per warp and round (a row: nh4 16-byte vectors)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const float4* G4 = reinterpret_cast<const float4*>(hy.G);
  for (int ib = i0 + 2 * wid; ib < i1; ib += 16) {
    float t[2] = {0.f, 0.f};
    for (int j0 = 0; j0 < nh4; j0 += 160) {
      float4 gv[2][5];
#pragma unroll
      for (int qr = 0; qr < 2; ++qr)
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          const int j = j0 + lane + 32 * k;
          gv[qr][k] = (ib + qr < i1 && j < nh4) ? __ldg(G4 + (int64_t)(ib + qr) * nh4 + j)
                                                 : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const int j = j0 + lane + 32 * k;
        if (j < nh4) {
          const float4 a4 = sp4[j];
#pragma unroll
          for (int qr = 0; qr < 2; ++qr) t[qr] += dot4(gv[qr][k], a4);
        }
      }
    }
    t[0] = warp_sum_f(t[0]);
    t[1] = warp_sum_f(t[1]);
    const int i = ib + (lane & 1);
    if (lane < 2 && i < i1) hy.dA[(int64_t)b * hy.nb + i] = double(lane == 0 ? t[0] : t[1]);
  }
}

template <typename T>
struct CGWork {
  T *r, *p, *q;
  double *sc, *part_a, *part_b;
  unsigned* counter;
  int nblk;
  CGHyper hy;  // hy.G == nullptr: the metric product handles the hyper block
  T* pn;
};

// The CG kernels take over the hyper block of FP32 power-model products
// (CGHyper) when the metric has the linearised amplitude model and the latent
// vector is exactly [field, hyper-parameters].
template <typename T>
CGHyper cg_hyper(nre_metric* m) {
  CGHyper h{};
  const nre_cf_plan* p = m->cf;
  if (sizeof(T) != 4 || m->model_kind != NRE_MODEL_CF || !m->amp_lin || m->precond != NRE_PRECOND_NONE ||
      p == nullptr || p->n_hyper <= 0 || m->latent != p->N + p->n_hyper)
    return h;
  h.G = m->amp_G.as<float>();
  h.Gt = m->amp_Gt.as<float>();
  h.dA = m->dA.as<double>();
  h.gsum = m->gsum.as<double>();
  h.nb = p->n_bins;
  h.nh = p->n_hyper;
  h.N = p->N;
  return h;
}

template <typename T>
CGWork<T> cg_work(nre_metric* m, int B) {
  CGWork<T> w;
  w.nblk = cg_blocks(m->latent, B);
  w.r = m->cg_r.as<T>();
  w.p = m->cg_p.as<T>();
  w.q = m->cg_q.as<T>();
  w.sc = m->cg_sc.as<double>();
  w.part_a = m->cg_part.as<double>();
  w.part_b = w.part_a + (size_t)B * w.nblk;
  w.counter = reinterpret_cast<unsigned*>(w.part_b + (size_t)B * w.nblk);
  w.hy = cg_hyper<T>(m);
  w.pn = m->cg_pn.as<T>();
  return w;
}

// Workspace, x = 0, r = p = b and the initial scalars; enqueue only.
template <typename T>
int cg_begin_t(nre_metric* m, const T* b, T* x, int B, double rtol, cudaStream_t st) {
  const int64_t n = m->latent, S = m->stride;
  NRE_TRY(ensure(m->cg_r, (size_t)B * S * sizeof(T)));
  NRE_TRY(ensure(m->cg_p, (size_t)B * S * sizeof(T)));
  NRE_TRY(ensure(m->cg_q, (size_t)B * S * sizeof(T)));
  NRE_TRY(ensure(m->cg_sc, (size_t)B * SC_N * sizeof(double)));
  const int nblk = cg_blocks(n, B);
  NRE_TRY(ensure(m->cg_part, (size_t)2 * B * nblk * sizeof(double) + (size_t)B * sizeof(unsigned)));
  if (m->model_kind == NRE_MODEL_CF) NRE_TRY(ensure(m->cg_dot, (size_t)B * kDotStride * sizeof(double)));
  if (cg_hyper<T>(m).G != nullptr) NRE_TRY(ensure(m->cg_pn, (size_t)B * m->cf->n_hyper * sizeof(T)));
  const CGWork<T> w = cg_work<T>(m, B);
  NRE_TRY_CUDA(cudaMemsetAsync(w.counter, 0, (size_t)B * sizeof(unsigned), st));
  const dim3 grid(nblk, B);
  const double vb = (double)B * n * sizeof(T);
  prof_begin("cg_init", 4 * vb, st);
  k_cg_init<T><<<grid, CG_THREADS, 0, st>>>(b, x, w.r, w.p, n, S, w.part_a);
  prof_end(st);
  prof_begin("cg_scalars", 0.0, st);
  k_cg_start<<<B, 32, 0, st>>>(w.sc, w.part_a, nblk, rtol);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  if (w.hy.G != nullptr) {
    // p_0 = b: its hyper block into pn, its dA, zero bin sums
    const int64_t N = w.hy.N;
    NRE_TRY_CUDA(cudaMemcpy2DAsync(w.pn, (size_t)w.hy.nh * sizeof(T), w.p + N, (size_t)S * sizeof(T),
                                   (size_t)w.hy.nh * sizeof(T), B, cudaMemcpyDeviceToDevice, st));
    NRE_TRY(amp_jvp_lin<T>(w.hy.G, w.hy.nb, w.hy.nh, w.p + N, S, w.hy.dA, B, st, w.hy.gsum));
  }
  return NRE_OK;
}

// `iters` iterations on the state left by cg_begin_t; enqueue only.
template <typename T>
int cg_iter_t(nre_metric* m, T* x, int B, int iters, double rtol, cudaStream_t st) {
  const int64_t n = m->latent, S = m->stride;
  const CGWork<T> w = cg_work<T>(m, B);
  const dim3 grid(w.nblk, B);
  const double vb = (double)B * n * sizeof(T);
  // correlated field: p.q comes fused with the metric product
  double* pq = m->model_kind == NRE_MODEL_CF ? m->cg_dot.as<double>() : nullptr;
  for (int it = 0; it < iters; ++it) {
    NRE_TRY(metric_apply_impl(m, w.p, w.q, B, st, pq, w.hy.G != nullptr && pq != nullptr));
    if (!pq) {
      prof_begin("cg_dot", 2 * vb, st);
      k_cg_dot<T><<<grid, CG_THREADS, 0, st>>>(w.p, w.q, n, S, w.part_a, w.counter, w.sc);
      prof_end(st);
    }
    prof_begin("cg_update", 3 * vb, st);
    k_cg_update<T><<<grid, CG_THREADS, 0, st>>>(w.r, w.p, w.q, n, S, w.sc, w.part_b, w.counter, rtol, pq,
                                                 pq ? w.hy : CGHyper{}, w.pn);
    prof_end(st);
    prof_begin("cg_pupdate", 5 * vb, st);
    k_cg_pupdate<T><<<grid, CG_THREADS, 0, st>>>(x, w.p, w.r, n, S, w.sc, pq ? w.hy : CGHyper{}, w.pn);
    prof_end(st);
    NRE_CHECK_LAUNCH();
  }
  return NRE_OK;
}

template <typename T>
int cg_t(nre_metric* m, const T* b, T* x, int B, double rtol, int maxiter, int* iters_out,
         double* relres_out, cudaStream_t st) {
  NRE_TRY(cg_begin_t<T>(m, b, x, B, rtol, st));
  const int check_every = 8;
  for (int it = 0; it < maxiter; it += check_every) {
    const int k = maxiter - it < check_every ? maxiter - it : check_every;
    NRE_TRY(cg_iter_t<T>(m, x, B, k, rtol, st));
    if (rtol > 0.0 && it + k < maxiter) {
      NRE_TRY(cg_read_scalars(m, B, st));
      if (!cg_any_active(m, B)) break;
    }
  }
  NRE_TRY(cg_read_scalars(m, B, st));
  return cg_report(m, B, rtol, maxiter, iters_out, relres_out, "CG");
}

}  // namespace

namespace nre {
int cg_read_scalars(nre_metric* m, int B, cudaStream_t st) {
  m->cg_host.resize((size_t)B * CG_SC_N);
  NRE_TRY_CUDA(cudaMemcpyAsync(m->cg_host.data(), m->cg_sc.p, (size_t)B * CG_SC_N * sizeof(double),
                               cudaMemcpyDeviceToHost, st));
  NRE_TRY_CUDA(cudaStreamSynchronize(st));
  return NRE_OK;
}

bool cg_any_active(const nre_metric* m, int B) {
  for (int i = 0; i < B; ++i)
    if (m->cg_host[(size_t)i * CG_SC_N + CG_SC_ACTIVE] != 0.0) return true;
  return false;
}

int cg_report(const nre_metric* m, int B, double rtol, int maxiter, int* iters_out, double* relres_out,
              const char* what) {
  bool conv = true;
  for (int i = 0; i < B; ++i) {
    const double* c = &m->cg_host[(size_t)i * CG_SC_N];
    const double rel = c[CG_SC_BB] > 0 ? std::sqrt(c[CG_SC_RR] / c[CG_SC_BB]) : 0.0;
    if (iters_out) iters_out[i] = (int)c[CG_SC_ITERS];
    if (relres_out) relres_out[i] = rel;
    if (rtol > 0.0 && rel > rtol) conv = false;
  }
  if (!conv) return set_error(NRE_ENOTCONV, "%s: some system missed rtol=%g within maxiter=%d", what, rtol, maxiter);
  return NRE_OK;
}

int cg_begin(nre_metric* m, const void* b, void* x, int B, double rtol, cudaStream_t st) {
  if (m->precond != NRE_PRECOND_NONE) return pcg_begin(m, b, x, B, rtol, st);
  if (m->dtype == NRE_F64) return cg_begin_t<double>(m, (const double*)b, (double*)x, B, rtol, st);
  return cg_begin_t<float>(m, (const float*)b, (float*)x, B, rtol, st);
}

int cg_iterate(nre_metric* m, void* x, int B, int iters, double rtol, cudaStream_t st) {
  if (m->precond != NRE_PRECOND_NONE) return pcg_iterate(m, x, B, iters, rtol, st);
  if (m->dtype == NRE_F64) return cg_iter_t<double>(m, (double*)x, B, iters, rtol, st);
  return cg_iter_t<float>(m, (float*)x, B, iters, rtol, st);
}
}  // namespace nre

extern "C" int cg_solve(nre_metric* m, const void* b, void* x, int batch, double rtol, int maxiter,
                        int* iters_out, double* relres_out, nre_stream_t stream) {
  clear_error();
  if (!m) return set_error(NRE_EINVAL, "metric must not be NULL");
  if (batch < 0 || batch > m->max_batch) return set_error(NRE_EINVAL, "batch %d outside [0, max_batch=%d]", batch, m->max_batch);
  if (maxiter < 0 || !(rtol >= 0.0)) return set_error(NRE_EINVAL, "maxiter must be >= 0 and rtol >= 0");
  if (batch == 0) return NRE_OK;
  if (!b || !x) return set_error(NRE_EINVAL, "NULL array argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (m->precond != NRE_PRECOND_NONE)
    return pcg_solve_impl(m, b, x, batch, rtol, maxiter, iters_out, relres_out, st);
  if (m->dtype == NRE_F64)
    return cg_t<double>(m, (const double*)b, (double*)x, batch, rtol, maxiter, iters_out, relres_out, st);
  return cg_t<float>(m, (const float*)b, (float*)x, batch, rtol, maxiter, iters_out, relres_out, st);
}
