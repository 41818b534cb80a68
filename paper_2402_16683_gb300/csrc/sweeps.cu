// Hartley sweeps of the correlated field: one HBM pass per sweep, each a batch
// of 1-D DHTs along one axis with fused prologue / middle / epilogue.
//
// Row sweep (last, contiguous axis).  A unit is a reflection orbit of rows of
// one sample (D = 2: rows {i, -i}; D = 3: rows {(+-i0, +-i1)}), or for D = 1 a
// pair of samples.  Two real rows form one complex line; after the FFT a thread
// owns the positions x and -x of every line of its unit, so the Hartley unpack,
// the reflection combination P and the epilogue run in registers.
//
// Column sweep (any other axis).  A unit is W adjacent grid columns of one
// outer index; columns 2p and 2p+1 form complex line p, which is one aligned
// 2-element vector load per position, so loads and stores stay coalesced.  The
// axis-0 sweep of the metric runs the first transform's last DHT, t = w * y and
// the second transform's first DHT back to back in shared memory.
#include "sweeps_launch.cuh"

namespace nre {

NRE_DECL_SWEEP_T(float)
NRE_DECL_SWEEP_T(double)

constexpr int SWEEP_THREADS = 256;

template <typename T, int PM, bool MID>
__global__ void __launch_bounds__(SWEEP_THREADS) k_row_sweep(RowArgs<T> a) {
  typedef typename CplxT<T>::type C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int LPU = (PM == 3) ? 2 : 1;  // complex lines per unit
  const int L = a.L, Lh = L >> 1;
  const int nl = a.nU * LPU;
  const LayRow lay{LayRow::stride(L)};
  C* bufA = reinterpret_cast<C*>(smem_raw);
  C* bufB = bufA + nl * lay.ls;
  // warp-private bin histograms: per warp nhist regions of nb (see warp_run_add)
  double* hist = reinterpret_cast<double*>(bufB + nl * lay.ls);
  const int nhist = (PM == 1) ? 2 * a.nU : 1;
  constexpr int NW = SWEEP_THREADS / 32;
  const bool bins = a.epi.mode == EPI_AMP && a.epi.bins;
  double* whist = hist + (threadIdx.x >> 5) * nhist * a.nb;
  if (bins)
    for (int i = threadIdx.x; i < NW * nhist * a.nb; i += blockDim.x) hist[i] = 0.0;
  const int bsample = (PM == 1) ? 0 : blockIdx.y;
  // output of one value; with bins its contribution goes to key keybase + bin
  // (every lane of the warp calls this, `ok` false for lanes without output)
  auto put = [&](int sb, int64_t flat, T val, int keybase, bool ok) {
    int bn = -1;
    T c = T(0);
    if (ok) a.epi.store(sb, flat, val, bn, c);
    if (bins) warp_run_add(bn >= 0 ? keybase + bn : -1, c, whist);
  };

  for (int u0 = blockIdx.x * a.nU; u0 < a.n_units; u0 += gridDim.x * a.nU) {
    // ---- load (prologue)
    for (int q = threadIdx.x; q < nl * L; q += blockDim.x) {
      const int line = q / L, x = q - line * L;
      const int u = line / LPU, li = line - u * LPU;
      const int unit = u0 + u;
      T re = T(0), im = T(0);
      if (unit < a.n_units) {
        if (PM == 1) {
          const int s0 = 2 * unit;
          re = a.pro.load(s0, x);
          if (s0 + 1 < a.B) im = a.pro.load(s0 + 1, x);
        } else {
          const int G = 2 * LPU;
          const int r0 = a.grows[unit * G + 2 * li], r1 = a.grows[unit * G + 2 * li + 1];
          re = a.pro.load(bsample, (int64_t)r0 * L + x);
          im = a.pro.load(bsample, (int64_t)r1 * L + x);
        }
      }
      bufA[lay.idx(line, x)] = cmake<C>(re, im);
    }
    __syncthreads();
    C* Z = block_fft(bufA, bufB, nl, L, a.log2L, a.tw, a.log2Lmax, lay);
    if constexpr (MID) {
      // D = 1 only: y = H u, t = w * y, then the second transform.
      for (int q = threadIdx.x; q < a.nU * (Lh + 1); q += blockDim.x) {
        const int u = q / (Lh + 1), x = q - u * (Lh + 1);
        const int xm = (L - x) & (L - 1);
        C z = Z[lay.idx(u, x)], zm = Z[lay.idx(u, xm)];
        T ha[2], hb[2];
        hartley_unpack<T>(z, zm, ha, hb);
        // the pair's samples 2 unit (real part) and 2 unit + 1 (imaginary part)
        const int sa = 2 * (u0 + u) < a.B ? 2 * (u0 + u) : a.B - 1;
        const int sb = sa + 1 < a.B ? sa + 1 : sa;
        Z[lay.idx(u, x)] = cmake<C>(a.mid.at(sa, x) * ha[0], a.mid.at(sb, x) * hb[0]);
        if (xm != x) Z[lay.idx(u, xm)] = cmake<C>(a.mid.at(sa, xm) * ha[1], a.mid.at(sb, xm) * hb[1]);
      }
      __syncthreads();
      C* other = (Z == bufA) ? bufB : bufA;
      Z = block_fft(Z, other, nl, L, a.log2L, a.tw, a.log2Lmax, lay);
    }
    // ---- unpack, P, epilogue (trip count uniform over the block: the bin
    // sums reduce over whole warps)
    const int nq = a.nU * (Lh + 1);
    for (int q0 = 0; q0 < nq; q0 += blockDim.x) {
      const int q = q0 + threadIdx.x;
      const int u = q < nq ? q / (Lh + 1) : 0, x = q < nq ? q - u * (Lh + 1) : 0;
      const int unit = u0 + u;
      const bool act = q < nq && unit < a.n_units;
      const int xm = (L - x) & (L - 1);
      if (PM == 1) {
        T ha[2], hb[2];
        hartley_unpack<T>(Z[lay.idx(u, x)], Z[lay.idx(u, xm)], ha, hb);
        const int s0 = 2 * unit;
        const int k0 = (2 * u) * a.nb;
        put(s0, x, ha[0], k0, act);
        put(s0, xm, ha[1], k0, act && xm != x);
        put(s0 + 1, x, hb[0], k0 + a.nb, act && s0 + 1 < a.B);
        put(s0 + 1, xm, hb[1], k0 + a.nb, act && s0 + 1 < a.B && xm != x);
      } else if (PM == 2) {
        T R[2][2];
        hartley_unpack<T>(Z[lay.idx(u, x)], Z[lay.idx(u, xm)], R[0], R[1]);
        const bool f0 = act && (a.gflags[unit] & 1);
        const T half = T(0.5);
        T V[2][2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
#pragma unroll
          for (int p = 0; p < 2; ++p)
            V[s][p] = half * (R[s][p] + pick2(R, s, f0, p) + R[s][1 - p] - pick2(R, s, f0, 1 - p));
        }
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int64_t row = act ? a.grows[unit * 2 + s] : 0;
          put(bsample, row * L + x, V[s][0], 0, act);
          put(bsample, row * L + xm, V[s][1], 0, act && xm != x);
        }
      } else {
        T R[4][2];
        hartley_unpack<T>(Z[lay.idx(2 * u, x)], Z[lay.idx(2 * u, xm)], R[0], R[1]);
        hartley_unpack<T>(Z[lay.idx(2 * u + 1, x)], Z[lay.idx(2 * u + 1, xm)], R[2], R[3]);
        const int fl = act ? a.gflags[unit] : 0;
        const bool f0 = fl & 1, f1 = fl & 2;
        const T half = T(0.5);
        T V[4][2];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
#pragma unroll
          for (int p = 0; p < 2; ++p)
            V[s][p] = half * (pick4(R, s, f0, false, p) + pick4(R, s, false, f1, p) + R[s][1 - p] -
                              pick4(R, s, f0, f1, 1 - p));
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int64_t row = act ? a.grows[unit * 4 + s] : 0;
          put(bsample, row * L + x, V[s][0], 0, act);
          put(bsample, row * L + xm, V[s][1], 0, act && xm != x);
        }
      }
    }
    __syncthreads();
  }
  if (bins) {
    __syncthreads();
    if (PM == 1) {
      // one CTA holds every pixel of its sample pairs: complete sums, the
      // warps' histograms folded in warp order
      for (int i = threadIdx.x; i < nhist * a.nb; i += blockDim.x) {
        const int hs = i / a.nb, bn = i - hs * a.nb;
        const int sample = 2 * (blockIdx.x * a.nU) + hs;
        double tot = 0.0;
        for (int w = 0; w < NW; ++w) tot += hist[w * nhist * a.nb + i];
        if (sample < a.B) (a.epi.gsum ? a.epi.gsum : a.partials)[(int64_t)sample * a.nb + bn] = tot;
      }
    } else {
      fold_bins(a.epi, a.partials, bsample, gridDim.x, blockIdx.x, hist, NW, a.nb, a.nb);
    }
  }
}

template <typename T, bool MID>
__global__ void __launch_bounds__(SWEEP_THREADS) k_col_sweep(ColArgs<T> a) {
  typedef typename CplxT<T>::type C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = a.L, Lh = L >> 1;
  const int nl = a.W >> 1;
  const LayCol lay{nl};
  C* bufA = reinterpret_cast<C*>(smem_raw);
  C* bufB = bufA + nl * L;
  double* hist = reinterpret_cast<double*>(bufB + nl * L);  // warp-private regions of nb
  constexpr int NW = SWEEP_THREADS / 32;
  double* whist = hist + (threadIdx.x >> 5) * a.nb;
  const bool bins = a.epi.mode == EPI_AMP && a.epi.bins;
  if (bins)
    for (int i = threadIdx.x; i < NW * a.nb; i += blockDim.x) hist[i] = 0.0;
  const int b = blockIdx.y;
  auto put = [&](int64_t flat, T val, bool ok) {
    int bn = -1;
    T c = T(0);
    if (ok) a.epi.store(b, flat, val, bn, c);
    if (bins) warp_run_add(bn, c, whist);
  };

  for (int64_t unit = blockIdx.x; unit < a.n_units; unit += gridDim.x) {
    const int64_t o = unit / a.nblk;
    const int64_t c0 = (unit - o * a.nblk) * a.W;
    const int64_t base = o * L * a.inner + c0;
    for (int q = threadIdx.x; q < nl * L; q += blockDim.x) {
      const int l = q / nl, p = q - l * nl;
      const int64_t flat = base + (int64_t)l * a.inner + 2 * p;
      bufA[lay.idx(p, l)] = cmake<C>(a.pro.load(b, flat), a.pro.load(b, flat + 1));
    }
    __syncthreads();
    C* Z = block_fft(bufA, bufB, nl, L, a.log2L, a.tw, a.log2Lmax, lay);
    if constexpr (MID) {
      for (int q = threadIdx.x; q < nl * (Lh + 1); q += blockDim.x) {
        const int l = q / nl, p = q - l * nl;
        const int lm = (L - l) & (L - 1);
        T ha[2], hb[2];
        hartley_unpack<T>(Z[lay.idx(p, l)], Z[lay.idx(p, lm)], ha, hb);
        const int64_t f0 = base + (int64_t)l * a.inner + 2 * p;
        const int64_t f1 = base + (int64_t)lm * a.inner + 2 * p;
        Z[lay.idx(p, l)] = cmake<C>(a.mid.apply(b, f0, ha[0]), a.mid.apply(b, f0 + 1, hb[0]));
        if (lm != l) Z[lay.idx(p, lm)] = cmake<C>(a.mid.apply(b, f1, ha[1]), a.mid.apply(b, f1 + 1, hb[1]));
      }
      __syncthreads();
      C* other = (Z == bufA) ? bufB : bufA;
      Z = block_fft(Z, other, nl, L, a.log2L, a.tw, a.log2Lmax, lay);
    }
    const int nq = nl * (Lh + 1);
    for (int q0 = 0; q0 < nq; q0 += blockDim.x) {  // uniform trip count (warp bin sums)
      const int q = q0 + threadIdx.x;
      const bool act = q < nq;
      const int l = act ? q / nl : 0, p = act ? q - l * nl : 0;
      const int lm = (L - l) & (L - 1);
      T ha[2], hb[2];
      hartley_unpack<T>(Z[lay.idx(p, l)], Z[lay.idx(p, lm)], ha, hb);
      const int64_t f0 = base + (int64_t)l * a.inner + 2 * p;
      const int64_t f1 = base + (int64_t)lm * a.inner + 2 * p;
      put(f0, ha[0], act);
      put(f0 + 1, hb[0], act);
      put(f1, ha[1], act && lm != l);
      put(f1 + 1, hb[1], act && lm != l);
    }
    __syncthreads();
  }
  if (bins) {
    __syncthreads();
    fold_bins(a.epi, a.partials, b, gridDim.x, blockIdx.x, hist, NW, a.nb, a.nb);
  }
}

// ------------------------------------------------------------------ launch
namespace {

// Complex lines a row-sweep CTA holds per iteration (>= 2 for D = 3).
int row_lines(int L) { return L >= 2048 ? 1 : 2048 / L; }
// Grid columns a column-sweep unit holds (even, divides inner).
int col_width(int L, int64_t inner, int csize) {
  int budget = (csize == 8) ? 4096 : 2048;  // complex elements per buffer
  int W = 2 * (budget / L);
  if (W > 32) W = 32;
  if (W < 2) W = 2;
  while (W > inner) W >>= 1;
  return W;
}

template <typename T>
size_t row_smem(int L, int nl, int nhist, int nb) {
  return (size_t)2 * nl * LayRow::stride(L) * sizeof(typename CplxT<T>::type) +
         (size_t)nhist * nb * sizeof(double);
}

template <typename T, int PM, bool MID>
int launch_row(const RowArgs<T>& a, dim3 grid, size_t smem, cudaStream_t st, int64_t N) {
  auto k = k_row_sweep<T, PM, MID>;
  NRE_TRY(raise_smem(k, smem));
  prof_begin(row_name(PM, MID, sizeof(T)), sweep_bytes<T>(a.pro, a.epi, &a.mid, MID, a.B, N), st);
  k<<<grid, SWEEP_THREADS, smem, st>>>(a);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  return NRE_OK;
}

template <typename T, bool MID>
int launch_col(const ColArgs<T>& a, dim3 grid, size_t smem, cudaStream_t st, int64_t N) {
  auto k = k_col_sweep<T, MID>;
  NRE_TRY(raise_smem(k, smem));
  const char* name = sizeof(T) == 8 ? (MID ? "col_sweep_f64_metric" : "col_sweep_f64")
                                    : (MID ? "col_sweep_f32_metric" : "col_sweep_f32");
  prof_begin(name, sweep_bytes<T>(a.pro, a.epi, &a.mid, MID, (int)grid.y, N), st);
  k<<<grid, SWEEP_THREADS, smem, st>>>(a);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  return NRE_OK;
}

// ---- register-resident kernels (lines of 8..4096): instantiated per
// (dtype, line length) in sweeps_inst.cu, declared in sweeps_launch.cuh.
#define NRE_L_CASE(K, LL, ...) \
  case K: {                      \
    constexpr int L = LL;        \
    __VA_ARGS__;                 \
  }
#define NRE_L_SWITCH(L2, ...)                \
  switch (L2) {                              \
    NRE_L_CASE(3, 8, __VA_ARGS__)            \
    NRE_L_CASE(4, 16, __VA_ARGS__)           \
    NRE_L_CASE(5, 32, __VA_ARGS__)           \
    NRE_L_CASE(6, 64, __VA_ARGS__)           \
    NRE_L_CASE(7, 128, __VA_ARGS__)          \
    NRE_L_CASE(8, 256, __VA_ARGS__)          \
    NRE_L_CASE(9, 512, __VA_ARGS__)          \
    NRE_L_CASE(10, 1024, __VA_ARGS__)        \
    NRE_L_CASE(11, 2048, __VA_ARGS__)        \
    NRE_L_CASE(12, 4096, __VA_ARGS__)        \
    default: break;                          \
  }

// Register-kernel sweeps.  *handled = false (nothing launched) when the line
// length or the shared-memory budget needs the generic kernels.
template <typename T>
int row_sweep_reg(RowArgs<T> a, bool mid, int B, bool bins, int* nparts, cudaStream_t st, int64_t N,
                  bool* handled) {
  *handled = false;
  dim3 grid;
  size_t smem = 0;
  NRE_L_SWITCH(a.log2L, {
    if (row_reg_plan<T, L>(a, B, bins, &grid, &smem, nparts) != NRE_OK) return NRE_OK;
    *handled = true;
    return row_reg_L<T, L>(a, mid, grid, smem, st, N);
  })
  return NRE_OK;
}

template <typename T>
int col_sweep_reg(ColArgs<T> a, int64_t outer, bool mid, int B, bool bins, int* nparts, cudaStream_t st,
                  int64_t N, bool* handled) {
  *handled = false;
  NRE_L_SWITCH(a.log2L, {
    if (ColSmem<T, L>::bytes(a.nb, bins ? (ColShape<L, sizeof(T)>::NT / 32) * a.nb : 0) > 200 * 1024) return NRE_OK;
    constexpr int CW = ColShape<L, sizeof(T)>::W;
    a.W = CW < a.inner ? CW : (int)a.inner;
    a.nblk = a.inner / a.W;
    a.n_units = outer * a.nblk;
    *handled = true;
    return col_reg_L<T, L>(a, mid, B, bins, nparts, st, N);
  })
  return NRE_OK;
}

// Partials of sum(base * y) over the N outputs of each sample (the fused inner
// product when the row kernel cannot produce it), in the Epi::dot layout.
template <typename T>
__global__ void __launch_bounds__(256) k_dot_fallback(const T* base, int64_t bs, const T* y, int64_t ys,
                                                     int64_t N, double* dot) {
  const int b = blockIdx.y;
  RunSum<T> acc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    acc.add(base[b * bs + i] * y[b * ys + i]);
  const double t = acc.block_sum();
  double* dp = dot + (int64_t)b * kDotStride;
  if (threadIdx.x == 0) dp[blockIdx.x] = t;
  if (blockIdx.x == 0)
    for (int i = gridDim.x + threadIdx.x; i < kDotStride; i += blockDim.x) dp[i] = 0.0;
}

template <typename T>
int row_sweep_dot(const nre_cf_plan* p, int B, const Pro<T>& pro, const Epi<T>& epi,
                  const Mid<T>* mid, double* partials, int* nparts, cudaStream_t st);

template <typename T>
int row_sweep(const nre_cf_plan* p, int B, const Pro<T>& pro, const Epi<T>& epi,
              const Mid<T>* mid, double* partials, int* nparts, cudaStream_t st) {
  if (epi.dot != nullptr) return row_sweep_dot<T>(p, B, pro, epi, mid, partials, nparts, st);
  RowArgs<T> a{};
  const int D = p->ndim;
  a.L = p->n[D - 1];
  a.log2L = p->l2[D - 1];
  a.log2Lmax = p->log2Lmax;
  a.tw = p->tw.as<typename CplxT<T>::type>();
  a.pm = D;
  a.B = B;
  a.pro = pro;
  a.epi = epi;
  if (mid) a.mid = *mid;
  a.nb = p->n_bins > 0 ? p->n_bins : 1;
  a.partials = partials;
  a.grows = p->grows.as<int>();
  a.gflags = p->gflags.as<int>();
  const bool bins = epi.mode == EPI_AMP && epi.bins;
  a.n_units = D == 1 ? (B + 1) / 2 : p->n_groups;
  bool handled = false;
  NRE_TRY(row_sweep_reg<T>(a, mid != nullptr, B, bins, nparts, st, p->N, &handled));
  if (handled) return NRE_OK;
  const int nl = row_lines(a.L);
  dim3 grid;
  int nhist;
  if (D == 1) {
    a.n_units = (B + 1) / 2;
    a.nU = nl < a.n_units ? nl : a.n_units;
    // keep the per-sample histograms (2 per unit, one copy per warp) within
    // 48 KB of shared memory
    const int hist_cap = (epi.mode == EPI_AMP && epi.bins) ? 3072 / (2 * (SWEEP_THREADS / 32) * a.nb) : nl;
    if (a.nU > hist_cap) a.nU = hist_cap < 1 ? 1 : hist_cap;
    grid = dim3((a.n_units + a.nU - 1) / a.nU, 1);
    nhist = 2 * a.nU;
    *nparts = 1;
  } else {
    const int lpu = (D == 3) ? 2 : 1;
    a.nU = nl / lpu < 1 ? 1 : nl / lpu;
    a.n_units = p->n_groups;
    int gx = (a.n_units + a.nU - 1) / a.nU;
    if (gx > kMaxGridX) gx = kMaxGridX;
    grid = dim3(gx, B);
    nhist = 1;
    *nparts = gx;
  }
  const int nlines = a.nU * ((D == 3) ? 2 : 1);
  const size_t smem = row_smem<T>(a.L, nlines, epi.mode == EPI_AMP && epi.bins ? (SWEEP_THREADS / 32) * nhist : 0, a.nb);
  if (D == 1) {
    return mid ? launch_row<T, 1, true>(a, grid, smem, st, p->N) : launch_row<T, 1, false>(a, grid, smem, st, p->N);
  }
  if (mid) return set_error(NRE_EINVAL, "internal: row sweep middle op needs D = 1");
  return D == 2 ? launch_row<T, 2, false>(a, grid, smem, st, p->N) : launch_row<T, 3, false>(a, grid, smem, st, p->N);
}

template <typename T>
int col_sweep(const nre_cf_plan* p, int axis, int B, const Pro<T>& pro, const Epi<T>& epi,
              const Mid<T>* mid, double* partials, int* nparts, cudaStream_t st) {
  ColArgs<T> a{};
  a.L = p->n[axis];
  a.log2L = p->l2[axis];
  a.log2Lmax = p->log2Lmax;
  a.tw = p->tw.as<typename CplxT<T>::type>();
  int64_t inner = 1, outer = 1;
  for (int d = axis + 1; d < p->ndim; ++d) inner *= p->n[d];
  for (int d = 0; d < axis; ++d) outer *= p->n[d];
  a.inner = inner;
  a.pro = pro;
  a.epi = epi;
  if (mid) a.mid = *mid;
  a.nb = p->n_bins > 0 ? p->n_bins : 1;
  a.partials = partials;
  bool handled = false;
  NRE_TRY(col_sweep_reg<T>(a, outer, mid != nullptr, B, epi.mode == EPI_AMP && epi.bins, nparts, st, p->N,
                           &handled));
  if (handled) return NRE_OK;
  a.W = col_width(a.L, inner, (int)sizeof(typename CplxT<T>::type));
  a.nblk = inner / a.W;
  a.n_units = outer * a.nblk;
  a.pro = pro;
  a.epi = epi;
  if (mid) a.mid = *mid;
  a.nb = p->n_bins > 0 ? p->n_bins : 1;
  a.partials = partials;
  int64_t gx = a.n_units < kMaxGridX ? a.n_units : kMaxGridX;
  *nparts = (int)gx;
  const size_t smem = (size_t)2 * (a.W / 2) * a.L * sizeof(typename CplxT<T>::type) +
                      (epi.mode == EPI_AMP && epi.bins ? (size_t)(SWEEP_THREADS / 32) * a.nb * sizeof(double) : 0);
  dim3 grid((unsigned)gx, B);
  return mid ? launch_col<T, true>(a, grid, smem, st, p->N) : launch_col<T, false>(a, grid, smem, st, p->N);
}

template <typename T>
Pro<T> pro_buf(const T* x, int64_t xs) {
  Pro<T> r{};
  r.mode = PRO_BUF;
  r.x = x;
  r.xs = xs;
  return r;
}
template <typename T>
Epi<T> epi_buf(T* y, int64_t ys) {
  Epi<T> r{};
  r.mode = EPI_BUF;
  r.y = y;
  r.ys = ys;
  return r;
}

// row_sweep with the fused inner product: the register kernel of a 2-D / 3-D
// grid accumulates it in its epilogue; otherwise a separate reduction follows.
template <typename T>
int row_sweep_dot(const nre_cf_plan* p, int B, const Pro<T>& pro, const Epi<T>& epi,
                  const Mid<T>* mid, double* partials, int* nparts, cudaStream_t st) {
  Epi<T> e = epi;
  double* dot = e.dot;
  const int64_t N = p->N;
  bool fused = false;
  if (p->ndim >= 2) {
    RowArgs<T> a{};
    const int D = p->ndim;
    a.L = p->n[D - 1];
    a.log2L = p->l2[D - 1];
    a.log2Lmax = p->log2Lmax;
    a.tw = p->tw.as<typename CplxT<T>::type>();
    a.pm = D;
    a.B = B;
    a.pro = pro;
    a.epi = e;
    if (mid) a.mid = *mid;
    a.nb = p->n_bins > 0 ? p->n_bins : 1;
    a.partials = partials;
    a.grows = p->grows.as<int>();
    a.gflags = p->gflags.as<int>();
    a.n_units = p->n_groups;
    NRE_TRY(row_sweep_reg<T>(a, mid != nullptr, B, e.mode == EPI_AMP && e.bins, nparts, st, N, &fused));
  }
  if (!fused) {
    e.dot = nullptr;
    NRE_TRY(row_sweep<T>(p, B, pro, e, mid, partials, nparts, st));
    int64_t gx = (N + 256 * 8 - 1) / (256 * 8);
    if (gx > kMaxGridX) gx = kMaxGridX;
    prof_begin("dot_fallback", (double)B * N * 2 * sizeof(T), st);
    k_dot_fallback<T><<<dim3((unsigned)gx, B), 256, 0, st>>>(e.base, e.bs, e.y, e.ys, N, dot);
    prof_end(st);
    NRE_CHECK_LAUNCH();
  }
  return NRE_OK;
}

}  // namespace

int max_parts(const nre_cf_plan* p) { return kMaxGridX; }

template <typename T>
int run_hartley(const nre_cf_plan* p, int B, const Pro<T>& pro, const Epi<T>& epi,
                const Mid<T>* mid, T* tmp0, T* tmp1, double* partials, int* nparts,
                cudaStream_t st) {
  const int D = p->ndim;
  const int64_t N = p->N;
  int np = 0;
  if (D == 1) return row_sweep<T>(p, B, pro, epi, mid, partials, nparts, st);
  if (D == 2) {
    if (!mid) {
      NRE_TRY(row_sweep<T>(p, B, pro, epi_buf<T>(tmp0, N), nullptr, nullptr, &np, st));
      return col_sweep<T>(p, 0, B, pro_buf<T>(tmp0, N), epi, nullptr, partials, nparts, st);
    }
    NRE_TRY(row_sweep<T>(p, B, pro, epi_buf<T>(tmp0, N), nullptr, nullptr, &np, st));
    NRE_TRY(col_sweep<T>(p, 0, B, pro_buf<T>(tmp0, N), epi_buf<T>(tmp1, N), mid, nullptr, &np, st));
    return row_sweep<T>(p, B, pro_buf<T>(tmp1, N), epi, nullptr, partials, nparts, st);
  }
  // D == 3
  if (!mid) {
    NRE_TRY(row_sweep<T>(p, B, pro, epi_buf<T>(tmp0, N), nullptr, nullptr, &np, st));
    NRE_TRY(col_sweep<T>(p, 1, B, pro_buf<T>(tmp0, N), epi_buf<T>(tmp1, N), nullptr, nullptr, &np, st));
    return col_sweep<T>(p, 0, B, pro_buf<T>(tmp1, N), epi, nullptr, partials, nparts, st);
  }
  NRE_TRY(row_sweep<T>(p, B, pro, epi_buf<T>(tmp0, N), nullptr, nullptr, &np, st));
  NRE_TRY(col_sweep<T>(p, 1, B, pro_buf<T>(tmp0, N), epi_buf<T>(tmp1, N), nullptr, nullptr, &np, st));
  NRE_TRY(col_sweep<T>(p, 0, B, pro_buf<T>(tmp1, N), epi_buf<T>(tmp0, N), mid, nullptr, &np, st));
  NRE_TRY(col_sweep<T>(p, 1, B, pro_buf<T>(tmp0, N), epi_buf<T>(tmp1, N), nullptr, nullptr, &np, st));
  return row_sweep<T>(p, B, pro_buf<T>(tmp1, N), epi, nullptr, partials, nparts, st);
}

template int run_hartley<float>(const nre_cf_plan*, int, const Pro<float>&, const Epi<float>&,
                                const Mid<float>*, float*, float*, double*, int*, cudaStream_t);
template int run_hartley<double>(const nre_cf_plan*, int, const Pro<double>&, const Epi<double>&,
                                 const Mid<double>*, double*, double*, double*, int*, cudaStream_t);

}  // namespace nre
