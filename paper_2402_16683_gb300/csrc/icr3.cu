// Iterative charted refinement on a 3-D chart (Sec. "Gaussian Processes", ICR
// paragraph; the three-dimensional setting of the paper's tomography
// application).
//
// Reading implemented here (no equations in the paper): level l has
// n_l = n0 2^l points per axis at u = (i+1/2)/n_l, v = (j+1/2)/n_l,
// t = (k+1/2)/n_l on a spherical log-radial shell, r = r_min (r_max/r_min)^u,
// polar angle theta = pi v, azimuth phi = 2 pi t; Matern-3/2 kernel;
// s_0 = chol(K0) xi_0 over the n0^3 level-0 points; coarse voxel (i, j, k) with
// its 3x3x3 neighbourhood (radial rows clamp(i-1, 0, n-3) + {0,1,2}, polar rows
// likewise, azimuthal columns k-1..k+1 mod n, ordered 9a + 3b + c) predicts its
// 2x2x2 children (order 4a + 2b + c): s_f = R s_nbhd + L xi_f with
// R = K_fc K_cc^-1 (8 x 27), L = chol(K_ff - R K_cf) (8 x 8).  Rotation about
// the polar axis makes R, L depend on (level, i, j); they are assembled in FP64
// on the host.
//
// Kernels: one CTA per coarse (i, j) row pair and sample, threads along the
// azimuth k with that pair's matrices in shared memory.  The adjoint is
// deterministic and runs in two phases per level: every coarse voxel writes
// L^T g of its children (the excitations' gradient) and the 27 entries of
// R^T g (one per neighbour), then every coarse voxel gathers the entries
// addressed to it from the voxels whose neighbourhood contains it (up to 5
// radial and 5 polar rows near the clamped edges, 3 azimuthal columns).
#include <cmath>
#include <vector>

#include "icr_internal.cuh"

namespace {

using nre::prof_begin;
using nre::prof_end;

constexpr int MAT3 = 280;  // 8 x 27 (R) + 8 x 8 (L)

struct P3 {
  double x, y, z;
};

P3 pos3(const nre_icr_plan* p, int level, int i, int j, int k) {
  const double n = p->sizes[level];
  const double u = (i + 0.5) / n, v = (j + 0.5) / n, t = (k + 0.5) / n;
  const double r = p->r_min * std::pow(p->r_max / p->r_min, u);
  const double th = M_PI * v, ph = 2.0 * M_PI * t;
  return {r * std::sin(th) * std::cos(ph), r * std::sin(th) * std::sin(ph), r * std::cos(th)};
}

double k32(const nre_icr_plan* p, P3 a, P3 b) {
  const double d = std::sqrt((a.x - b.x) * (a.x - b.x) + (a.y - b.y) * (a.y - b.y) + (a.z - b.z) * (a.z - b.z));
  const double x = std::sqrt(3.0) * d / p->rho;
  return p->var * (1.0 + x) * std::exp(-x);
}

// Lower Cholesky of the row-major n x n matrix A in place; false if not SPD.
bool chol(std::vector<double>& A, int n) {
  for (int j = 0; j < n; ++j) {
    double s = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
    if (!(s > 0.0)) return false;
    const double d = std::sqrt(s);
    A[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
      A[(size_t)i * n + j] = t / d;
    }
    for (int k = j + 1; k < n; ++k) A[(size_t)j * n + k] = 0.0;
  }
  return true;
}

bool chol_jitter(std::vector<double> A, int n, double jitter, std::vector<double>& L) {
  L = A;
  if (chol(L, n)) return true;
  for (int i = 0; i < n; ++i) A[(size_t)i * n + i] += jitter;
  L = A;
  return chol(L, n);
}

__host__ __device__ inline int win(int n, int i) {
  int w = i - 1;
  if (w < 0) w = 0;
  if (w > n - 3) w = n - 3;
  return w;
}

// R (8 x 27) and L (8 x 8) of coarse (level, i, j, k = 0) into out[280].
bool pair_matrices(const nre_icr_plan* p, int level, int i, int j, double* out) {
  const int nc = p->sizes[level];
  const int wi = win(nc, i), wj = win(nc, j);
  P3 pc[27], pf[8];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) pc[9 * a + 3 * b + c] = pos3(p, level, wi + a, wj + b, (c - 1 + nc) % nc);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int c = 0; c < 2; ++c) pf[4 * a + 2 * b + c] = pos3(p, level + 1, 2 * i + a, 2 * j + b, c);
  std::vector<double> Kcc(27 * 27), X(27 * 8), Kff(64);
  for (int r = 0; r < 27; ++r)
    for (int c = 0; c < 27; ++c) Kcc[r * 27 + c] = k32(p, pc[r], pc[c]);
  for (int r = 0; r < 27; ++r)
    for (int c = 0; c < 8; ++c) X[r * 8 + c] = k32(p, pc[r], pf[c]);  // K_cf
  const std::vector<double> Kcf = X;
  for (int r = 0; r < 8; ++r)
    for (int c = 0; c < 8; ++c) Kff[r * 8 + c] = k32(p, pf[r], pf[c]);
  std::vector<double> Lcc;
  if (!chol_jitter(Kcc, 27, 1e-10 * p->var, Lcc)) return false;
  for (int c = 0; c < 8; ++c) {  // X = K_cc^-1 K_cf by two triangular solves
    for (int r = 0; r < 27; ++r) {
      double s = X[r * 8 + c];
      for (int k = 0; k < r; ++k) s -= Lcc[r * 27 + k] * X[k * 8 + c];
      X[r * 8 + c] = s / Lcc[r * 27 + r];
    }
    for (int r = 26; r >= 0; --r) {
      double s = X[r * 8 + c];
      for (int k = r + 1; k < 27; ++k) s -= Lcc[k * 27 + r] * X[k * 8 + c];
      X[r * 8 + c] = s / Lcc[r * 27 + r];
    }
  }
  for (int m = 0; m < 8; ++m)
    for (int n = 0; n < 27; ++n) out[m * 27 + n] = X[n * 8 + m];  // R = X^T
  std::vector<double> D(64);
  for (int r = 0; r < 8; ++r)
    for (int c = 0; c < 8; ++c) {
      double s = Kff[r * 8 + c];
      for (int n = 0; n < 27; ++n) s -= out[r * 27 + n] * Kcf[n * 8 + c];
      D[r * 8 + c] = s;
    }
  for (int r = 0; r < 8; ++r)
    for (int c = 0; c < r; ++c) D[r * 8 + c] = D[c * 8 + r] = 0.5 * (D[r * 8 + c] + D[c * 8 + r]);
  std::vector<double> LD;
  if (!chol_jitter(D, 8, 1e-10 * p->var, LD)) return false;
  for (int k = 0; k < 64; ++k) out[216 + k] = LD[k];
  return true;
}

// ---------------------------------------------------------------- kernels
// s0[b] = L0 xi0[b]: one warp per output row.
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

template <typename T>
__global__ void k_icr3_level0(const T* L0, const T* xi, int64_t xs, T* s0, int64_t ss, int n) {
  const int b = blockIdx.y, lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const T* x = xi + b * xs;
  T acc = T(0);
  for (int c = lane; c <= row; c += 32) acc += L0[(int64_t)row * n + c] * x[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) s0[b * ss + row] = acc;
}

// out[b] = (base ? base[b] : 0) + L0^T g0[b] over the level-0 latent entries.
template <typename T>
__global__ void k_icr3_level0_t(const T* L0, const T* g0, int64_t gs, T* out, int64_t os, const T* base,
                                int64_t bs, int n) {
  const int b = blockIdx.y, lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= n) return;
  const T* g = g0 + b * gs;
  T acc = T(0);
  for (int r = col + lane; r < n; r += 32) acc += L0[(int64_t)r * n + col] * g[r];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[b * os + col] = (base ? base[b * bs + col] : T(0)) + acc;
}

// One refinement: coarse level sc (nc^3) -> fine level sf ((2nc)^3) for the
// (i, j) pair blockIdx.x and sample blockIdx.y; scale (optional) multiplies
// the fine values (the metric's weights on the last level).
template <typename T>
__global__ void __launch_bounds__(128) k_icr3_refine(int nc, const T* __restrict__ mats, const T* sc, int64_t scs,
                                                    const T* xif, int64_t xs, T* sf, int64_t sfs,
                                                    const T* __restrict__ scale) {
  __shared__ T M[MAT3];
  const int i = blockIdx.x / nc, j = blockIdx.x - i * nc, b = blockIdx.y;
  for (int e = threadIdx.x; e < MAT3; e += blockDim.x) M[e] = mats[(int64_t)blockIdx.x * MAT3 + e];
  __syncthreads();
  const int wi = win(nc, i), wj = win(nc, j), nf = 2 * nc;
  const T* c = sc + b * scs;
  const T* x = xif + b * xs;
  T* f = sf + b * sfs;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    T nb[27];
    const int km = k == 0 ? nc - 1 : k - 1, kp = k == nc - 1 ? 0 : k + 1;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int bb = 0; bb < 3; ++bb) {
        const T* rowp = c + ((int64_t)(wi + a) * nc + (wj + bb)) * nc;
        nb[9 * a + 3 * bb + 0] = rowp[km];
        nb[9 * a + 3 * bb + 1] = rowp[k];
        nb[9 * a + 3 * bb + 2] = rowp[kp];
      }
    T xe[8];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int bb = 0; bb < 2; ++bb) {
        const int64_t o = ((int64_t)(2 * i + a) * nf + (2 * j + bb)) * nf + 2 * k;
        xe[4 * a + 2 * bb] = x[o];
        xe[4 * a + 2 * bb + 1] = x[o + 1];
      }
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      T acc = T(0);
#pragma unroll
      for (int n = 0; n < 27; ++n) acc += M[m * 27 + n] * nb[n];
#pragma unroll
      for (int q = 0; q <= m; ++q) acc += M[216 + m * 8 + q] * xe[q];
      const int a = m >> 2, bb = (m >> 1) & 1, cc = m & 1;
      const int64_t o = ((int64_t)(2 * i + a) * nf + (2 * j + bb)) * nf + 2 * k + cc;
      f[o] = scale ? acc * scale[o] : acc;
    }
  }
}

// Forward with four consecutive coarse voxels (k0 .. k0 + 3) per thread, for
// coarse sides of 64 and up (nc % 4 == 0): each matrix entry read from shared
// memory serves four voxels, the 3 x 3 neighbourhood rows move as 16-byte
// vectors plus one halo value on either side (periodic in k), and the
// children of each (a, b) child row go out as two 16-byte stores.  A CTA of
// 128 threads covers 128 / (nc / 4) pairs (i, j), each with its matrices in
// shared memory.  Same arithmetic and order per output as k_icr3_refine.
constexpr int ICR3_T = 128;

template <typename T>
__global__ void __launch_bounds__(ICR3_T, 4) k_icr3_refine4(int nc, const T* __restrict__ mats, const T* sc,
                                                            int64_t scs, const T* xif, int64_t xs, T* sf, int64_t sfs,
                                                            const T* __restrict__ scale) {
  extern __shared__ __align__(16) unsigned char sm3_raw[];
  T* Ms = reinterpret_cast<T*>(sm3_raw);
  const int tp = nc / 4, pp = ICR3_T / tp;  // threads per pair, pairs per CTA
  const int b = blockIdx.y;
  const int64_t pair0 = (int64_t)blockIdx.x * pp;
  for (int e = threadIdx.x; e < pp * MAT3; e += blockDim.x) Ms[e] = mats[pair0 * MAT3 + e];
  __syncthreads();
  const int pl = threadIdx.x / tp, t = threadIdx.x - pl * tp;
  const int64_t pair = pair0 + pl;
  const int i = (int)(pair / nc), j = (int)(pair - (int64_t)i * nc);
  const T* M = Ms + pl * MAT3;
  const int wi = win(nc, i), wj = win(nc, j), nf = 2 * nc;
  const int k0 = 4 * t;
  const int km = k0 == 0 ? nc - 1 : k0 - 1, kp = k0 + 4 == nc ? 0 : k0 + 4;
  const T* c = sc + b * scs;
  // neighbourhood rows (A, B): entries k0 - 1 .. k0 + 4
  T nbv[9][6];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int bb = 0; bb < 3; ++bb) {
      const T* rowp = c + ((int64_t)(wi + a) * nc + (wj + bb)) * nc;
      T* r = nbv[3 * a + bb];
      r[0] = rowp[km];
      ld4v(rowp + k0, r + 1);
      r[5] = rowp[kp];
    }
  // excitations of the children rows (a, b): entries 2 k0 .. 2 k0 + 7
  T xe[4][8];
  const T* x = xif + b * xs;
#pragma unroll
  for (int ab = 0; ab < 4; ++ab) {
    const int64_t o = ((int64_t)(2 * i + (ab >> 1)) * nf + (2 * j + (ab & 1))) * nf + 2 * k0;
    ld4v(x + o, xe[ab]);
    ld4v(x + o + 4, xe[ab] + 4);
  }
  T* f = sf + b * sfs;
#pragma unroll
  for (int ab = 0; ab < 4; ++ab) {
    T out[8];  // entry 2 kk + cc
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
      const int m = 2 * ab + cc;
      T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int n = 0; n < 27; ++n) {
        const T w = M[m * 27 + n];
        const T* r = nbv[n / 3];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) acc[kk] += w * r[kk + n % 3];
      }
#pragma unroll
      for (int q = 0; q <= m; ++q) {
        const T w = M[216 + m * 8 + q];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) acc[kk] += w * xe[q >> 1][2 * kk + (q & 1)];
      }
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) out[2 * kk + cc] = acc[kk];
    }
    const int64_t o = ((int64_t)(2 * i + (ab >> 1)) * nf + (2 * j + (ab & 1))) * nf + 2 * k0;
    if (scale) {
      T sv[8];
      ld4v(scale + o, sv);
      ld4v(scale + o + 4, sv + 4);
#pragma unroll
      for (int e = 0; e < 8; ++e) out[e] *= sv[e];
    }
    st4v(f + o, out);
    st4v(f + o + 4, out + 4);
  }
}

// Adjoint phase 1: for the children gradient gf of coarse voxel (i, j, k):
// gxi = L^T gf into the excitations' gradient (plus base), U[n][v] = (R^T gf)_n
// (27 planes of stride ps, so that both phases read and write along k).
template <typename T>
__global__ void __launch_bounds__(128) k_icr3_refine_t1(int nc, const T* __restrict__ mats, const T* gf, int64_t gfs,
                                                       T* gxi, int64_t gxs, const T* base, int64_t bs, T* U,
                                                       int64_t us, int64_t ps) {
  __shared__ T M[MAT3];
  const int i = blockIdx.x / nc, j = blockIdx.x - i * nc, b = blockIdx.y;
  for (int e = threadIdx.x; e < MAT3; e += blockDim.x) M[e] = mats[(int64_t)blockIdx.x * MAT3 + e];
  __syncthreads();
  const int nf = 2 * nc;
  const T* g = gf + b * gfs;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    T ge[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int a = m >> 2, bb = (m >> 1) & 1, cc = m & 1;
      ge[m] = g[((int64_t)(2 * i + a) * nf + (2 * j + bb)) * nf + 2 * k + cc];
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      T acc = T(0);
#pragma unroll
      for (int m = q; m < 8; ++m) acc += M[216 + m * 8 + q] * ge[m];
      const int a = q >> 2, bb = (q >> 1) & 1, cc = q & 1;
      const int64_t o = ((int64_t)(2 * i + a) * nf + (2 * j + bb)) * nf + 2 * k + cc;
      gxi[b * gxs + o] = (base ? base[b * bs + o] : T(0)) + acc;
    }
    // U in planes: entry n of voxel v at n * ps + v (coalesced along k)
    T* u = U + b * us + ((int64_t)i * nc + j) * nc + k;
#pragma unroll
    for (int n = 0; n < 27; ++n) {
      T acc = T(0);
#pragma unroll
      for (int m = 0; m < 8; ++m) acc += M[m * 27 + n] * ge[m];
      u[n * ps] = acc;
    }
  }
}

// Phase 1 with four consecutive coarse voxels per thread (FP32, coarse sides
// 64..512 with nc / 4 dividing the CTA): the layout and the CTA shape of
// k_icr3_refine4; same arithmetic and order per output as k_icr3_refine_t1.
template <typename T>
__global__ void __launch_bounds__(ICR3_T, 4) k_icr3_refine_t1_4(int nc, const T* __restrict__ mats, const T* gf,
                                                                int64_t gfs, T* gxi, int64_t gxs, const T* base,
                                                                int64_t bs, T* U, int64_t us, int64_t ps) {
  extern __shared__ __align__(16) unsigned char sm3_raw[];
  T* Ms = reinterpret_cast<T*>(sm3_raw);
  const int tp = nc / 4, pp = ICR3_T / tp;
  const int b = blockIdx.y;
  const int64_t pair0 = (int64_t)blockIdx.x * pp;
  for (int e = threadIdx.x; e < pp * MAT3; e += blockDim.x) Ms[e] = mats[pair0 * MAT3 + e];
  __syncthreads();
  const int pl = threadIdx.x / tp, t = threadIdx.x - pl * tp;
  const int64_t pair = pair0 + pl;
  const int i = (int)(pair / nc), j = (int)(pair - (int64_t)i * nc);
  const T* M = Ms + pl * MAT3;
  const int nf = 2 * nc, k0 = 4 * t;
  const T* g = gf + b * gfs;
  // children gradient of the four voxels: ge[ab][2 kk + cc]
  T ge[4][8];
#pragma unroll
  for (int ab = 0; ab < 4; ++ab) {
    const int64_t o = ((int64_t)(2 * i + (ab >> 1)) * nf + (2 * j + (ab & 1))) * nf + 2 * k0;
    ld4v(g + o, ge[ab]);
    ld4v(g + o + 4, ge[ab] + 4);
  }
  // gxi = L^T g (+ base), child q = 2 ab + cc
#pragma unroll
  for (int ab = 0; ab < 4; ++ab) {
    const int64_t o = ((int64_t)(2 * i + (ab >> 1)) * nf + (2 * j + (ab & 1))) * nf + 2 * k0;
    T outv[8];
    if (base) {
      ld4v(base + b * bs + o, outv);
      ld4v(base + b * bs + o + 4, outv + 4);
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) outv[e] = T(0);
    }
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
      const int q = 2 * ab + cc;
      T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int m = q; m < 8; ++m) {
        const T w = M[216 + m * 8 + q];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) acc[kk] += w * ge[m >> 1][2 * kk + (m & 1)];
      }
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) outv[2 * kk + cc] = outv[2 * kk + cc] + acc[kk];
    }
    T* go = gxi + b * gxs + o;
    st4v(go, outv);
    st4v(go + 4, outv + 4);
  }
  // U[n][v] = (R^T g)_n for v = (i, j, k0 .. k0 + 3)
  T* u = U + b * us + ((int64_t)i * nc + j) * nc + k0;
#pragma unroll
  for (int n = 0; n < 27; ++n) {
    T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const T w = M[m * 27 + n];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) acc[kk] += w * ge[m >> 1][2 * kk + (m & 1)];
    }
    st4v(u + n * ps, acc);
  }
}

// Adjoint phase 2: gc(i, j, k) = sum of U[idx][v'] over the coarse voxels v'
// whose neighbourhood holds (i, j, k) at position idx (fixed loop order).
template <typename T>
__global__ void k_icr3_refine_t2(int nc, const T* U, int64_t us, int64_t ps, T* gc, int64_t gcs) {
  const int b = blockIdx.y;
  const int64_t n3 = (int64_t)nc * nc * nc;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n3; v += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(v % nc), j = (int)((v / nc) % nc), i = (int)(v / ((int64_t)nc * nc));
    T acc = T(0);
    for (int ip = i - 2; ip <= i + 2; ++ip) {
      if (ip < 0 || ip >= nc) continue;
      const int a = i - win(nc, ip);
      if (a < 0 || a > 2) continue;
      for (int jp = j - 2; jp <= j + 2; ++jp) {
        if (jp < 0 || jp >= nc) continue;
        const int bb = j - win(nc, jp);
        if (bb < 0 || bb > 2) continue;
#pragma unroll
        for (int d = -1; d <= 1; ++d) {
          const int kp = (k - d + nc) % nc;  // k = kp + d: position d + 1 in the neighbourhood of kp
          acc += U[b * us + (int64_t)(9 * a + 3 * bb + (d + 1)) * ps + ((int64_t)ip * nc + jp) * nc + kp];
        }
      }
    }
    gc[b * gcs + v] = acc;
  }
}

template <typename T>
int ensure_ws3(nre_icr_plan* p, int B) {
  const int64_t big = (int64_t)p->sizes[p->n_levels - 1];
  const int64_t lv = big * big * big;  // largest level below the finest
  NRE_TRY(nre::ensure(p->ws_a, (size_t)B * lv * sizeof(T)));
  NRE_TRY(nre::ensure(p->ws_b, (size_t)B * lv * sizeof(T)));
  NRE_TRY(nre::ensure(p->ws_c, (size_t)B * lv * 27 * sizeof(T)));
  return NRE_OK;
}

}  // namespace

namespace nre {

int icr3_setup(nre_icr_plan* p) {
  int64_t off = 0;
  p->sizes.clear();
  p->offsets.clear();
  for (int l = 0; l <= p->n_levels; ++l) {
    const int n = p->n0 << l;
    p->sizes.push_back(n);
    p->offsets.push_back(off);
    off += (int64_t)n * n * n;
  }
  p->latent = off;
  p->stride = (off + 63) / 64 * 64;
  p->n_out = (int64_t)p->sizes.back() * p->sizes.back() * p->sizes.back();
  const int n0 = p->n0, n3 = n0 * n0 * n0;
  std::vector<double> K0((size_t)n3 * n3), L0;
  for (int a = 0; a < n3; ++a)
    for (int b = 0; b < n3; ++b)
      K0[(size_t)a * n3 + b] = k32(p, pos3(p, 0, a / (n0 * n0), (a / n0) % n0, a % n0),
                                   pos3(p, 0, b / (n0 * n0), (b / n0) % n0, b % n0));
  if (!chol_jitter(K0, n3, 1e-10 * p->var, L0))
    return set_error(NRE_EINVAL, "level-0 kernel matrix is not positive definite");
  std::vector<double> mats;
  p->mat_off.clear();
  for (int l = 0; l < p->n_levels; ++l) {
    p->mat_off.push_back((int64_t)mats.size());
    const int nc = p->sizes[l];
    for (int i = 0; i < nc; ++i)
      for (int j = 0; j < nc; ++j) {
        double buf[MAT3];
        if (!pair_matrices(p, l, i, j, buf))
          return set_error(NRE_EINVAL, "refinement matrices of level %d rows (%d, %d) are not positive definite", l,
                           i, j);
        mats.insert(mats.end(), buf, buf + MAT3);
      }
  }
  if (p->dtype == NRE_F64) {
    NRE_TRY(p->L0.upload(L0.data(), L0.size() * sizeof(double)));
    NRE_TRY(p->mats.upload(mats.data(), mats.size() * sizeof(double)));
  } else {
    std::vector<float> l0(L0.begin(), L0.end()), m(mats.begin(), mats.end());
    NRE_TRY(p->L0.upload(l0.data(), l0.size() * sizeof(float)));
    NRE_TRY(p->mats.upload(m.data(), m.size() * sizeof(float)));
  }
  return NRE_OK;
}

template <typename T>
int icr3_forward_t(nre_icr_plan* p, const T* xi, T* s, int B, const T* scale, cudaStream_t st) {
  NRE_TRY(ensure_ws3<T>(p, B));
  const int L = p->n_levels;
  const int64_t big = (int64_t)p->sizes[L - 1] * p->sizes[L - 1] * p->sizes[L - 1];
  T* bufs[2] = {p->ws_a.as<T>(), p->ws_b.as<T>()};
  const T* mats = p->mats.as<T>();
  const int n3 = p->n0 * p->n0 * p->n0;
  prof_begin("icr3_level0", (double)B * n3 * sizeof(T) * 2 + (double)n3 * n3 * sizeof(T) / 2, st);
  k_icr3_level0<T><<<dim3((n3 + 7) / 8, B), 256, 0, st>>>(p->L0.as<T>(), xi, p->stride, bufs[0], big, n3);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  for (int l = 0; l < L; ++l) {
    const int nc = p->sizes[l];
    const int64_t nf3 = (int64_t)8 * nc * nc * nc;
    const bool last = l == L - 1;
    T* out = last ? s : bufs[(l + 1) & 1];
    const int64_t os = last ? p->n_out : big;
    prof_begin("icr3_refine", (double)B * nf3 * sizeof(T) * (2.0 + 1.0 / 8) + (double)nc * nc * MAT3 * sizeof(T), st);
    bool done = false;
    if constexpr (sizeof(T) == 4) {
      // whole pairs per CTA (nc / 4 a power of two up to the CTA size) and
      // 16-byte aligned rows of every array the kernel reads as vectors
      auto al = [](const void* q) { return reinterpret_cast<uintptr_t>(q) % 16 == 0; };
      const T* xl = xi + p->offsets[l + 1];
      if (nc >= 64 && nc % 4 == 0 && nc / 4 <= ICR3_T && ICR3_T % (nc / 4) == 0 && al(xl) && al(out) &&
          al(bufs[l & 1]) && p->stride % 4 == 0 && os % 4 == 0 && big % 4 == 0 && (!last || !scale || al(scale))) {
        const int pp = ICR3_T / (nc / 4);
        k_icr3_refine4<T><<<dim3((unsigned)((int64_t)nc * nc / pp), B), ICR3_T, pp * MAT3 * sizeof(T), st>>>(
            nc, mats + p->mat_off[l], bufs[l & 1], big, xi + p->offsets[l + 1], p->stride, out, os,
            last ? scale : nullptr);
        done = true;
      }
    }
    if (!done) {
      k_icr3_refine<T><<<dim3(nc * nc, B), 128, 0, st>>>(nc, mats + p->mat_off[l], bufs[l & 1], big,
                                                          xi + p->offsets[l + 1], p->stride, out, os,
                                                          last ? scale : nullptr);
    }
    prof_end(st);
    NRE_CHECK_LAUNCH();
  }
  return NRE_OK;
}

template <typename T>
int icr3_vjp_t(nre_icr_plan* p, const T* ct, int64_t cts, T* g, const T* base, int B, cudaStream_t st) {
  NRE_TRY(ensure_ws3<T>(p, B));
  const int L = p->n_levels;
  const int64_t big = (int64_t)p->sizes[L - 1] * p->sizes[L - 1] * p->sizes[L - 1];
  T* bufs[2] = {p->ws_a.as<T>(), p->ws_b.as<T>()};
  T* U = p->ws_c.as<T>();
  const T* mats = p->mats.as<T>();
  const T* gf = ct;
  int64_t gfs = cts;
  for (int l = L - 1; l >= 0; --l) {
    const int nc = p->sizes[l];
    const int64_t n3 = (int64_t)nc * nc * nc;
    T* gc = bufs[l & 1];
    prof_begin("icr3_refine_t", (double)B * n3 * sizeof(T) * (8.0 * 3 + 27 * 2 + 1) + (double)nc * nc * MAT3 * sizeof(T),
               st);
    bool done = false;
    if constexpr (sizeof(T) == 4) {
      auto al = [](const void* q) { return reinterpret_cast<uintptr_t>(q) % 16 == 0; };
      const T* bl = base ? base + p->offsets[l + 1] : nullptr;
      T* gl = g + p->offsets[l + 1];
      if (nc >= 64 && nc % 4 == 0 && nc / 4 <= ICR3_T && ICR3_T % (nc / 4) == 0 && al(gf) && al(gl) &&
          (!bl || al(bl)) && al(U) && gfs % 4 == 0 && p->stride % 4 == 0 && big % 4 == 0) {
        const int pp = ICR3_T / (nc / 4);
        k_icr3_refine_t1_4<T><<<dim3((unsigned)((int64_t)nc * nc / pp), B), ICR3_T, pp * MAT3 * sizeof(T), st>>>(
            nc, mats + p->mat_off[l], gf, gfs, gl, p->stride, bl, p->stride, U, big * 27, big);
        done = true;
      }
    }
    if (!done)
      k_icr3_refine_t1<T><<<dim3(nc * nc, B), 128, 0, st>>>(nc, mats + p->mat_off[l], gf, gfs,
                                                             g + p->offsets[l + 1], p->stride,
                                                             base ? base + p->offsets[l + 1] : nullptr, p->stride, U,
                                                             big * 27, big);
    int blocks = (int)((n3 + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    k_icr3_refine_t2<T><<<dim3(blocks, B), 256, 0, st>>>(nc, U, big * 27, big, gc, big);
    prof_end(st);
    NRE_CHECK_LAUNCH();
    gf = gc;
    gfs = big;
  }
  const int n3 = p->n0 * p->n0 * p->n0;
  prof_begin("icr3_level0_t", (double)B * n3 * sizeof(T) * 3 + (double)n3 * n3 * sizeof(T) / 2, st);
  k_icr3_level0_t<T><<<dim3((n3 + 7) / 8, B), 256, 0, st>>>(p->L0.as<T>(), gf, gfs, g, p->stride, base, p->stride,
                                                            n3);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  return NRE_OK;
}

template int icr3_forward_t<float>(nre_icr_plan*, const float*, float*, int, const float*, cudaStream_t);
template int icr3_forward_t<double>(nre_icr_plan*, const double*, double*, int, const double*, cudaStream_t);
template int icr3_vjp_t<float>(nre_icr_plan*, const float*, int64_t, float*, const float*, int, cudaStream_t);
template int icr3_vjp_t<double>(nre_icr_plan*, const double*, int64_t, double*, const double*, int, cudaStream_t);

}  // namespace nre
