// Iterative charted refinement (ICR) on a 2-D log-radial chart.
//
// Sec. "Gaussian Processes", ICR paragraph: a GP on a deformed space, built by
// refining a coarse draw level by level from nearest-neighbour relations on
// coarsenings of the chart.  Reading implemented here (no equations in the
// paper): level l has n_l = n0 2^l points per axis at u = (i+1/2)/n_l,
// v = (j+1/2)/n_l, mapped by r = r_min (r_max/r_min)^u, phi = 2 pi v; Matern-3/2
// kernel; s_0 = chol(K0) xi_0; coarse pixel (i, j) with its 3x3 neighbourhood
// (rows clamp(i-1, 0, n-3) + {0,1,2}, columns j-1..j+1 mod n) predicts its 2x2
// children: s_f = R_i s_nbhd + L_i xi_f, R_i = K_fc K_cc^-1,
// L_i = chol(K_ff - R_i K_cf).  Rotation invariance makes R, L depend only on
// (level, radial row); they are assembled in FP64 on the host.
//
// Kernels: four coarse pixels per thread (one per thread when the level size
// is not a multiple of 4).  The forward reads the row's matrices once, the
// 3 x 6 neighbourhood window (coalesced along the angular axis) and the 2 x 8
// excitations as 16-byte vectors, and writes the children the same way.  The adjoint is a deterministic
// gather: each coarse pixel collects R^T g from the children of every coarse
// pixel whose neighbourhood contains it (up to 5 radial rows near the clamped
// edges), and writes L^T g for its own children.
#include <cmath>
#include <vector>

#include "metric_internal.cuh"

#include "icr_internal.cuh"
#include "tma.cuh"

namespace {

using nre::prof_begin;
using nre::prof_end;

constexpr int ICR_THREADS = 256;
constexpr int MAT = 52;  // 36 (R) + 16 (L)

// ---------------------------------------------------------------- host math
struct P2 {
  double x, y;
};

P2 chart_pos(const nre_icr_plan* p, int level, double i, double j) {
  const double n = p->sizes[level];
  const double u = (i + 0.5) / n, v = (j + 0.5) / n;
  const double r = p->r_min * std::pow(p->r_max / p->r_min, u);
  const double phi = 2.0 * M_PI * v;
  return {r * std::cos(phi), r * std::sin(phi)};
}

double matern32(const nre_icr_plan* p, P2 a, P2 b) {
  const double d = std::sqrt((a.x - b.x) * (a.x - b.x) + (a.y - b.y) * (a.y - b.y));
  const double t = std::sqrt(3.0) * d / p->rho;
  return p->var * (1.0 + t) * std::exp(-t);
}

// In-place lower Cholesky of the n x n row-major matrix; false if not SPD.
bool cholesky(std::vector<double>& A, int n) {
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
    if (!(s > 0.0)) return false;
    const double d = std::sqrt(s);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = t / d;
    }
    for (int k = j + 1; k < n; ++k) A[j * n + k] = 0.0;
  }
  return true;
}

bool cholesky_jitter(std::vector<double> A, int n, double jitter, std::vector<double>& L) {
  L = A;
  if (cholesky(L, n)) return true;
  for (int i = 0; i < n; ++i) A[i * n + i] += jitter;
  L = A;
  return cholesky(L, n);
}

// Solve (L L^T) X = Bm for X (n x m), L lower n x n, Bm row-major n x m.
void chol_solve(const std::vector<double>& L, int n, std::vector<double>& X, int m) {
  for (int c = 0; c < m; ++c) {
    for (int i = 0; i < n; ++i) {  // forward
      double s = X[i * m + c];
      for (int k = 0; k < i; ++k) s -= L[i * n + k] * X[k * m + c];
      X[i * m + c] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {  // backward with L^T
      double s = X[i * m + c];
      for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * X[k * m + c];
      X[i * m + c] = s / L[i * n + i];
    }
  }
}

__host__ __device__ inline int window(int n, int i) {
  int w = i - 1;
  if (w < 0) w = 0;
  if (w > n - 3) w = n - 3;
  return w;
}

// R (4x9) and L (4x4) for coarse row i of `level`, appended to out.
bool level_row_matrices(const nre_icr_plan* p, int level, int i, double* out) {
  const int nc = p->sizes[level];
  const int w = window(nc, i);
  P2 pc[9], pf[4];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) pc[3 * a + b] = chart_pos(p, level, w + a, (b - 1 + nc) % nc);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) pf[2 * a + b] = chart_pos(p, level + 1, 2 * i + a, b);
  std::vector<double> Kcc(81), X(36), Kff(16);
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) Kcc[r * 9 + c] = matern32(p, pc[r], pc[c]);
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 4; ++c) X[r * 4 + c] = matern32(p, pc[r], pf[c]);  // K_cf
  std::vector<double> Kcf = X;
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) Kff[r * 4 + c] = matern32(p, pf[r], pf[c]);
  std::vector<double> Lcc;
  if (!cholesky_jitter(Kcc, 9, 1e-10 * p->var, Lcc)) return false;
  chol_solve(Lcc, 9, X, 4);  // X = K_cc^-1 K_cf (9x4); R = X^T
  double* R = out;
  for (int k = 0; k < 4; ++k)
    for (int n = 0; n < 9; ++n) R[k * 9 + n] = X[n * 4 + k];
  std::vector<double> D(16);
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      double s = Kff[r * 4 + c];
      for (int n = 0; n < 9; ++n) s -= R[r * 9 + n] * Kcf[n * 4 + c];
      D[r * 4 + c] = s;
    }
  for (int r = 0; r < 4; ++r)  // symmetrise the rounding of the Schur complement
    for (int c = 0; c < r; ++c) D[r * 4 + c] = D[c * 4 + r] = 0.5 * (D[r * 4 + c] + D[c * 4 + r]);
  std::vector<double> LD;
  if (!cholesky_jitter(D, 4, 1e-10 * p->var, LD)) return false;
  for (int k = 0; k < 16; ++k) out[36 + k] = LD[k];
  return true;
}

// ---------------------------------------------------------------- kernels
template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// s_0 = L0 xi_0 per sample: one warp per output row (lanes along the row), all
// rows in flight at once.
template <typename T>
__global__ void k_icr_level0(const T* L0, const T* xi, int64_t xs, T* s0, int64_t ss, int n2) {
  const int b = blockIdx.y, lane = threadIdx.x & 31, nw = (blockDim.x >> 5) * gridDim.x;
  for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n2; i += nw) {
    T acc = T(0);
    for (int j = lane; j <= i; j += 32) acc += L0[i * n2 + j] * xi[b * xs + j];
    acc = warp_sum_t(acc);
    if (lane == 0) s0[b * ss + i] = acc;
  }
}

// out = base + L0^T g0 per sample: one warp per output (lanes down the column).
template <typename T>
__global__ void k_icr_level0_t(const T* L0, const T* g0, int64_t gs, T* out, int64_t os,
                               const T* base, int64_t bs, int n2) {
  const int b = blockIdx.y, lane = threadIdx.x & 31, nw = (blockDim.x >> 5) * gridDim.x;
  for (int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n2; j += nw) {
    T acc = T(0);
    for (int i = j + lane; i < n2; i += 32) acc += L0[i * n2 + j] * g0[b * gs + i];
    acc = warp_sum_t(acc);
    if (lane == 0) out[b * os + j] = acc + (base ? base[b * bs + j] : T(0));
  }
}

// s_f = R s_nbhd + L xi_f for every coarse pixel; optional pointwise weight
// `scale` [nf^2] applied to s_f (the metric's w * L v).
template <typename T>
__global__ void __launch_bounds__(ICR_THREADS) k_icr_refine(int nc, const T* __restrict__ mats,
                                                           const T* s_c, int64_t scs,
                                                           const T* xi_f, int64_t xs, T* s_f,
                                                           int64_t sfs, const T* scale) {
  typedef typename nre::CplxT<T>::type V2;
  const int b = blockIdx.y;
  const int64_t pix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pix >= (int64_t)nc * nc) return;
  const int i = (int)(pix / nc), j = (int)(pix - (int64_t)i * nc);
  const T* M = mats + (int64_t)i * MAT;
  const int w = window(nc, i);
  const int jm = j == 0 ? nc - 1 : j - 1, jp = j == nc - 1 ? 0 : j + 1;
  const T* sc = s_c + b * scs;
  T nb[9];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T* row = sc + (int64_t)(w + a) * nc;
    nb[3 * a + 0] = row[jm];
    nb[3 * a + 1] = row[j];
    nb[3 * a + 2] = row[jp];
  }
  const int nf = 2 * nc;
  const T* xf = xi_f + b * xs;
  const V2 x0 = *reinterpret_cast<const V2*>(xf + (int64_t)(2 * i) * nf + 2 * j);
  const V2 x1 = *reinterpret_cast<const V2*>(xf + (int64_t)(2 * i + 1) * nf + 2 * j);
  const T e[4] = {x0.x, x0.y, x1.x, x1.y};
  T o[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T acc = T(0);
#pragma unroll
    for (int n = 0; n < 9; ++n) acc += __ldg(&M[k * 9 + n]) * nb[n];
#pragma unroll
    for (int m = 0; m <= k; ++m) acc += __ldg(&M[36 + k * 4 + m]) * e[m];
    o[k] = acc;
  }
  const int64_t f0 = (int64_t)(2 * i) * nf + 2 * j, f1 = f0 + nf;
  if (scale) {
    o[0] *= scale[f0];
    o[1] *= scale[f0 + 1];
    o[2] *= scale[f1];
    o[3] *= scale[f1 + 1];
  }
  T* sf = s_f + b * sfs;
  V2 y0, y1;
  y0.x = o[0];
  y0.y = o[1];
  y1.x = o[2];
  y1.y = o[3];
  *reinterpret_cast<V2*>(sf + f0) = y0;
  *reinterpret_cast<V2*>(sf + f1) = y1;
}

// Adjoint of one refinement: g_c = sum R^T g_children (gather), and
// g_xi_f = base + L^T g_children for this pixel's own children.
template <typename T>
__global__ void __launch_bounds__(ICR_THREADS) k_icr_refine_t(int nc, const T* __restrict__ mats,
                                                             const T* g_f, int64_t gfs, T* g_c,
                                                             int64_t gcs, T* g_xi, int64_t gxs,
                                                             const T* base, int64_t bs) {
  typedef typename nre::CplxT<T>::type V2;
  const int b = blockIdx.y;
  const int64_t pix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pix >= (int64_t)nc * nc) return;
  const int ip = (int)(pix / nc), jp = (int)(pix - (int64_t)ip * nc);
  const int nf = 2 * nc;
  const T* gf = g_f + b * gfs;
  // own children: L^T g
  {
    const int64_t f0 = (int64_t)(2 * ip) * nf + 2 * jp, f1 = f0 + nf;
    const V2 a0 = *reinterpret_cast<const V2*>(gf + f0);
    const V2 a1 = *reinterpret_cast<const V2*>(gf + f1);
    const T g[4] = {a0.x, a0.y, a1.x, a1.y};
    const T* M = mats + (int64_t)ip * MAT + 36;
    T o[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      T acc = T(0);
#pragma unroll
      for (int k = m; k < 4; ++k) acc += __ldg(&M[k * 4 + m]) * g[k];
      o[m] = acc;
    }
    T* gx = g_xi + b * gxs;
    if (base) {
      const T* bb = base + b * bs;
      o[0] += bb[f0];
      o[1] += bb[f0 + 1];
      o[2] += bb[f1];
      o[3] += bb[f1 + 1];
    }
    V2 y0, y1;
    y0.x = o[0];
    y0.y = o[1];
    y1.x = o[2];
    y1.y = o[3];
    *reinterpret_cast<V2*>(gx + f0) = y0;
    *reinterpret_cast<V2*>(gx + f1) = y1;
  }
  // gather R^T g from the coarse pixels whose neighbourhood holds (ip, jp)
  T acc = T(0);
  const int i_lo = ip - 2 < 0 ? 0 : ip - 2, i_hi = ip + 2 > nc - 1 ? nc - 1 : ip + 2;
  for (int i = i_lo; i <= i_hi; ++i) {
    const int a = ip - window(nc, i);
    if (a < 0 || a > 2) continue;
    const T* M = mats + (int64_t)i * MAT;
#pragma unroll
    for (int bcol = 0; bcol < 3; ++bcol) {
      int j = jp - (bcol - 1);
      j = j < 0 ? j + nc : (j >= nc ? j - nc : j);
      const int64_t f0 = (int64_t)(2 * i) * nf + 2 * j;
      const V2 a0 = *reinterpret_cast<const V2*>(gf + f0);
      const V2 a1 = *reinterpret_cast<const V2*>(gf + f0 + nf);
      const int n = 3 * a + bcol;
      acc += __ldg(&M[0 * 9 + n]) * a0.x + __ldg(&M[1 * 9 + n]) * a0.y + __ldg(&M[2 * 9 + n]) * a1.x +
             __ldg(&M[3 * 9 + n]) * a1.y;
    }
  }
  g_c[b * gcs + pix] = acc;
}

// Four consecutive values at p (16-byte aligned for float, two 16-byte
// vectors for double).
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T* o) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(p), c = *reinterpret_cast<const double2*>(p + 2);
    o[0] = a.x; o[1] = a.y; o[2] = c.x; o[3] = c.y;
  }
}
template <typename T>
__device__ __forceinline__ void st4(T* p, const T* o) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(o[2], o[3]);
  }
}

// Four coarse pixels per thread (columns j0..j0+3 of radial row i; block
// (32, 4): 128 columns x 4 rows): the row's matrices, the 3 x 6 neighbourhood
// window and the 2 x 8 children are read once for the four, with 16-byte
// loads.  Needs nc % 4 == 0 and 16-byte aligned level offsets (n0 % 4 == 0).
constexpr int ICR4_X = 32, ICR4_Y = 4;

template <typename T>
__global__ void __launch_bounds__(ICR4_X * ICR4_Y) k_icr_refine4(int nc, const T* __restrict__ mats,
                                                                const T* s_c, int64_t scs, const T* xi_f,
                                                                int64_t xs, T* s_f, int64_t sfs, const T* scale) {
  const int i = blockIdx.y * ICR4_Y + threadIdx.y, b = blockIdx.z;
  const int j0 = 4 * (blockIdx.x * ICR4_X + threadIdx.x);
  if (i >= nc || j0 >= nc) return;
  const T* M = mats + (int64_t)i * MAT;
  T m[MAT];
#pragma unroll
  for (int k = 0; k < MAT; ++k) m[k] = __ldg(&M[k]);
  const int w = window(nc, i);
  const int jm = j0 == 0 ? nc - 1 : j0 - 1, jp = j0 + 4 == nc ? 0 : j0 + 4;
  const T* sc = s_c + b * scs;
  T nb[3][6];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T* row = sc + (int64_t)(w + a) * nc;
    nb[a][0] = row[jm];
    ld4(row + j0, &nb[a][1]);
    nb[a][5] = row[jp];
  }
  const int nf = 2 * nc;
  const int64_t f0 = (int64_t)(2 * i) * nf + 2 * j0;
  const T* xf = xi_f + b * xs + f0;
  T e0[8], e1[8];
  ld4(xf, e0);
  ld4(xf + 4, e0 + 4);
  ld4(xf + nf, e1);
  ld4(xf + nf + 4, e1 + 4);
  T o0[8], o1[8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const T nq[9] = {nb[0][q], nb[0][q + 1], nb[0][q + 2], nb[1][q], nb[1][q + 1],
                     nb[1][q + 2], nb[2][q], nb[2][q + 1], nb[2][q + 2]};
    const T e[4] = {e0[2 * q], e0[2 * q + 1], e1[2 * q], e1[2 * q + 1]};
    T o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      T acc = T(0);
#pragma unroll
      for (int n = 0; n < 9; ++n) acc += m[k * 9 + n] * nq[n];
#pragma unroll
      for (int mm = 0; mm <= k; ++mm) acc += m[36 + k * 4 + mm] * e[mm];
      o[k] = acc;
    }
    o0[2 * q] = o[0];
    o0[2 * q + 1] = o[1];
    o1[2 * q] = o[2];
    o1[2 * q + 1] = o[3];
  }
  if (scale) {
    T s0[8], s1[8];
    ld4(scale + f0, s0);
    ld4(scale + f0 + 4, s0 + 4);
    ld4(scale + f0 + nf, s1);
    ld4(scale + f0 + nf + 4, s1 + 4);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      o0[k] *= s0[k];
      o1[k] *= s1[k];
    }
  }
  T* sf = s_f + b * sfs + f0;
  st4(sf, o0);
  st4(sf + 4, o0 + 4);
  st4(sf + nf, o1);
  st4(sf + nf + 4, o1 + 4);
}

// Adjoint with four coarse pixels per thread (as k_icr_refine_t).
template <typename T>
__global__ void __launch_bounds__(ICR4_X * ICR4_Y) k_icr_refine4_t(int nc, const T* __restrict__ mats,
                                                                  const T* g_f, int64_t gfs, T* g_c, int64_t gcs,
                                                                  T* g_xi, int64_t gxs, const T* base, int64_t bs) {
  const int ip = blockIdx.y * ICR4_Y + threadIdx.y, b = blockIdx.z;
  const int jp0 = 4 * (blockIdx.x * ICR4_X + threadIdx.x);
  if (ip >= nc || jp0 >= nc) return;
  const int nf = 2 * nc;
  const T* gf = g_f + b * gfs;
  // own children: L^T g (+ base)
  {
    const int64_t f0 = (int64_t)(2 * ip) * nf + 2 * jp0;
    T g0[8], g1[8];
    ld4(gf + f0, g0);
    ld4(gf + f0 + 4, g0 + 4);
    ld4(gf + f0 + nf, g1);
    ld4(gf + f0 + nf + 4, g1 + 4);
    const T* ML = mats + (int64_t)ip * MAT + 36;
    T l[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) l[k] = __ldg(&ML[k]);
    T o0[8], o1[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T g[4] = {g0[2 * q], g0[2 * q + 1], g1[2 * q], g1[2 * q + 1]};
      T o[4];
#pragma unroll
      for (int mm = 0; mm < 4; ++mm) {
        T acc = T(0);
#pragma unroll
        for (int k = mm; k < 4; ++k) acc += l[k * 4 + mm] * g[k];
        o[mm] = acc;
      }
      o0[2 * q] = o[0];
      o0[2 * q + 1] = o[1];
      o1[2 * q] = o[2];
      o1[2 * q + 1] = o[3];
    }
    if (base) {
      const T* bb = base + b * bs + f0;
      T b0[8], b1[8];
      ld4(bb, b0);
      ld4(bb + 4, b0 + 4);
      ld4(bb + nf, b1);
      ld4(bb + nf + 4, b1 + 4);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        o0[k] += b0[k];
        o1[k] += b1[k];
      }
    }
    T* gx = g_xi + b * gxs + f0;
    st4(gx, o0);
    st4(gx + 4, o0 + 4);
    st4(gx + nf, o1);
    st4(gx + nf + 4, o1 + 4);
  }
  // gather R^T g over the coarse pixels whose neighbourhood holds (ip, jp0 + q):
  // coarse columns jp0 - 1 .. jp0 + 4, i.e. fine columns 2 jp0 - 2 .. 2 jp0 + 9
  T acc[4] = {T(0), T(0), T(0), T(0)};
  const int jm = jp0 == 0 ? nc - 1 : jp0 - 1, jpp = jp0 + 4 == nc ? 0 : jp0 + 4;
  const int i_lo = ip - 2 < 0 ? 0 : ip - 2, i_hi = ip + 2 > nc - 1 ? nc - 1 : ip + 2;
  for (int i = i_lo; i <= i_hi; ++i) {
    const int a = ip - window(nc, i);
    if (a < 0 || a > 2) continue;
    const T* MR = mats + (int64_t)i * MAT;
    T G[2][12];  // fine rows 2i, 2i+1; entry 2 (jj + 1) + c for coarse column jp0 + jj, child column c
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const T* row = gf + (int64_t)(2 * i + r) * nf;
      G[r][0] = row[2 * jm];
      G[r][1] = row[2 * jm + 1];
      ld4(row + 2 * jp0, &G[r][2]);
      ld4(row + 2 * jp0 + 4, &G[r][6]);
      G[r][10] = row[2 * jpp];
      G[r][11] = row[2 * jpp + 1];
    }
#pragma unroll
    for (int bcol = 0; bcol < 3; ++bcol) {
      const int n = 3 * a + bcol;
      const T r0 = __ldg(&MR[0 * 9 + n]), r1 = __ldg(&MR[1 * 9 + n]), r2 = __ldg(&MR[2 * 9 + n]),
              r3 = __ldg(&MR[3 * 9 + n]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int t0 = 2 * (q - bcol + 2);  // coarse column jp0 + q - (bcol - 1)
        acc[q] += r0 * G[0][t0] + r1 * G[0][t0 + 1] + r2 * G[1][t0] + r3 * G[1][t0 + 1];
      }
    }
  }
  st4(g_c + b * gcs + (int64_t)ip * nc + jp0, acc);
}

// Adjoint with four coarse pixels per thread, its fine rows staged by bulk
// tensor copies.  A CTA covers coarse rows ip0 .. ip0 + 3 and coarse columns
// jc0 .. jc0 + 127; the gathers of its threads read fine rows 2 ip0 - 4 ..
// 2 ip0 + 11 (the children of coarse rows ip0 - 2 .. ip0 + 5) at fine columns
// 2 jc0 - 2 .. 2 jc0 + 257.  One elected thread loads them as three boxes of
// the 16 rows: the main box of BW = min(256, 2 nc) columns at x = 2 jc0 and
// four columns on either side, wrapped around the angular axis (x rounded to
// 16 bytes; the needed pair is the upper half of the left box and the lower
// half of the right one).  Rows outside the chart read as zero and are never
// used (the gather skips coarse rows outside 0 .. nc - 1).  Same arithmetic
// and order as k_icr_refine4_t.
constexpr int TRows = 16, TMainMax = 256;

template <typename T>
__global__ void __launch_bounds__(ICR4_X * ICR4_Y) k_icr_refine4_t_tma(int nc, const T* __restrict__ mats,
                                                                      const __grid_constant__ CUtensorMap tm_main,
                                                                      const __grid_constant__ CUtensorMap tm_halo,
                                                                      T* g_c, int64_t gcs, T* g_xi, int64_t gxs,
                                                                      const T* base, int64_t bs, unsigned* status) {
  __shared__ __align__(128) T gm[TRows * TMainMax];
  __shared__ __align__(128) T hl[TRows * 4];
  __shared__ __align__(128) T hr[TRows * 4];
  __shared__ __align__(8) uint64_t bar;
  const int nf = 2 * nc, BW = nf < TMainMax ? nf : TMainMax;
  const int tid = threadIdx.y * ICR4_X + threadIdx.x, b = blockIdx.z;
  const int ip0 = blockIdx.y * ICR4_Y, jc0 = blockIdx.x * (4 * ICR4_X);
  const int y0 = 2 * ip0 - 4;
  if (tid == 0) {
    nre::mbar_init(&bar, 1);
    nre::mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0) {
    nre::mbar_arrive_tx(&bar, (unsigned)((BW + 8) * TRows * sizeof(T)));
    nre::tma_load_3d(gm, &tm_main, 2 * jc0, y0, b, &bar);
    nre::tma_load_3d(hl, &tm_halo, jc0 == 0 ? nf - 4 : 2 * jc0 - 4, y0, b, &bar);
    nre::tma_load_3d(hr, &tm_halo, jc0 + 4 * ICR4_X >= nc ? 0 : 2 * jc0 + 8 * ICR4_X, y0, b, &bar);
  }
  const int ip = ip0 + threadIdx.y, jp0 = jc0 + 4 * threadIdx.x;
  const bool act = ip < nc && jp0 < nc;
  const int64_t f0 = (int64_t)(2 * ip) * nf + 2 * jp0;
  // base values while the copies land
  T b0[8], b1[8];
  if (act && base) {
    const T* bb = base + b * bs + f0;
    ld4(bb, b0);
    ld4(bb + 4, b0 + 4);
    ld4(bb + nf, b1);
    ld4(bb + nf + 4, b1 + 4);
  }
  if (!nre::mbar_wait(&bar, 0)) {
    // give up on this tile; wait (bounded) for the copies in flight before the
    // shared memory is released
    if (tid == 0) nre::note_timeout(status);
    nre::mbar_wait(&bar, 0);
    return;
  }
  if (!act) return;
  const int lx = 8 * threadIdx.x;  // local fine column of 2 jp0
  // own children: L^T g (+ base)
  {
    const T* r0 = gm + (2 * threadIdx.y + 4) * BW + lx;
    T g0[8], g1[8];
    ld4(r0, g0);
    ld4(r0 + 4, g0 + 4);
    ld4(r0 + BW, g1);
    ld4(r0 + BW + 4, g1 + 4);
    const T* ML = mats + (int64_t)ip * MAT + 36;
    T l[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) l[k] = __ldg(&ML[k]);
    T o0[8], o1[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T g[4] = {g0[2 * q], g0[2 * q + 1], g1[2 * q], g1[2 * q + 1]};
      T o[4];
#pragma unroll
      for (int mm = 0; mm < 4; ++mm) {
        T acc = T(0);
#pragma unroll
        for (int k = mm; k < 4; ++k) acc += l[k * 4 + mm] * g[k];
        o[mm] = acc;
      }
      o0[2 * q] = o[0];
      o0[2 * q + 1] = o[1];
      o1[2 * q] = o[2];
      o1[2 * q + 1] = o[3];
    }
    if (base) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        o0[k] += b0[k];
        o1[k] += b1[k];
      }
    }
    T* gx = g_xi + b * gxs + f0;
    st4(gx, o0);
    st4(gx + 4, o0 + 4);
    st4(gx + nf, o1);
    st4(gx + nf + 4, o1 + 4);
  }
  // gather R^T g over the coarse pixels whose neighbourhood holds (ip, jp0 + q)
  T acc[4] = {T(0), T(0), T(0), T(0)};
  // the right neighbour column wraps to 0 at the chart's end, which need not
  // be the end of the main box (nc not a multiple of 128)
  const bool left_halo = threadIdx.x == 0, right_halo = lx + 8 >= BW || jp0 + 4 >= nc;
  const int i_lo = ip - 2 < 0 ? 0 : ip - 2, i_hi = ip + 2 > nc - 1 ? nc - 1 : ip + 2;
  for (int i = i_lo; i <= i_hi; ++i) {
    const int a = ip - window(nc, i);
    if (a < 0 || a > 2) continue;
    const T* MR = mats + (int64_t)i * MAT;
    T G[2][12];  // fine rows 2i, 2i+1; entry 2 (jj + 1) + c for coarse column jp0 + jj, child column c
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int lr = 2 * i + r - y0;
      const T* row = gm + lr * BW;
      G[r][0] = left_halo ? hl[lr * 4 + 2] : row[lx - 2];
      G[r][1] = left_halo ? hl[lr * 4 + 3] : row[lx - 1];
      ld4(row + lx, &G[r][2]);
      ld4(row + lx + 4, &G[r][6]);
      G[r][10] = right_halo ? hr[lr * 4] : row[lx + 8];
      G[r][11] = right_halo ? hr[lr * 4 + 1] : row[lx + 9];
    }
#pragma unroll
    for (int bcol = 0; bcol < 3; ++bcol) {
      const int n = 3 * a + bcol;
      const T r0 = __ldg(&MR[0 * 9 + n]), r1 = __ldg(&MR[1 * 9 + n]), r2 = __ldg(&MR[2 * 9 + n]),
              r3 = __ldg(&MR[3 * 9 + n]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int t0 = 2 * (q - bcol + 2);
        acc[q] += r0 * G[0][t0] + r1 * G[0][t0 + 1] + r2 * G[1][t0] + r3 * G[1][t0 + 1];
      }
    }
  }
  st4(g_c + b * gcs + (int64_t)ip * nc + jp0, acc);
}

// The coarse end of a chart, level 0 and the refinements whose coarse side is
// at most kSmallN, in one CTA per sample with the levels in shared memory:
// as separate launches they were a chain of short latency-bound kernels.
constexpr int kSmallN = 32;
constexpr int SMALL_THREADS = 1024;
struct IcrSmall {
  int n0, nlev;            // fused refinements: levels 0 .. nlev - 1
  int nc[10];              // coarse side of level l
  int64_t mat_off[10];     // its matrices in mats
  int64_t xi_off[10];      // its fine excitations in the latent vector
};

// Shared memory of the fused forward (two level buffers, one level's fine
// excitations and one level's matrices) and adjoint (the finest fused fine
// level, one coarse level and one level's matrices), in elements.
inline int64_t small_smem(const IcrSmall& sp, bool adjoint) {
  const int64_t n = sp.nc[sp.nlev - 1];
  return (adjoint ? 5 : 6) * n * n + n * MAT;
}

// Forward: s_0 = L_K0 xi_0, then s_f = R s_nbhd + L xi_f level by level; the
// last fused level goes to out (times `scale` when given).
template <typename T>
__global__ void __launch_bounds__(SMALL_THREADS) k_icr_small(IcrSmall sp, const T* __restrict__ L0,
                                                            const T* __restrict__ mats, const T* xi, int64_t xs,
                                                            T* out, int64_t os, const T* scale) {
  extern __shared__ __align__(16) unsigned char small_raw[];
  const int ncl = sp.nc[sp.nlev - 1];
  T* cur = reinterpret_cast<T*>(small_raw);
  T* nxt = cur + ncl * ncl;
  T* sxi = nxt + ncl * ncl;      // [4 ncl^2]: this level's fine excitations
  T* smat = sxi + 4 * ncl * ncl;
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
  const T* x = xi + b * xs;
  const int n2 = sp.n0 * sp.n0;
  for (int i = tid >> 5; i < n2; i += SMALL_THREADS / 32) {
    T acc = T(0);
    for (int j = lane; j <= i; j += 32) acc += L0[i * n2 + j] * x[j];
    acc = warp_sum_t(acc);
    if (lane == 0) cur[i] = acc;
  }
  for (int l = 0; l < sp.nlev; ++l) {
    const int nc = sp.nc[l], nf = 2 * nc;
    for (int k = tid; k < nc * MAT; k += SMALL_THREADS) smat[k] = mats[sp.mat_off[l] + k];
    for (int k = tid; k < nf * nf; k += SMALL_THREADS) sxi[k] = x[sp.xi_off[l] + k];
    __syncthreads();  // this level's input, excitations and matrices are in place
    const bool last = l == sp.nlev - 1;
    T* dst = last ? out + b * os : nxt;
    const T* xf = sxi;
    for (int pix = tid; pix < nc * nc; pix += SMALL_THREADS) {
      const int i = pix / nc, j = pix - i * nc;
      const T* m = smat + i * MAT;
      const int w = window(nc, i);
      const int jm = j == 0 ? nc - 1 : j - 1, jp = j == nc - 1 ? 0 : j + 1;
      T nq[9];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const T* row = cur + (w + a) * nc;
        nq[3 * a] = row[jm];
        nq[3 * a + 1] = row[j];
        nq[3 * a + 2] = row[jp];
      }
      const int64_t f0 = (int64_t)(2 * i) * nf + 2 * j, f1 = f0 + nf;
      const T e[4] = {xf[f0], xf[f0 + 1], xf[f1], xf[f1 + 1]};
      T o[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        T acc = T(0);
#pragma unroll
        for (int n = 0; n < 9; ++n) acc += m[k * 9 + n] * nq[n];
#pragma unroll
        for (int mm = 0; mm <= k; ++mm) acc += m[36 + k * 4 + mm] * e[mm];
        o[k] = acc;
      }
      if (last && scale) {
        o[0] *= scale[f0];
        o[1] *= scale[f0 + 1];
        o[2] *= scale[f1];
        o[3] *= scale[f1 + 1];
      }
      dst[f0] = o[0];
      dst[f0 + 1] = o[1];
      dst[f1] = o[2];
      dst[f1 + 1] = o[3];
    }
    __syncthreads();  // the next level reads nxt; cur and the matrices are rewritten
    T* t = cur;
    cur = nxt;
    nxt = t;
  }
}

// Adjoint of the fused levels: from g at the finest fused level (gin), per
// level g_xi_f = base + L^T g_children and the gather g_c = sum R^T g_children,
// then level 0: g_0 = base + L_K0^T g.
template <typename T>
__global__ void __launch_bounds__(SMALL_THREADS) k_icr_small_t(IcrSmall sp, const T* __restrict__ L0,
                                                              const T* __restrict__ mats, const T* gin,
                                                              int64_t gis, T* g, int64_t gs, const T* base,
                                                              int64_t bs) {
  extern __shared__ __align__(16) unsigned char small_raw[];
  const int ncl = sp.nc[sp.nlev - 1], nfl = 2 * ncl;
  T* fine = reinterpret_cast<T*>(small_raw);  // [nfl^2], later a coarse level
  T* coarse = fine + nfl * nfl;                 // [ncl^2], later a fine level
  T* smat = coarse + ncl * ncl;
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
  for (int k = tid; k < nfl * nfl; k += SMALL_THREADS) fine[k] = gin[b * gis + k];
  for (int l = sp.nlev - 1; l >= 0; --l) {
    const int nc = sp.nc[l], nf = 2 * nc;
    for (int k = tid; k < nc * MAT; k += SMALL_THREADS) smat[k] = mats[sp.mat_off[l] + k];
    __syncthreads();  // this level's g and matrices are in place
    T* gx = g + b * gs + sp.xi_off[l];
    const T* bb = base ? base + b * bs + sp.xi_off[l] : nullptr;
    for (int pix = tid; pix < nc * nc; pix += SMALL_THREADS) {
      const int ip = pix / nc, jp = pix - ip * nc;
      {
        const int64_t f0 = (int64_t)(2 * ip) * nf + 2 * jp, f1 = f0 + nf;
        const T gc[4] = {fine[f0], fine[f0 + 1], fine[f1], fine[f1 + 1]};
        const T* M = smat + ip * MAT + 36;
        T o[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          T acc = T(0);
#pragma unroll
          for (int k = m; k < 4; ++k) acc += M[k * 4 + m] * gc[k];
          o[m] = acc;
        }
        if (bb) {
          o[0] += bb[f0];
          o[1] += bb[f0 + 1];
          o[2] += bb[f1];
          o[3] += bb[f1 + 1];
        }
        gx[f0] = o[0];
        gx[f0 + 1] = o[1];
        gx[f1] = o[2];
        gx[f1 + 1] = o[3];
      }
      T acc = T(0);
      const int i_lo = ip - 2 < 0 ? 0 : ip - 2, i_hi = ip + 2 > nc - 1 ? nc - 1 : ip + 2;
      for (int i = i_lo; i <= i_hi; ++i) {
        const int a = ip - window(nc, i);
        if (a < 0 || a > 2) continue;
        const T* M = smat + i * MAT;
#pragma unroll
        for (int bcol = 0; bcol < 3; ++bcol) {
          int j = jp - (bcol - 1);
          j = j < 0 ? j + nc : (j >= nc ? j - nc : j);
          const int f0 = 2 * i * nf + 2 * j;
          const int n = 3 * a + bcol;
          acc += M[0 * 9 + n] * fine[f0] + M[1 * 9 + n] * fine[f0 + 1] + M[2 * 9 + n] * fine[f0 + nf] +
                 M[3 * 9 + n] * fine[f0 + nf + 1];
        }
      }
      coarse[pix] = acc;
    }
    __syncthreads();  // the next level reads coarse as its fine level
    T* t = fine;
    fine = coarse;
    coarse = t;
  }
  const int n2 = sp.n0 * sp.n0;
  for (int j = tid >> 5; j < n2; j += SMALL_THREADS / 32) {
    T acc = T(0);
    for (int i = j + lane; i < n2; i += 32) acc += L0[i * n2 + j] * fine[i];
    acc = warp_sum_t(acc);
    if (lane == 0) g[b * gs + j] = acc + (base ? base[b * bs + j] : T(0));
  }
}

// The fused coarse levels of the plan: refinements 0 .. K - 1 with coarse side
// at most kSmallN (K = 0: none).
IcrSmall small_plan(const nre_icr_plan* p) {
  IcrSmall sp{};
  sp.n0 = p->n0;
  int K = 0;
  while (K < p->n_levels && p->sizes[K] <= kSmallN) {
    sp.nc[K] = p->sizes[K];
    sp.mat_off[K] = p->mat_off[K];
    sp.xi_off[K] = p->offsets[K + 1];
    ++K;
  }
  sp.nlev = K;
  return sp;
}

template <typename T>
__global__ void k_scale_sqrt(const T* w, const T* x, int64_t xs, T* y, int64_t ys, int64_t n) {
  const int b = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[b * ys + i] = sqrt(w[i]) * x[b * xs + i];
}

template <typename T>
__global__ void k_fill_inv_var(T* w, const T* mask, T inv, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    w[i] = mask ? inv * mask[i] : inv;
}

dim3 pix_grid(int64_t npix, int B) { return dim3((unsigned)((npix + ICR_THREADS - 1) / ICR_THREADS), B); }

template <typename T>
int ensure_ws(nre_icr_plan* p, int B) {
  const int64_t big = (int64_t)p->sizes[p->n_levels - 1] * p->sizes[p->n_levels - 1];
  NRE_TRY(nre::ensure(p->ws_a, (size_t)B * big * sizeof(T)));
  NRE_TRY(nre::ensure(p->ws_b, (size_t)B * big * sizeof(T)));
  return NRE_OK;
}

// Runs f(b0, Bh, stream) over the batch: as two halves on two streams when
// B >= 2 and the plan has its second stream (the small levels of one half
// are latency-bound chains of short launches; the other half's launches fill
// the SMs meanwhile), else once.  Launch tracing serialises (one call).
template <class F>
int icr_split(nre_icr_plan* p, int B, cudaStream_t st, F f) {
  if (B < 2 || nre::prof_tracing()) return f(0, B, st);
  if (!p->side) {
    // created on first use outside a stream capture (never inside one)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    NRE_TRY_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return f(0, B, st);
    NRE_TRY_CUDA(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking));
    NRE_TRY_CUDA(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
    NRE_TRY_CUDA(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
  }
  NRE_TRY_CUDA(cudaEventRecord(p->ev_fork, st));
  NRE_TRY_CUDA(cudaStreamWaitEvent(p->side, p->ev_fork, 0));
  const int B0 = (B + 1) / 2;
  NRE_TRY(f(0, B0, st));
  NRE_TRY(f(B0, B - B0, p->side));
  NRE_TRY_CUDA(cudaEventRecord(p->ev_join, p->side));
  NRE_TRY_CUDA(cudaStreamWaitEvent(st, p->ev_join, 0));
  return NRE_OK;
}

// s = ICR(xi) (optionally times `scale`) for samples b0 .. b0 + B - 1 of the
// batch (level buffers at their own samples' offsets).
template <typename T>
int icr_forward_range(nre_icr_plan* p, const T* xi, T* s, int b0, int B, const T* scale, cudaStream_t st) {
  const int64_t big = (int64_t)p->sizes[p->n_levels - 1] * p->sizes[p->n_levels - 1];
  T* bufs[2] = {p->ws_a.as<T>() + b0 * big, p->ws_b.as<T>() + b0 * big};
  xi += b0 * p->stride;
  s += b0 * p->n_out;
  const int n0 = p->n0, n2 = n0 * n0;
  const T* L0 = p->L0.as<T>();
  const T* mats = p->mats.as<T>();
  const IcrSmall sp = small_plan(p);
  if (sp.nlev > 0) {
    // level 0 and the coarse refinements in one CTA per sample
    const bool all = sp.nlev == p->n_levels;
    const int ncl = sp.nc[sp.nlev - 1];
    const size_t smem = (size_t)small_smem(sp, false) * sizeof(T);
    NRE_TRY(nre::raise_smem(k_icr_small<T>, smem));
    double xib = 0.0;
    for (int l = 0; l < sp.nlev; ++l) xib += 4.0 * sp.nc[l] * sp.nc[l];
    prof_begin("icr_small", (double)B * sizeof(T) * (n2 + xib + 4.0 * ncl * ncl * (all && scale ? 2 : 1)), st);
    k_icr_small<T><<<B, SMALL_THREADS, smem, st>>>(sp, L0, mats, xi, p->stride, all ? s : bufs[sp.nlev & 1],
                                                   all ? p->n_out : big, all ? scale : nullptr);
    prof_end(st);
    NRE_CHECK_LAUNCH();
  } else {
    prof_begin("icr_level0", (double)B * 2 * n2 * sizeof(T), st);
    k_icr_level0<T><<<dim3((n2 + 7) / 8, B), 256, 0, st>>>(L0, xi, p->stride, bufs[0], big, n2);
    prof_end(st);
    NRE_CHECK_LAUNCH();
  }
  for (int l = sp.nlev; l < p->n_levels; ++l) {
    const int nc = p->sizes[l];
    const bool last = l == p->n_levels - 1;
    T* out = last ? s : bufs[(l + 1) & 1];
    const int64_t os = last ? p->n_out : big;
    prof_begin("icr_refine", (double)nc * nc * sizeof(T) * (9.0 * B + (last && scale ? 4.0 : 0.0)), st);
    if (nc % 4 == 0 && p->n0 % 4 == 0)
      k_icr_refine4<T><<<dim3((nc / 4 + ICR4_X - 1) / ICR4_X, (nc + ICR4_Y - 1) / ICR4_Y, B),
                         dim3(ICR4_X, ICR4_Y), 0, st>>>(nc, mats + p->mat_off[l], bufs[l & 1], big,
                                                        xi + p->offsets[l + 1], p->stride, out, os,
                                                        last ? scale : nullptr);
    else
      k_icr_refine<T><<<pix_grid((int64_t)nc * nc, B), ICR_THREADS, 0, st>>>(
          nc, mats + p->mat_off[l], bufs[l & 1], big, xi + p->offsets[l + 1], p->stride, out, os,
          last ? scale : nullptr);
    prof_end(st);
    NRE_CHECK_LAUNCH();
  }
  return NRE_OK;
}

// s = ICR(xi) (optionally times `scale`), batch B.
template <typename T>
int icr_forward_t(nre_icr_plan* p, const T* xi, T* s, int B, const T* scale, cudaStream_t st) {
  if (p->ndim == 3) return nre::icr3_forward_t<T>(p, xi, s, B, scale, st);
  NRE_TRY(ensure_ws<T>(p, B));
  return icr_split(p, B, st, [&](int b0, int Bh, cudaStream_t sh) {
    return icr_forward_range<T>(p, xi, s, b0, Bh, scale, sh);
  });
}

// g = base + ICR^T ct for samples b0 .. b0 + B - 1 (ct: [batch][cts]).
template <typename T>
int icr_vjp_range(nre_icr_plan* p, const T* ct, int64_t cts, T* g, const T* base, int b0, int B,
                  cudaStream_t st) {
  const int64_t big = (int64_t)p->sizes[p->n_levels - 1] * p->sizes[p->n_levels - 1];
  T* bufs[2] = {p->ws_a.as<T>() + b0 * big, p->ws_b.as<T>() + b0 * big};
  ct += b0 * cts;
  g += b0 * p->stride;
  if (base) base += b0 * p->stride;
  const T* mats = p->mats.as<T>();
  const T* gin = ct;
  int64_t gis = cts;
  int which = 0;
  const IcrSmall sp = small_plan(p);
  for (int l = p->n_levels - 1; l >= sp.nlev; --l) {
    const int nc = p->sizes[l];
    T* gc = bufs[which];
    prof_begin("icr_refine_t", (double)nc * nc * sizeof(T) * B * (base ? 13.0 : 9.0), st);
    const dim3 g4((nc / 4 + ICR4_X - 1) / ICR4_X, (nc + ICR4_Y - 1) / ICR4_Y, B);
    const bool tma_ok = p->use_tma && reinterpret_cast<uintptr_t>(gin) % 16 == 0 &&
                        ((uint64_t)gis * sizeof(T)) % 16 == 0;
    if (nc % 4 == 0 && p->n0 % 4 == 0 && tma_ok) {
      // the fine gradient [B][nf][nf] (batch stride gis) as a 3-D tensor
      const int nf = 2 * nc;
      const uint64_t dims[3] = {(uint64_t)nf, (uint64_t)nf, (uint64_t)B};
      const uint64_t strides[2] = {(uint64_t)nf * sizeof(T), (uint64_t)gis * sizeof(T)};
      const uint32_t box_m[3] = {(uint32_t)(nf < TMainMax ? nf : TMainMax), (uint32_t)TRows, 1u};
      const uint32_t box_h[3] = {4u, (uint32_t)TRows, 1u};
      const CUtensorMapDataType dt = sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
      CUtensorMap tm, th;
      NRE_TRY(nre::tmap_tiled(&tm, dt, 3, gin, dims, strides, box_m));
      NRE_TRY(nre::tmap_tiled(&th, dt, 3, gin, dims, strides, box_h));
      k_icr_refine4_t_tma<T><<<g4, dim3(ICR4_X, ICR4_Y), 0, st>>>(
          nc, mats + p->mat_off[l], tm, th, gc, big, g + p->offsets[l + 1], p->stride,
          base ? base + p->offsets[l + 1] : nullptr, p->stride, p->status);
    } else if (nc % 4 == 0 && p->n0 % 4 == 0)
      k_icr_refine4_t<T><<<g4, dim3(ICR4_X, ICR4_Y), 0, st>>>(nc, mats + p->mat_off[l], gin, gis, gc, big,
                                                             g + p->offsets[l + 1], p->stride,
                                                             base ? base + p->offsets[l + 1] : nullptr, p->stride);
    else
      k_icr_refine_t<T><<<pix_grid((int64_t)nc * nc, B), ICR_THREADS, 0, st>>>(
          nc, mats + p->mat_off[l], gin, gis, gc, big, g + p->offsets[l + 1], p->stride,
          base ? base + p->offsets[l + 1] : nullptr, p->stride);
    prof_end(st);
    NRE_CHECK_LAUNCH();
    gin = gc;
    gis = big;
    which ^= 1;
  }
  const int n2 = p->n0 * p->n0;
  if (sp.nlev > 0) {
    // the coarse refinements and level 0 in one CTA per sample
    const int ncl = sp.nc[sp.nlev - 1];
    const size_t smem = (size_t)small_smem(sp, true) * sizeof(T);
    NRE_TRY(nre::raise_smem(k_icr_small_t<T>, smem));
    double xib = 0.0;
    for (int l = 0; l < sp.nlev; ++l) xib += 4.0 * sp.nc[l] * sp.nc[l];
    prof_begin("icr_small_t", (double)B * sizeof(T) * (4.0 * ncl * ncl + (xib + n2) * (base ? 2 : 1)), st);
    k_icr_small_t<T><<<B, SMALL_THREADS, smem, st>>>(sp, p->L0.as<T>(), mats, gin, gis, g, p->stride, base,
                                                     p->stride);
    prof_end(st);
    NRE_CHECK_LAUNCH();
    return NRE_OK;
  }
  prof_begin("icr_level0_t", (double)B * (base ? 3 : 2) * n2 * sizeof(T), st);
  k_icr_level0_t<T><<<dim3((n2 + 7) / 8, B), 256, 0, st>>>(p->L0.as<T>(), gin, gis, g, p->stride, base, p->stride, n2);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  return NRE_OK;
}

// g = base + ICR^T ct, batch B (ct: [B][cts]).
template <typename T>
int icr_vjp_t(nre_icr_plan* p, const T* ct, int64_t cts, T* g, const T* base, int B, cudaStream_t st) {
  if (p->ndim == 3) return nre::icr3_vjp_t<T>(p, ct, cts, g, base, B, st);
  NRE_TRY(ensure_ws<T>(p, B));
  return icr_split(p, B, st, [&](int b0, int Bh, cudaStream_t sh) {
    return icr_vjp_range<T>(p, ct, cts, g, base, b0, Bh, sh);
  });
}

template <typename T>
int upload_tables(nre_icr_plan* p, const std::vector<double>& L0, const std::vector<double>& mats) {
  std::vector<T> a(L0.begin(), L0.end()), m(mats.begin(), mats.end());
  NRE_TRY(p->L0.upload(a.data(), a.size() * sizeof(T)));
  NRE_TRY(p->mats.upload(m.data(), m.size() * sizeof(T)));
  return NRE_OK;
}

}  // namespace

namespace nre {

int icr_layout(const nre_icr_plan* p, int64_t* n_out, int64_t* latent, int64_t* stride, int* dtype) {
  *n_out = p->n_out;
  *latent = p->latent;
  *stride = p->stride;
  *dtype = p->dtype;
  return NRE_OK;
}

int icr_metric_setup(nre_metric* m, cudaStream_t st) {
  const size_t es = m->dtype == NRE_F64 ? 8 : 4;
  NRE_TRY(m->w.alloc(m->n_data * es));
  NRE_TRY(m->tmp0.alloc((size_t)m->max_batch * m->n_data * es));
  const double inv = 1.0 / (m->lik.sig_or_scale * m->lik.sig_or_scale);
  if (m->dtype == NRE_F64) {
    if (!m->lik.mask.empty()) NRE_TRY(m->mask.upload(m->lik.mask.data(), m->lik.mask.size() * 8));
    prof_begin("icr_fill", 0.0, st);
    k_fill_inv_var<double><<<64, 256, 0, st>>>(m->w.as<double>(), m->mask.p ? m->mask.as<double>() : nullptr, inv, m->n_data);
    prof_end(st);
  } else {
    if (!m->lik.mask.empty()) {
      std::vector<float> mk(m->lik.mask.begin(), m->lik.mask.end());
      NRE_TRY(m->mask.upload(mk.data(), mk.size() * 4));
    }
    prof_begin("icr_fill", 0.0, st);
    k_fill_inv_var<float><<<64, 256, 0, st>>>(m->w.as<float>(), m->mask.p ? m->mask.as<float>() : nullptr, (float)inv, m->n_data);
  }
  prof_end(st);
  NRE_CHECK_LAUNCH();
  return NRE_OK;
}

template <typename T>
static int icr_metric_apply_t(nre_metric* m, const T* v, T* out, int B, cudaStream_t st) {
  T* s = m->tmp0.as<T>();
  NRE_TRY(icr_forward_t<T>(m->icr, v, s, B, m->w.as<T>(), st));
  return icr_vjp_t<T>(m->icr, s, m->n_data, out, v, B, st);
}

int icr_metric_apply(nre_metric* m, const void* v, void* out, int B, cudaStream_t st) {
  if (m->dtype == NRE_F64) return icr_metric_apply_t<double>(m, (const double*)v, (double*)out, B, st);
  return icr_metric_apply_t<float>(m, (const float*)v, (float*)out, B, st);
}

template <typename T>
static int icr_rhs_t(nre_metric* m, const T* xi_prime, const T* eta, T* b, int B, cudaStream_t st) {
  T* t = m->tmp0.as<T>();
  prof_begin("icr_scale", (double)m->n_data * sizeof(T) * (2.0 * B + 1.0), st);
  k_scale_sqrt<T><<<dim3(64, B), 256, 0, st>>>(m->w.as<T>(), eta, m->n_data, t, m->n_data, m->n_data);
  prof_end(st);
  NRE_CHECK_LAUNCH();
  return icr_vjp_t<T>(m->icr, t, m->n_data, b, xi_prime, B, st);
}

int icr_mgvi_rhs(nre_metric* m, const void* xi_prime, const void* eta, void* b, int B, cudaStream_t st) {
  if (m->dtype == NRE_F64)
    return icr_rhs_t<double>(m, (const double*)xi_prime, (const double*)eta, (double*)b, B, st);
  return icr_rhs_t<float>(m, (const float*)xi_prime, (const float*)eta, (float*)b, B, st);
}

}  // namespace nre

using namespace nre;

extern "C" {

int icr_create(nre_icr_plan** plan, const icr_chart_params* chart, const icr_kernel_params* kernel,
               int n_levels, int dtype) {
  clear_error();
  if (!plan || !chart || !kernel) return set_error(NRE_EINVAL, "NULL argument");
  *plan = nullptr;
  if (chart->ndim != 0 && chart->ndim != 2 && chart->ndim != 3) return set_error(NRE_EINVAL, "ndim must be 2 or 3");
  if (chart->ndim == 3) {
    if (chart->n0 < 3 || chart->n0 > 8) return set_error(NRE_EINVAL, "3-D charts need n0 in [3, 8]");
    if (n_levels < 1 || n_levels > 8) return set_error(NRE_EINVAL, "n_levels must be in [1, 8]");
    if ((int64_t)chart->n0 << n_levels > 512) return set_error(NRE_EINVAL, "3-D charts need n0 * 2^n_levels <= 512");
    if (!(chart->r_min > 0 && chart->r_max > chart->r_min)) return set_error(NRE_EINVAL, "need 0 < r_min < r_max");
    if (!(kernel->rho > 0 && kernel->var > 0)) return set_error(NRE_EINVAL, "need rho > 0 and var > 0");
    if (dtype != NRE_F32 && dtype != NRE_F64) return set_error(NRE_EINVAL, "dtype must be NRE_F32 or NRE_F64");
    nre_icr_plan* p = new nre_icr_plan();
    p->ndim = 3;
    p->dtype = dtype;
    p->n0 = chart->n0;
    p->n_levels = n_levels;
    p->r_min = chart->r_min;
    p->r_max = chart->r_max;
    p->rho = kernel->rho;
    p->var = kernel->var;
    const int s3 = nre::icr3_setup(p);
    if (s3 != NRE_OK) {
      delete p;
      return s3;
    }
    *plan = p;
    return NRE_OK;
  }
  if (chart->n0 < 4 || chart->n0 > 64 || (chart->n0 & 1))
    return set_error(NRE_EINVAL, "n0 must be even and in [4, 64] (levels are read as 2-vectors)");
  if (n_levels < 1 || n_levels > 10) return set_error(NRE_EINVAL, "n_levels must be in [1, 10]");
  if ((int64_t)chart->n0 << n_levels > 4096) return set_error(NRE_EINVAL, "n0 * 2^n_levels must be <= 4096");
  if (!(chart->r_min > 0 && chart->r_max > chart->r_min)) return set_error(NRE_EINVAL, "need 0 < r_min < r_max");
  if (!(kernel->rho > 0 && kernel->var > 0)) return set_error(NRE_EINVAL, "need rho > 0 and var > 0");
  if (dtype != NRE_F32 && dtype != NRE_F64) return set_error(NRE_EINVAL, "dtype must be NRE_F32 or NRE_F64");
  nre_icr_plan* p = new nre_icr_plan();
  p->dtype = dtype;
  p->n0 = chart->n0;
  p->n_levels = n_levels;
  p->r_min = chart->r_min;
  p->r_max = chart->r_max;
  p->rho = kernel->rho;
  p->var = kernel->var;
  p->status = nre::timeout_word();
  p->use_tma = p->status != nullptr;
  int64_t off = 0;
  for (int l = 0; l <= n_levels; ++l) {
    const int n = p->n0 << l;
    p->sizes.push_back(n);
    p->offsets.push_back(off);
    off += (int64_t)n * n;
  }
  p->latent = off;
  p->stride = round_up(off, 64);
  p->n_out = (int64_t)p->sizes.back() * p->sizes.back();
  // level 0
  const int n2 = p->n0 * p->n0;
  std::vector<double> K0((size_t)n2 * n2), L0;
  for (int a = 0; a < n2; ++a)
    for (int b = 0; b < n2; ++b)
      K0[(size_t)a * n2 + b] = matern32(p, chart_pos(p, 0, a / p->n0, a % p->n0), chart_pos(p, 0, b / p->n0, b % p->n0));
  if (!cholesky_jitter(K0, n2, 1e-10 * p->var, L0)) {
    delete p;
    return set_error(NRE_EINVAL, "level-0 kernel matrix is not positive definite");
  }
  std::vector<double> mats;
  for (int l = 0; l < n_levels; ++l) {
    p->mat_off.push_back((int64_t)mats.size());
    const int nc = p->sizes[l];
    for (int i = 0; i < nc; ++i) {
      double buf[MAT];
      if (!level_row_matrices(p, l, i, buf)) {
        delete p;
        return set_error(NRE_EINVAL, "refinement matrices of level %d row %d are not positive definite", l, i);
      }
      mats.insert(mats.end(), buf, buf + MAT);
    }
  }
  const int s = dtype == NRE_F64 ? upload_tables<double>(p, L0, mats) : upload_tables<float>(p, L0, mats);
  if (s != NRE_OK) {
    delete p;
    return s;
  }
  *plan = p;
  return NRE_OK;
}

int icr_destroy(nre_icr_plan* plan) {
  delete plan;
  return NRE_OK;
}

int icr_latent_layout(const nre_icr_plan* p, int64_t* n_out, int64_t* latent_size, int64_t* stride) {
  clear_error();
  if (!p) return set_error(NRE_EINVAL, "plan must not be NULL");
  if (n_out) *n_out = p->n_out;
  if (latent_size) *latent_size = p->latent;
  if (stride) *stride = p->stride;
  return NRE_OK;
}

#define NRE_ICR_CHECK(ptrs)                                                   \
  clear_error();                                                              \
  if (!plan) return set_error(NRE_EINVAL, "plan must not be NULL");           \
  if (batch < 0 || batch > 65535) return set_error(NRE_EINVAL, "batch must be in [0, 65535]"); \
  if (batch == 0) return NRE_OK;                                              \
  if (!(ptrs)) return set_error(NRE_EINVAL, "NULL array argument");

int icr_forward(nre_icr_plan* plan, const void* xi, void* s, int batch, nre_stream_t stream) {
  NRE_ICR_CHECK(xi && s);
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->dtype == NRE_F64) return icr_forward_t<double>(plan, (const double*)xi, (double*)s, batch, nullptr, st);
  return icr_forward_t<float>(plan, (const float*)xi, (float*)s, batch, nullptr, st);
}

int icr_jvp(nre_icr_plan* plan, const void* xi_p, const void* v, void* jv, int batch, nre_stream_t stream) {
  (void)xi_p;
  NRE_ICR_CHECK(v && jv);
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->dtype == NRE_F64) return icr_forward_t<double>(plan, (const double*)v, (double*)jv, batch, nullptr, st);
  return icr_forward_t<float>(plan, (const float*)v, (float*)jv, batch, nullptr, st);
}

int icr_vjp(nre_icr_plan* plan, const void* xi_p, const void* ct, void* g, int batch, nre_stream_t stream) {
  (void)xi_p;
  NRE_ICR_CHECK(ct && g);
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->dtype == NRE_F64)
    return icr_vjp_t<double>(plan, (const double*)ct, plan->n_out, (double*)g, nullptr, batch, st);
  return icr_vjp_t<float>(plan, (const float*)ct, plan->n_out, (float*)g, nullptr, batch, st);
}

}  // extern "C"
