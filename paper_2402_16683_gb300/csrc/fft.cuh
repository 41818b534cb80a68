// Block-level complex FFT of several lines held in shared memory.
//
// Each transform is a self-sorting (Stockham) sequence of radix-8 passes
// followed by one radix-4 or radix-2 pass for the remaining factor; pass p with
// radix R and Ns = product of the earlier radices maps
//     v_r = in[j + r L/R] * W_{Ns R}^{(j mod Ns) r},  v <- DFT_R(v),
//     out[(j div Ns) Ns R + (j mod Ns) + r Ns] = v_r,
// ping-ponging between two shared buffers.  Forward sign: exp(-2 pi i kx/L).
// Twiddles W_Lmax^m = exp(-2 pi i m / Lmax) come from a table of the longest
// line length of the plan (computed on the host in FP64).
//
// Two shared-memory layouts:
//   LayRow - line-major with one pad element every 8 (lines = rows of a grid);
//   LayCol - element-major, lines interleaved (lines = adjacent grid columns).
// The butterfly enumeration follows the layout so that consecutive threads touch
// consecutive shared addresses in the read phase.
#pragma once

#include "common.cuh"

namespace nre {

struct LayRow {
  int ls;  // line stride in complex elements: L + L/8
  __device__ __forceinline__ int idx(int line, int e) const { return line * ls + e + (e >> 3); }
  __device__ __forceinline__ void split(int q, int nl, int lr, int& line, int& j) const {
    line = q / lr;
    j = q - line * lr;
  }
  static __host__ __device__ int stride(int L) { return L + L / 8; }
};

struct LayCol {
  int nl;  // number of interleaved lines
  __device__ __forceinline__ int idx(int line, int e) const { return e * nl + line; }
  __device__ __forceinline__ void split(int q, int nl_, int lr, int& line, int& j) const {
    j = q / nl;
    line = q - j * nl;
  }
};

template <typename C>
__device__ __forceinline__ void dft2(C* v) {
  C a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <typename C>
__device__ __forceinline__ void dft4(C& x0, C& x1, C& x2, C& x3) {
  C t0 = cadd(x0, x2), t1 = csub(x0, x2);
  C t2 = cadd(x1, x3), t3 = cmul_mi(csub(x1, x3));
  x0 = cadd(t0, t2);
  x2 = csub(t0, t2);
  x1 = cadd(t1, t3);
  x3 = csub(t1, t3);
}

template <typename C>
__device__ __forceinline__ void dft8(C* v) {
  typedef decltype(C::x) T;
  const T h = T(0.70710678118654752440);  // 1/sqrt(2)
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4(e0, e1, e2, e3);
  dft4(o0, o1, o2, o3);
  // twiddles W8^k, k = 1..3: (1 - i)/sqrt2, -i, (-1 - i)/sqrt2
  C t1 = cmake<C>(h * (o1.x + o1.y), h * (o1.y - o1.x));
  C t2 = cmul_mi(o2);
  C t3 = cmake<C>(h * (o3.y - o3.x), -h * (o3.x + o3.y));
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, t1);
  v[5] = csub(e1, t1);
  v[2] = cadd(e2, t2);
  v[6] = csub(e2, t2);
  v[3] = cadd(e3, t3);
  v[7] = csub(e3, t3);
}

template <int R, typename C>
__device__ __forceinline__ void dftR(C* v) {
  if constexpr (R == 8) dft8(v);
  else if constexpr (R == 4) dft4(v[0], v[1], v[2], v[3]);
  else dft2(v);
}

// One Stockham pass over nl lines of length L.
template <int R, typename C, class Lay>
__device__ __forceinline__ void stockham_pass(const C* __restrict__ in, C* __restrict__ out, int nl,
                                              int L, int Ns, const C* __restrict__ tw,
                                              int tw_shift, Lay lay) {
  const int lr = L / R;
  const int nb = nl * lr;
  const int step = (lr / Ns) << tw_shift;  // L/(Ns R) in units of the Lmax table
  for (int q = threadIdx.x; q < nb; q += blockDim.x) {
    int line, j;
    lay.split(q, nl, lr, line, j);
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[lay.idx(line, j + r * lr)];
    const int k = j & (Ns - 1);
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], __ldg(&tw[k * r * step]));
    }
    dftR<R>(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) out[lay.idx(line, base + r * Ns)] = v[r];
  }
}

// Full forward FFT of nl lines of length L = 2^log2L held in buffer a (b is
// scratch of the same size).  Returns the buffer holding the result.  Ends
// with a __syncthreads().  Precondition: the data in `a` are visible to the
// block (a __syncthreads() after writing them).
template <typename C, class Lay>
__device__ C* block_fft(C* a, C* b, int nl, int L, int log2L, const C* __restrict__ tw,
                        int log2Lmax, Lay lay) {
  int Ns = 1, rem = log2L;
  const int tw_shift = log2Lmax - log2L;
  while (rem > 0) {
    if (rem >= 3) {
      stockham_pass<8>(a, b, nl, L, Ns, tw, tw_shift, lay);
      Ns <<= 3;
      rem -= 3;
    } else if (rem == 2) {
      stockham_pass<4>(a, b, nl, L, Ns, tw, tw_shift, lay);
      Ns <<= 2;
      rem -= 2;
    } else {
      stockham_pass<2>(a, b, nl, L, Ns, tw, tw_shift, lay);
      Ns <<= 1;
      rem -= 1;
    }
    __syncthreads();
    C* t = a;
    a = b;
    b = t;
  }
  return a;
}

// Hartley unpack of a complex line Z = FFT(a + i b) at positions x and
// x' = -x mod L:  H_a[x] = (X + X' - Y + Y')/2,  H_b[x] = (X - X' + Y + Y')/2,
// with Z[x] = X + iY, Z[x'] = X' + iY'.  ha/hb [0] at x, [1] at x'.
template <typename T, typename C>
__device__ __forceinline__ void hartley_unpack(C z, C zm, T* ha, T* hb) {
  const T half = T(0.5);
  ha[0] = half * (z.x + zm.x - z.y + zm.y);
  hb[0] = half * (z.x - zm.x + z.y + zm.y);
  ha[1] = half * (zm.x + z.x - zm.y + z.y);
  hb[1] = half * (zm.x - z.x + zm.y + z.y);
}

// R[s ^ m] of the reflection-orbit values of one column with s known at
// compile time (unrolled loops) and the mask m = f0 + 2 f1 known only at run
// time, written as selects so that R stays in registers.
template <typename T>
__device__ __forceinline__ T pick2(const T (&R)[2][2], int s, bool f0, int c) {
  return f0 ? R[s ^ 1][c] : R[s][c];
}
template <typename T>
__device__ __forceinline__ T pick4(const T (&R)[4][2], int s, bool f0, bool f1, int c) {
  const T a = f0 ? R[s ^ 1][c] : R[s][c];
  const T b = f0 ? R[s ^ 3][c] : R[s ^ 2][c];
  return f1 ? b : a;
}

}  // namespace nre
