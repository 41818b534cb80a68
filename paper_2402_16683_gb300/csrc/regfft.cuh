// Register-resident complex FFT of one line per thread group.
//
// A line of L = 2^n complex values is held by L/8 threads, 8 values each.  The
// transform is the self-sorting (Stockham) sequence of radix-8 passes and one
// final radix-4 or radix-2 pass (forward sign exp(-2 pi i k x / L)):
//   pass with radix R, Ns = product of earlier radices, butterflies j < L/R:
//     v_r = in[j + r L/R] * W_{Ns R}^{(j mod Ns) r},  v <- DFT_R(v),
//     out[(j div Ns) Ns R + (j mod Ns) + r Ns] = v_r.
// Thread t owns the butterflies j = t + (L/8) m, m < 8/R, so the first pass
// reads in[t + s L/8] (s = 0..7): exactly the elements the thread loads from
// global memory, coalesced across threads.  After the last pass the thread
// owns X[t + s L/8] in natural order, which feeds the Hartley unpack, the
// epilogue stores or the next transform without another pass through shared
// memory.  Between passes the values go through a padded shared buffer of the
// line (one pad element per 16).
#pragma once

#include <type_traits>

#include "fft.cuh"

namespace nre {

__host__ __device__ constexpr int rpad(int e) { return e + (e >> 4); }
// Exchange layouts: element e of a line at e + Q (e div 16), Q pad elements per
// 16.  Which Q keeps a half-warp's 8-byte accesses on distinct banks depends
// on the exchange (a model of the access patterns, checked for every line of
// 256..4096 points): after the first radix-8 pass Q = 1, after the second
// Q = 2 (with Q = 1 its scatter puts two lanes of each half-warp on one bank),
// the mirror exchange Q = 0 (its reversed reads collide at every other Q).
// Lines of up to 128 points (several lines per warp) and 16-byte elements
// keep Q = 1 throughout.
template <int Q>
__host__ __device__ constexpr int qpad(int e) { return e + Q * (e >> 4); }
template <typename C, int L, int NS>
__host__ __device__ constexpr int exch_q() { return (sizeof(C) == 8 && L / 8 >= 32 && NS == 8) ? 2 : 1; }
template <typename C, int L>
__host__ __device__ constexpr int mirror_q() { return (sizeof(C) == 8 && L / 8 >= 32) ? 0 : 1; }
// Line stride: room for the widest layout (Q = 2 from 256 points on: highest
// index L + L/8 - 3; the mirror exchange's extra element at qpad(L) with Q <= 1);
// up to 128 points an odd number of complex elements, so that the lines that
// share a warp sit on different banks (from 256 points on a warp holds one
// line, and the lines' relative banks do not matter).
__host__ __device__ constexpr int rline(int L) { return L >= 256 ? L + L / 8 : L + L / 16 + 1; }
// Line stride when NL lines are interleaved across the lanes of a warp: the
// lines start 16/NL complex elements apart modulo 16.
__host__ __device__ constexpr int rline_il(int L, int NL) { return L + L / 16 + (NL < 16 ? 16 / NL : 1); }

struct SyncBlock {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct SyncWarp {
  __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
// Named barrier of the `count` threads of one line (ids 1..15; 0 is __syncthreads).
struct SyncNamed {
  int id, count;
  __device__ __forceinline__ void operator()() const {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
  }
};

// Twiddles in shared memory, one table per pass with twiddles: the pass with
// stride NS and radix R stores W_{NS R}^{k r} at tw_off(L, NS) + (r - 1) NS + k
// (k < NS, 1 <= r < R), so a thread reads its R - 1 twiddles at one base
// address plus compile-time offsets.  The tables total fewer than L entries.
__host__ __device__ constexpr int pass_radix(int L, int NS) { return L / NS >= 8 ? 8 : L / NS; }
__host__ __device__ constexpr int tw_off(int L, int NS) {
  int off = 0;
  for (int ns = 8; ns < NS; ns *= 8) off += (pass_radix(L, ns) - 1) * ns;
  return off;
}
__host__ __device__ constexpr int tw_total(int L) { return tw_off(L, L); }

// Offset of qpad<Q>(base + r * NS) from qpad<Q>(base) for a pass's scatter,
// where base = (j - k) R + k with k = j mod NS (base mod 16 + r NS never
// crosses a 16-block other than through r NS itself).
__host__ __device__ constexpr int scatter_off(int NS, int r, int Q) {
  return NS == 1 ? r : (NS < 16 ? r * NS + Q * ((r * NS) >> 4) : r * NS + Q * r * (NS >> 4));
}

template <typename C, int L, int NS, int LPT>
struct RegPass {
  static constexpr int REM = L / NS;
  static constexpr int R = REM >= 8 ? 8 : REM;
  static constexpr int T8 = L / 8;
  static constexpr int M = 8 / R;
  static constexpr bool LAST = (NS * R == L);

  // T8 a multiple of 16 (L >= 128): the padded index of every scatter /
  // gather is one per-thread base plus a compile-time offset.
  static constexpr bool FAST = (T8 % 16) == 0;

  template <class Sync>
  __device__ __forceinline__ static void run(C (&v)[LPT][8], C* const* sm,
                                             const C* __restrict__ tw, int t, Sync sync) {
#pragma unroll
    for (int m = 0; m < M; ++m) {
      if constexpr (NS > 1) {
        const int j = t + T8 * m;
        const C* tk = tw + tw_off(L, NS) + (j & (NS - 1)) - NS;  // entry (r - 1) NS + k at tk + r NS
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const C w = tk[r * NS];
#pragma unroll
          for (int q = 0; q < LPT; ++q) v[q][m * R + r] = cmul(v[q][m * R + r], w);
        }
      }
#pragma unroll
      for (int q = 0; q < LPT; ++q) dftR<R>(&v[q][m * R]);
    }
    if constexpr (LAST) {
#pragma unroll
      for (int q = 0; q < LPT; ++q) {
        C o[8];
#pragma unroll
        for (int m = 0; m < M; ++m)
#pragma unroll
          for (int r = 0; r < R; ++r) o[m + r * M] = v[q][m * R + r];
#pragma unroll
        for (int s = 0; s < 8; ++s) v[q][s] = o[s];
      }
    } else {
      typedef RegPass<C, L, NS * R, LPT> Next;
      constexpr int R2 = Next::R, M2 = 8 / R2;
      constexpr int Q = exch_q<C, L, NS>();
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int j = t + T8 * m;
        const int k = j & (NS - 1);
        const int base = (j - k) * R + k;
        if constexpr (FAST) {
          const int pb = qpad<Q>(base);
#pragma unroll
          for (int q = 0; q < LPT; ++q)
#pragma unroll
            for (int r = 0; r < R; ++r) sm[q][pb + scatter_off(NS, r, Q)] = v[q][m * R + r];
        } else {
#pragma unroll
          for (int q = 0; q < LPT; ++q)
#pragma unroll
            for (int r = 0; r < R; ++r) sm[q][qpad<Q>(base + r * NS)] = v[q][m * R + r];
        }
      }
      sync();
      if constexpr (FAST) {
        // qpad(t + T8 s') = qpad(t) + s' (T8 + Q T8 / 16)
        const int pt = qpad<Q>(t);
#pragma unroll
        for (int q = 0; q < LPT; ++q)
#pragma unroll
          for (int m = 0; m < M2; ++m)
#pragma unroll
            for (int r = 0; r < R2; ++r) v[q][m * R2 + r] = sm[q][pt + (m + r * M2) * (T8 + Q * (T8 / 16))];
      } else {
#pragma unroll
        for (int q = 0; q < LPT; ++q)
#pragma unroll
          for (int m = 0; m < M2; ++m)
#pragma unroll
            for (int r = 0; r < R2; ++r) v[q][m * R2 + r] = sm[q][qpad<Q>(t + T8 * m + r * (L / R2))];
      }
      sync();
      Next::run(v, sm, tw, t, sync);
    }
  }
};

// Forward FFT of LPT lines; v[q][s] = line_q[t + s L/8] in and X_q[t + s L/8] out.
template <typename C, int L, int LPT, class Sync>
__device__ __forceinline__ void reg_fft(C (&v)[LPT][8], C* const* sm, const C* tw, int t, Sync sync) {
  RegPass<C, L, 1, LPT>::run(v, sm, tw, t, sync);
}

// zm[q][s] = X_q[-(t + s L/8) mod L] through the shared line buffers.
// For T8 a multiple of 16 the mirror reads qpad(L - t) - s (T8 + Q T8/16);
// thread 0's X[0] is also stored at qpad(L) (past the line's last element)
// for its s = 0 read.
template <typename C, int L, int LPT, class Sync>
__device__ __forceinline__ void reg_mirror(const C (&v)[LPT][8], C (&zm)[LPT][8], C* const* sm, int t,
                                           Sync sync) {
  constexpr int T8 = L / 8;
  if constexpr ((T8 % 16) == 0) {
    constexpr int Q = mirror_q<C, L>();
    constexpr int ST = T8 + Q * (T8 / 16);
    const int pt = qpad<Q>(t), pm = qpad<Q>(L - t);
#pragma unroll
    for (int q = 0; q < LPT; ++q) {
#pragma unroll
      for (int s = 0; s < 8; ++s) sm[q][pt + s * ST] = v[q][s];
      if (t == 0) sm[q][qpad<Q>(L)] = v[q][0];
    }
    sync();
#pragma unroll
    for (int q = 0; q < LPT; ++q)
#pragma unroll
      for (int s = 0; s < 8; ++s) zm[q][s] = sm[q][pm - s * ST];
    sync();
  } else {
#pragma unroll
    for (int q = 0; q < LPT; ++q)
#pragma unroll
      for (int s = 0; s < 8; ++s) sm[q][rpad(t + T8 * s)] = v[q][s];
    sync();
#pragma unroll
    for (int q = 0; q < LPT; ++q)
#pragma unroll
      for (int s = 0; s < 8; ++s) zm[q][s] = sm[q][rpad((L - (t + T8 * s)) & (L - 1))];
    sync();
  }
}

// Sum `val` over the runs of equal `key` among the lanes of a warp (runs are
// maximal ranges of consecutive lanes with the same key) and add each run's
// total to whist[key] from its last lane.  key < 0: no contribution.
// whist is a histogram that only this warp writes (a warp-private region of
// shared memory), so the result does not depend on how warps or CTAs are
// scheduled: runs of the same key that are not adjacent are added one after
// another in lane order (ranked with __match_any_sync), and successive calls
// add in program order.  The caller folds the warps'
// histograms in a fixed order (fold_bins).  The run sums are formed in V (the
// plan's value type: FP32 products of FP32 data are summed over at most 32
// lanes) and added to whist in H (FP32 for FP32 plans: an FP64 add and
// conversion per run costs more than the rest of the epilogue on this part,
// whose FP64 rate is a small fraction of its FP32 rate).
template <typename V, typename H>
__device__ __forceinline__ void warp_run_add(int key, V val, H* whist) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int prev = __shfl_up_sync(full, key, 1);
  const bool head = lane == 0 || prev != key;
  const unsigned heads = __ballot_sync(full, head);
  if (__all_sync(full, key < 0)) return;
  // first lane of this lane's run (lane 0 always heads a run)
  const int seg = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
  // steps of the segmented scan up to the longest run of the warp (the offsets
  // beyond it add nothing, so the sums are those of the full 5-step scan)
  const int maxrun = (int)__reduce_max_sync(full, (unsigned)(lane - seg + 1));
  for (int o = 1; o < maxrun; o <<= 1) {
    const V ov = __shfl_up_sync(full, val, o);
    if (lane - o >= seg) val += ov;
  }
  const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
  const bool act = tail && key >= 0;
  // The adds are shared-memory atomics so that they need no read round trip;
  // only this warp writes whist, in program order, so their order is fixed.
  // Keys monotone along the lanes (the sweeps' usual case: consecutive |k|)
  // give every run its own key, and the tails add at once.
  const bool mono = __all_sync(full, lane == 0 || prev <= key) || __all_sync(full, lane == 0 || prev >= key);
  if (mono) {
    if (act) atomicAdd(&whist[key], H(val));
  } else {
    // tails of other runs with the same key (inactive lanes get unique keys)
    const unsigned same = __match_any_sync(full, act ? key : -1 - lane);
    const int rank = __popc(same & ((1u << lane) - 1u));
    for (int r = 0; __any_sync(full, act && rank >= r); ++r) {
      if (act && rank == r) atomicAdd(&whist[key], H(val));
      __syncwarp();
    }
  }
}

// Adds the contributions c[s] of slots with bins bn[s] (all into the same
// warp-private histogram): slots sharing a bin are summed first, then each
// distinct bin is reduced over the warp.  Must be called by all lanes of the
// warp.
template <int S, typename V, typename H>
__device__ __forceinline__ void add_slots(const int (&bn)[S], const V (&c)[S], H* hist) {
#pragma unroll
  for (int s = 0; s < S; ++s) {
    int key = bn[s];
    V val = c[s];
#pragma unroll
    for (int s2 = 0; s2 < s; ++s2)
      if (bn[s2] == bn[s]) key = -1;
#pragma unroll
    for (int s2 = s + 1; s2 < S; ++s2)
      if (bn[s2] == bn[s]) val += c[s2];
    if (s == 0 || __any_sync(0xffffffffu, key >= 0)) warp_run_add(key, val, hist);
  }
}

}  // namespace nre
