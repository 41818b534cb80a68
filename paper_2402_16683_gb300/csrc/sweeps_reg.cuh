// Register-resident, pipelined Hartley sweeps (line lengths 8..4096).
//
// Row sweep: a unit is a reflection orbit of rows (D = 2: {i, -i}; D = 3:
// {(+-i0, +-i1)}) or, for D = 1, a pair of samples.  Two real rows form one
// complex line held by L/8 threads; each thread takes its 8 elements of both
// rows into the first radix-8 butterfly, runs the transform in registers,
// fetches the mirror elements X[-x] through shared memory, and applies the
// Hartley unpack, the reflection combination P (D >= 2; for D = 3 a thread owns
// both lines of its unit) and the epilogue in registers.  For D = 1 the
// metric's t = w * y and the second transform follow directly.
//
// Column sweep: a unit is a tile of W adjacent grid columns (all L rows of one
// outer index); columns 2p and 2p+1 form complex line p.  The tile is staged
// into shared memory row by row, each line is transformed by L/8 consecutive
// threads, and the results go back through a shared output tile so that global
// stores cover whole 32-byte sectors.  The axis-0 sweep of the 2-D / 3-D
// metric runs y = H_0 u, t = w * y and H_0 t back to back in registers, with
// the w tile staged beside the input tile.
//
// Both kernels are persistent over their units: while a CTA transforms one
// group, the inputs of its next group stream into the other half of a double
// buffer, so HBM reads overlap the arithmetic: whole rows by bulk copies
// (one per lane of warp 0, completing on an mbarrier) in the row sweep,
// tiles by bulk tensor copies in the FP32 column sweep (k_col_tma), 16-byte
// cp.async copies elsewhere.
// The threads of one line synchronise with warp or named barriers only.
// Per-bin amplitude tables (A and the tangent's dA) of the CTA's sample sit in
// shared memory; only the int16 bin index is read per pixel.  Log-|k| bin sums
// of the epilogue are reduced over runs of equal bins within each warp and
// added to the warp's own histogram (no atomics); the CTA folds its warps'
// histograms in order into one FP64 partial per sample (fold_bins).
#pragma once

#include "cf_internal.cuh"
#include "regfft.cuh"
#include "tma.cuh"

namespace nre {

template <int L>
struct RowShape {
  static constexpr int T8 = L / 8;
  static constexpr int NT = T8 > 256 ? T8 : 256;
  static constexpr int NU = NT / T8;  // units per CTA iteration
  static constexpr int NW = NT / 32;  // warps
  // Warp-private bin histograms (regions of nb entries): D >= 2 one per warp;
  // D = 1 two per unit (one per sample of the pair) while a unit fits in one
  // warp, else two per warp (the unit's warps fold theirs in order).
  __host__ __device__ static constexpr int hist_regions(int pm) { return pm == 1 ? (T8 <= 32 ? 2 * NU : 2 * NW) : NW; }
};

// Column tiles: NL complex lines (2 NL grid columns) per CTA.  FP32 tiles of
// lines >= 1024 take 512 threads so that a tile row spans 8 columns (32 bytes).
template <int L, int ES>
struct ColShape {
  static constexpr int T8 = L / 8;
  static constexpr int NTMIN = (ES == 4 && L >= 1024) ? 512 : 256;
  static constexpr int NT = T8 > NTMIN ? T8 : NTMIN;
  static constexpr int NL = NT / T8;            // complex lines per tile
  static constexpr int W = 2 * NL;              // grid columns per tile
  static constexpr int WP = W + 4;              // padded tile row (16-byte multiple)
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Per-pass twiddle tables (see tw_off) from the plan's table W_{Lmax}^m.
template <int L, typename C>
__device__ __forceinline__ void load_twiddles(C* tw, const C* gtw, int shift) {
  for (int i = threadIdx.x; i < tw_total(L); i += blockDim.x) {
    int ns = 8, off = 0;
    while (i >= off + (pass_radix(L, ns) - 1) * ns) {
      off += (pass_radix(L, ns) - 1) * ns;
      ns *= 8;
    }
    const int R = pass_radix(L, ns), e = i - off, r = e / ns + 1, k = e - (r - 1) * ns;
    tw[i] = gtw[(k * r * (L / (ns * R))) << shift];
  }
}

// Barrier of the T8 threads of line `u` (consecutive threads).
template <int T8>
struct LineSync {
  int id;
  __device__ __forceinline__ void operator()() const {
    if constexpr (T8 <= 32) {
      __syncwarp();
    } else {
      asm volatile("bar.sync %0, %1;\n" ::"r"(id), "n"(T8) : "memory");
    }
  }
};

// Per-bin tables of one sample in shared memory: A (from the per-bin model
// amplitude) into sA and the tangent's dA into sdA.  Returns whether the
// prologue / epilogue should read them (*use_dA: the dA table).  Called by all
// threads; a barrier must follow before use.
// With zero_slot, also sA[-1] = the zero mode's amplitude and sdA[-1] = 0, so
// that bin -1 (k = 0) indexes the tables like any other bin.
template <typename T>
__device__ __forceinline__ bool load_tables(const Pro<T>& pro, const Epi<T>& epi, int b, T* sA, T* sdA, int nb,
                                            bool* use_dA, bool zero_slot = false) {
  const AmpView<T>& v = pro.mode == PRO_AMP ? pro.av : epi.av;
  *use_dA = false;
  if (v.abin == nullptr || (v.mode != AMPV_MODEL && v.mode != AMPV_PIX)) return false;
  if (!(pro.mode == PRO_AMP || epi.mode == EPI_AMP)) return false;
  const bool dA = pro.mode == PRO_AMP && pro.dA != nullptr;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    sA[i] = T(v.abin[b * v.astride + i]);
    if (dA) sdA[i] = T(pro.dA[b * pro.nb + i]);
  }
  if (zero_slot && threadIdx.x == 0) {
    sA[-1] = v.a0t;
    sdA[-1] = T(0);
  }
  *use_dA = dA;
  return true;
}

// Shared-memory plan of the row kernel (element counts in T).
template <typename T, int L, int PM>
struct RowSmem {
  static constexpr int LPU = (PM == 3) ? 2 : 1;
  static constexpr int SLOTS = 2 * LPU;
  static constexpr int NU = RowShape<L>::NU;
  static constexpr int XSZ = NU * SLOTS * L;              // staged input rows
  static constexpr int LNSZ = NU * LPU * rline(L) * 2;    // exchange lines (complex)
  static constexpr int STG = (XSZ > LNSZ ? XSZ : LNSZ);
  static constexpr int STGA = (STG + 3) / 4 * 4;          // 16-byte multiple
  // the per-bin tables take 4 leading entries each (the zero mode at [-1])
  static size_t bytes(bool base, int nb, int nhist_bins) {
    return (size_t)2 * L * sizeof(T) + (size_t)2 * STGA * sizeof(T) + (base ? (size_t)XSZ * sizeof(T) : 0) +
           (size_t)(2 * ((nb + 3) / 4 * 4 + 4)) * sizeof(T) + (size_t)nhist_bins * sizeof(T);
  }
};

// Prologue / epilogue specialisations (compile time): GEN = the runtime
// functor of the arguments, BUF = plain copy, TAB = the metric's amplitude with
// per-pixel int16 bins and per-bin tables in shared memory.
enum { SK_GEN = 0, SK_BUF = 1, SK_TAB = 2 };

// CTAs per SM the sweeps are compiled for (the minimum of their
// __launch_bounds__; the host sizes persistent grids with it): four 256-thread
// CTAs for FP32 lines (at most 64 registers, measured without spills), three
// for FP64 lines and for the row sweep with the metric's epilogue at
// L >= 1024 (four would spill there), two for 3-D orbits (two lines per
// thread), one for wider CTAs.
__host__ __device__ constexpr int row_min_ctas(int nt, int pm, int ek, int es, int l) {
  return nt <= 256 ? (pm == 3 ? 2 : (((ek == SK_TAB && l >= 1024) || es == 8) ? 3 : 4)) : 1;
}
// The row sweep with the metric's epilogue loads its base values straight from
// global memory (with its other per-pixel loads) where that lets four CTAs
// share an SM; elsewhere the base rows are staged like the input rows, which
// hides their latency better at the lower occupancy.
__host__ __device__ constexpr bool row_direct_base(int nt, int pm, int ek, int es, int l) {
  return ek == SK_TAB && row_min_ctas(nt, pm, ek, es, l) >= 4;
}
__host__ __device__ constexpr int col_min_ctas(int nt, int es) { return nt <= 256 ? (es == 8 ? 3 : 4) : (nt <= 512 ? 2 : 1); }

// Bulk copies of one stage of a row sweep, issued by warp 0: lane i copies
// staged row i (unit group ug + i / SLOTS, slot i % SLOTS) of L elements from
// global memory (rows of `src`, samples `ss` elements apart) to shared address
// dst + i L elements, completing on the mbarrier at `bar`, whose transaction
// count lane 0 sets to the bytes of the valid rows.  Out of line: it runs once
// or twice per unit group and keeps its registers out of the sweep's.
template <typename T, int L, int PM, int SLOTS, int NROWS>
__device__ __noinline__ void row_issue_bulk(const T* src, int64_t ss, const int* grows, int n_units, int B, int ug,
                                            int bsample, unsigned dst, unsigned bar) {
  const int lane = threadIdx.x & 31;
  bool ok = false;
  const T* g = nullptr;
  if (lane < NROWS) {
    const int uu = lane / SLOTS, sl = lane - uu * SLOTS;
    const int un = ug + uu;
    const int samp = PM == 1 ? 2 * un + sl : bsample;
    ok = un < n_units && (PM != 1 || samp < B);
    if (ok) {
      const int row = PM == 1 ? 0 : __ldg(&grows[un * SLOTS + sl]);
      g = src + samp * ss + (int64_t)row * L;
    }
  }
  const unsigned nv = __popc(__ballot_sync(0xffffffffu, ok));
  constexpr unsigned RB = (unsigned)(L * sizeof(T));
  if (lane == 0) mbar_arrive_tx_at(bar, nv * RB);
  __syncwarp();
  if (ok) bulk_g2s(dst + (unsigned)lane * RB, g, RB, bar);
}

template <typename T, int L, int PM, bool MID, int PK, int EK>
__global__ void __launch_bounds__(RowShape<L>::NT, row_min_ctas(RowShape<L>::NT, PM, EK, sizeof(T), L))
    k_row_reg(RowArgs<T> a) {
  typedef typename CplxT<T>::type C;
  typedef RowSmem<T, L, PM> SM;
  constexpr int T8 = L / 8, NU = SM::NU, LPU = SM::LPU, SLOTS = SM::SLOTS, LS = rline(L);
  constexpr int CH = 16 / sizeof(T), CPR = L / CH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  T* stage = reinterpret_cast<T*>(tw + L);                  // [2][STGA]
  const bool sbase = a.epi.mode == EPI_AMP && a.epi.base != nullptr;
  constexpr bool DIRECT_BASE = row_direct_base(RowShape<L>::NT, PM, EK, sizeof(T), L);
  const bool bstaged = sbase && !DIRECT_BASE;
  T* bstage = stage + 2 * SM::STGA;                          // [XSZ]: the current units' base rows
  const int nbp = (a.nb + 3) / 4 * 4;
  T* sA = bstage + (bstaged ? SM::XSZ : 0) + 4;  // sA[-1], sdA[-1]: the zero mode (bin -1)
  T* sdA = sA + nbp + 4;
  T* hist = sdA + nbp;  // warp-private per-bin sums in T (FP32: see warp_run_add)
  const bool bins = a.epi.mode == EPI_AMP && a.epi.bins;
  constexpr int NW = RowShape<L>::NW, WPU = T8 > 32 ? T8 / 32 : 1;  // warps, warps per unit
  const int nhreg = RowShape<L>::hist_regions(PM);
  const int warp = threadIdx.x >> 5;
  // this warp's histogram: D >= 2 region `warp`; D = 1 with units inside one
  // warp the regions 2u, 2u + 1 of its units (keys offset by 2u nb), else the
  // two regions of the warp
  T* whist = PM == 1 ? (T8 <= 32 ? hist : hist + warp * 2 * a.nb) : hist + warp * a.nb;
  const int bsample = (PM == 1) ? 0 : blockIdx.y;
  const Pro<T>& pro = a.pro;
  const Epi<T>& epi = a.epi;
  load_twiddles<L>(tw, a.tw, a.log2Lmax - a.log2L);
  bool use_dA = false;
  const bool use_tab = (PM != 1) && load_tables<T>(pro, epi, bsample, sA, sdA, a.nb, &use_dA, true);
  const T* stab = use_tab ? sA : nullptr;
  const T* stdA = use_dA ? sdA : nullptr;
  if (bins)
    for (int i = threadIdx.x; i < nhreg * a.nb; i += blockDim.x) hist[i] = T(0);
  const int u = threadIdx.x / T8, t = threadIdx.x - u * T8;
  const LineSync<T8> sync{1 + u};

  // input rows of unit group ug into stage half buf (prefetched one iteration
  // ahead); with base, the base rows of ug into bstage (issued at the start of
  // their own iteration: they are read only by the epilogue, so one buffer
  // suffices and the staging plan stays small).  BULK (at most 32 rows per
  // stage): each lane of warp 0 copies one row with a bulk copy that
  // completes on the half's (bstage's) mbarrier, whose waits are bounded;
  // otherwise every thread copies 16-byte chunks with cp.async.
  constexpr int NROWS = NU * SLOTS;
  constexpr bool BULK = NROWS <= 32;
  __shared__ __align__(8) uint64_t sbar[3];  // stage halves, base rows
  if constexpr (BULK) {
    if (threadIdx.x == 0) {
#pragma unroll
      for (int i = 0; i < 3; ++i) mbar_init(&sbar[i], 1);
      mbar_fence_init();
    }
    __syncthreads();
  }
  auto issue_bulk = [&](int ug, int buf, bool base_only) {  // warp 0
    if (base_only)
      row_issue_bulk<T, L, PM, SLOTS, NROWS>(a.epi.base, a.epi.bs, a.grows, a.n_units, a.B, ug, bsample,
                                             smem_u32(bstage), smem_u32(&sbar[2]));
    else
      row_issue_bulk<T, L, PM, SLOTS, NROWS>(a.pro.x, a.pro.xs, a.grows, a.n_units, a.B, ug, bsample,
                                             smem_u32(stage + buf * SM::STGA), smem_u32(&sbar[buf]));
  };
  auto issue = [&](int ug, int buf, bool base_only) {
    T* dst = stage + buf * SM::STGA;
    T* bdst = bstage;
    // a whole number of chunks per thread (the block has RowShape<L>::NT threads)
    constexpr int NCH = NU * SLOTS * CPR, TRIPS = NCH / RowShape<L>::NT;
    static_assert(NCH % RowShape<L>::NT == 0, "chunks per thread");
#pragma unroll
    for (int k = 0; k < TRIPS; ++k) {
      const int c = threadIdx.x + k * RowShape<L>::NT;
      const int rr = c / CPR, j = c - rr * CPR;
      const int uu = rr / SLOTS, sl = rr - uu * SLOTS;
      const int un = ug + uu;
      const int samp = PM == 1 ? 2 * un + sl : bsample;
      if (un < a.n_units && (PM != 1 || samp < a.B)) {
        const int row = PM == 1 ? 0 : __ldg(&a.grows[un * SLOTS + sl]);
        const int64_t g = (int64_t)row * L + j * CH;
        if (base_only) cp_async16(bdst + rr * L + j * CH, a.epi.base + samp * a.epi.bs + g);
        else cp_async16(dst + rr * L + j * CH, a.pro.x + samp * a.pro.xs + g);
      }
    }
  };

  // fused inner product sum(base * y) of a metric product (see Epi::dot)
  const bool dot = PM >= 2 && epi.dot != nullptr;
  RunSum<T> dacc;
  const int ustride = gridDim.x * NU;
  int u0 = blockIdx.x * NU;
  int it = 0;
  bool timed_out = false;
  if constexpr (BULK) {
    if (threadIdx.x < 32 && u0 < a.n_units) issue_bulk(u0, 0, false);
  } else {
    if (u0 < a.n_units) issue(u0, 0, false);
    cp_commit();
  }
  for (; u0 < a.n_units && !timed_out; u0 += ustride, ++it) {
    const int cur = it & 1;
    if constexpr (BULK) {
      if (threadIdx.x < 32) {
        if (bstaged) issue_bulk(u0, 0, true);                                 // this iteration's base rows
        if (u0 + ustride < a.n_units) issue_bulk(u0 + ustride, cur ^ 1, false);  // next input
      }
      // this iteration's input rows
      const bool ok = mbar_wait(&sbar[cur], (unsigned)(it >> 1) & 1u);
      // a wait that ran out ends the loop after this iteration (its results
      // are void; the count in a.status tells the host)
      if (__syncthreads_or(!ok)) timed_out = true;
    } else {
      if (bstaged) issue(u0, 0, true);  // group B: this iteration's base rows
      cp_commit();
      if (u0 + ustride < a.n_units) issue(u0 + ustride, cur ^ 1, false);  // group A: next input
      cp_commit();
      cp_wait<2>();  // everything but B and A: this iteration's input rows
      __syncthreads();
    }
    const int unit = u0 + u;
    const bool valid = unit < a.n_units;
    int row[SLOTS], samp[SLOTS];
    bool sval[SLOTS];
#pragma unroll
    for (int sl = 0; sl < SLOTS; ++sl) {
      if (PM == 1) {
        samp[sl] = 2 * unit + sl;
        row[sl] = 0;
        sval[sl] = valid && samp[sl] < a.B;
      } else {
        samp[sl] = bsample;
        row[sl] = valid ? __ldg(&a.grows[unit * SLOTS + sl]) : 0;
        sval[sl] = valid;
      }
    }
    const T* X = stage + cur * SM::STGA + u * SLOTS * L;
    C v[LPU][8];
    if constexpr (PK == SK_GEN) {
#pragma unroll
      for (int q = 0; q < LPU; ++q)
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          const int x = t + T8 * s;
          const T re =
              sval[2 * q] ? pro.apply(samp[2 * q], (int64_t)row[2 * q] * L + x, X[(2 * q) * L + x], stab, stdA) : T(0);
          const T im = sval[2 * q + 1] ? pro.apply(samp[2 * q + 1], (int64_t)row[2 * q + 1] * L + x,
                                                   X[(2 * q + 1) * L + x], stab, stdA)
                                       : T(0);
          v[q][s] = cmake<C>(re, im);
        }
    } else if constexpr (PK == SK_BUF) {
#pragma unroll
      for (int q = 0; q < LPU; ++q)
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          const int x = t + T8 * s;
          v[q][s] = cmake<C>(sval[2 * q] ? X[(2 * q) * L + x] : T(0), sval[2 * q + 1] ? X[(2 * q + 1) * L + x] : T(0));
        }
    } else {
      // u = A[bin] v + dA[bin] xi_p (bins per pixel, tables in shared memory;
      // the metric's prologue always has the tangent's dA).  Rows that are
      // mirror images in the orbit (flags) share their bin row: only the
      // canonical slot's bins are loaded.
      const int16_t* bp = pro.av.bpix;
      const T* xp = pro.xi_p + (int64_t)bsample * pro.ps;
      const T a0 = pro.av.a0t;
      const int fl = valid ? __ldg(&a.gflags[unit]) : 0;
      const bool f0 = fl & 1;  // mirror rows of a 2-D orbit share the canonical slot's bins
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int x = t + T8 * s;
        int bn[LPU][2];
        T xv[LPU][2];
#pragma unroll
        for (int q = 0; q < LPU; ++q)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (PM == 2 && h == 1 && f0) bn[q][1] = bn[q][0];
            else bn[q][h] = valid ? (int)__ldg(&bp[row[2 * q + h] * L + x]) : -1;
            // the expansion point does not depend on the bin: its load goes
            // out with the bin's instead of after it
            xv[q][h] = __ldg(&xp[row[2 * q + h] * L + x]);
          }
#pragma unroll
        for (int q = 0; q < LPU; ++q) {
          T e[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int b_ = bn[q][h];
            T val = sA[b_] * X[(2 * q + h) * L + x];
            val += sdA[b_] * xv[q][h];  // (sdA[-1] = 0)
            e[h] = sval[2 * q + h] ? val : T(0);
          }
          v[q][s] = cmake<C>(e[0], e[1]);
        }
      }
    }
    __syncthreads();  // the stage half becomes the exchange buffer
    C* sm[LPU];
#pragma unroll
    for (int q = 0; q < LPU; ++q) sm[q] = reinterpret_cast<C*>(stage + cur * SM::STGA) + (u * LPU + q) * LS;
    C* const* smc = sm;
    reg_fft<C, L, LPU>(v, smc, tw, t, sync);
    C zm[LPU][8];
    if constexpr (MID) {
      reg_mirror<C, L, LPU>(v, zm, smc, t, sync);
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int x = t + T8 * s;
        T ha[2], hb[2];
        hartley_unpack<T>(v[0][s], zm[0][s], ha, hb);
        // samples of the pair (clamped into the batch: lanes of a missing
        // sample carry zeros)
        const int sa = samp[0] < a.B ? samp[0] : a.B - 1, sb = samp[1] < a.B ? samp[1] : a.B - 1;
        v[0][s] = cmake<C>(a.mid.at(sa, x) * ha[0], a.mid.at(sb, x) * hb[0]);
      }
      reg_fft<C, L, LPU>(v, smc, tw, t, sync);
    }
    reg_mirror<C, L, LPU>(v, zm, smc, t, sync);
    if (bstaged) {
      if constexpr (BULK) {
        const bool ok = mbar_wait(&sbar[2], (unsigned)it & 1u);
        if (__syncthreads_or(!ok)) timed_out = true;
      } else {
        cp_wait<1>();  // everything but group A: the base rows
        __syncthreads();
      }
    }
    const T* BV = bstage + u * SLOTS * L;
    if constexpr (EK == SK_TAB && PM >= 2) {
      // The metric's epilogue over column pairs: column x = t + T8 s (s < 4,
      // so x < L / 2) and its mirror x' = L - x.  Both outputs come
      // from the pair (z(x), z(x')) that the unpack reads (the mirror's with
      // the two columns' roles swapped: the same arithmetic as the unpack at
      // x' itself), and the bins, which depend on |k| only, are the same at x
      // and x', so each slot's two contributions go into one warp reduction.
      // Thread 0's pair at s = 0 is x = 0 and L / 2, each its own mirror.
      // Per phase of ECH pairs: A) the per-pixel loads (bins, expansion point,
      // base), all in flight before they are used, B) values, stores, bin
      // reductions.
      const int16_t* bp = epi.av.bpix;
      const T* xp = epi.xi_p + (int64_t)bsample * epi.ps;
      const T* bsrc = epi.base + (int64_t)bsample * epi.bs;  // the TAB epilogue always has a base
      T* yo = epi.y + (int64_t)bsample * epi.ys;
      const int fl = valid ? __ldg(&a.gflags[unit]) : 0;
      const bool f0 = fl & 1, f1 = fl & 2;
      const T half = T(0.5), a0 = epi.av.a0t;
      const bool t0 = t == 0;
      T dsum = T(0);
      // ECH column pairs per phase: all their loads go out before the first
      // is used (two pairs measured 0.6 % faster than one for FP32 2-D orbits
      // of 512 points and 4.5 % for 3-D orbits of 256; one where two would
      // spill more than a few bytes)
      constexpr int ECH = ((PM == 2 || PM == 3) && sizeof(T) == 4 && L >= 128) ? 2 : 1;
#pragma unroll
      for (int s0 = 0; s0 < 4; s0 += ECH) {
        int bnA[ECH][SLOTS], bn2A[ECH][SLOTS];
        T xvA[ECH][2][SLOTS], bvvA[ECH][2][SLOTS];
#pragma unroll
        for (int cc = 0; cc < ECH; ++cc) {
          const int s = s0 + cc;
          const int x = t + T8 * s;
          const bool sp = s == 0 && t0;
          const int x2 = sp ? L / 2 : L - x;
          int(&bn)[SLOTS] = bnA[cc];
          int(&bn2)[SLOTS] = bn2A[cc];
#pragma unroll
          for (int sl = 0; sl < SLOTS; ++sl) {
            // mirror rows of a 2-D orbit share the canonical slot's bins
            const int f = row[sl] * L + x, f2 = row[sl] * L + x2;
            if (PM == 2 && sl == 1 && f0) {
              bn[1] = bn[0];
              if (s == 0) bn2[1] = bn2[0];
            } else {
              bn[sl] = valid ? (int)__ldg(&bp[f]) : -1;
              if (s == 0) bn2[sl] = (valid && sp) ? (int)__ldg(&bp[f2]) : bn[sl];
            }
            if (s != 0) bn2[sl] = bn[sl];
            xvA[cc][0][sl] = valid ? __ldg(&xp[f]) : T(0);
            xvA[cc][1][sl] = valid ? __ldg(&xp[f2]) : T(0);
            if constexpr (DIRECT_BASE) {
              bvvA[cc][0][sl] = valid ? bsrc[f] : T(0);
              bvvA[cc][1][sl] = valid ? bsrc[f2] : T(0);
            } else {
              bvvA[cc][0][sl] = BV[sl * L + x];
              bvvA[cc][1][sl] = BV[sl * L + x2];
            }
          }
        }
#pragma unroll
        for (int cc = 0; cc < ECH; ++cc) {
          const int s = s0 + cc;
          const int x = t + T8 * s;
          const bool sp = s == 0 && t0;
          const int x2 = sp ? L / 2 : L - x;
          const int(&bn)[SLOTS] = bnA[cc];
          const int(&bn2)[SLOTS] = bn2A[cc];
          T (&xv)[2][SLOTS] = xvA[cc];
          T (&bvv)[2][SLOTS] = bvvA[cc];
          T val[2][SLOTS];
          if constexpr (PM == 2) {
            T R[2][2], R2[2][2];
            hartley_unpack<T>(v[0][s], zm[0][s], R[0], R[1]);
            if (s == 0) {
              hartley_unpack<T>(sp ? v[0][4] : v[0][0], sp ? zm[0][4] : zm[0][0], R2[0], R2[1]);
            } else {
#pragma unroll
              for (int i = 0; i < 2; ++i) R2[i][0] = R[i][0], R2[i][1] = R[i][1];
            }
#pragma unroll
            for (int sl = 0; sl < 2; ++sl) {
              val[0][sl] = half * (R[sl][0] + pick2(R, sl, f0, 0) + R[sl][1] - pick2(R, sl, f0, 1));
              val[1][sl] = half * (R2[sl][1] + pick2(R2, sl, f0, 1) + R2[sl][0] - pick2(R2, sl, f0, 0));
            }
          } else {
            T R[4][2], R2[4][2];
            hartley_unpack<T>(v[0][s], zm[0][s], R[0], R[1]);
            hartley_unpack<T>(v[1][s], zm[1][s], R[2], R[3]);
            if (s == 0) {
              hartley_unpack<T>(sp ? v[0][4] : v[0][0], sp ? zm[0][4] : zm[0][0], R2[0], R2[1]);
              hartley_unpack<T>(sp ? v[1][4] : v[1][0], sp ? zm[1][4] : zm[1][0], R2[2], R2[3]);
            } else {
#pragma unroll
              for (int i = 0; i < 4; ++i) R2[i][0] = R[i][0], R2[i][1] = R[i][1];
            }
#pragma unroll
            for (int sl = 0; sl < 4; ++sl) {
              val[0][sl] = half * (pick4(R, sl, f0, false, 0) + pick4(R, sl, false, f1, 0) + R[sl][1] -
                                   pick4(R, sl, f0, f1, 1));
              val[1][sl] = half * (pick4(R2, sl, f0, false, 1) + pick4(R2, sl, false, f1, 1) + R2[sl][0] -
                                   pick4(R2, sl, f0, f1, 0));
            }
          }
          T c[2 * SLOTS];
          int kb[2 * SLOTS];
#pragma unroll
          for (int sl = 0; sl < SLOTS; ++sl) {
            const T o = sA[bn[sl]] * val[0][sl] + bvv[0][sl];  // (sA[-1] = a0)
            const T o2 = sA[bn2[sl]] * val[1][sl] + bvv[1][sl];
            if (valid) {
              yo[row[sl] * L + x] = o;
              yo[row[sl] * L + x2] = o2;
              dsum += bvv[0][sl] * o;
              dsum += bvv[1][sl] * o2;
            }
            c[sl] = xv[0][sl] * val[0][sl];
            c[SLOTS + sl] = xv[1][sl] * val[1][sl];
            kb[sl] = bn[sl];
            kb[SLOTS + sl] = bn2[sl];
          }
          // the TAB epilogue always sums the bins
          if (s == 0) {
            add_slots<2 * SLOTS, T>(kb, c, whist);  // thread 0's second column has its own bins
          } else {
            T cm[SLOTS];
#pragma unroll
            for (int sl = 0; sl < SLOTS; ++sl) cm[sl] = c[sl] + c[SLOTS + sl];
            add_slots<SLOTS, T>(bn, cm, whist);
          }
        }
      }
      if (dot) dacc.add(dsum);
    } else {
    T dsum = T(0);
    // output of slot value `val` at row `rw`, column x of sample `sp`
    auto put = [&](int sp, int rw, int x, T val, T bval, int& bn, T& c) {
      if constexpr (EK == SK_BUF) {
        epi.y[(int64_t)sp * epi.ys + rw * L + x] = val;
        bn = -1;
        c = T(0);
      } else if constexpr (EK == SK_TAB) {
        const int f = rw * L + x;
        bn = __ldg(&epi.av.bpix[f]);
        epi.y[(int64_t)sp * epi.ys + f] = (bn < 0 ? epi.av.a0t : sA[bn]) * val + bval;
        c = (bins && bn >= 0) ? __ldg(&epi.xi_p[(int64_t)sp * epi.ps + f]) * val : T(0);
        if (!bins) bn = -1;
      } else {
        const T o = epi.store_b(sp, (int64_t)rw * L + x, val, bval, bn, c, stab);
        dsum += bval * o;
      }
    };
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int x = t + T8 * s;
      if (PM == 1) {
        T ha[2], hb[2];
        hartley_unpack<T>(v[0][s], zm[0][s], ha, hb);
        int bn[2] = {-1, -1};
        T c[2] = {T(0), T(0)};
        if (sval[0]) put(samp[0], 0, x, ha[0], sbase ? BV[x] : T(0), bn[0], c[0]);
        if (sval[1]) put(samp[1], 0, x, hb[0], sbase ? BV[L + x] : T(0), bn[1], c[1]);
        if (bins) {
          const int ub = T8 <= 32 ? 2 * u : 0;  // the unit's regions within whist
          warp_run_add(bn[0] >= 0 ? ub * a.nb + bn[0] : -1, c[0], whist);
          if (__any_sync(0xffffffffu, bn[1] >= 0))
            warp_run_add(bn[1] >= 0 ? (ub + 1) * a.nb + bn[1] : -1, c[1], whist);
        }
      } else if (PM == 2) {
        T R[2][2];
        hartley_unpack<T>(v[0][s], zm[0][s], R[0], R[1]);
        const bool f0 = valid && (a.gflags[unit] & 1);
        const T half = T(0.5);
        int bn[2] = {-1, -1};
        T c[2] = {T(0), T(0)};
#pragma unroll
        for (int sl = 0; sl < 2; ++sl) {
          const T val = half * (R[sl][0] + pick2(R, sl, f0, 0) + R[sl][1] - pick2(R, sl, f0, 1));
          if (valid) put(bsample, row[sl], x, val, sbase ? BV[sl * L + x] : T(0), bn[sl], c[sl]);
        }
        if (bins) add_slots<2, T>(bn, c, whist);
      } else {
        T R[4][2];
        hartley_unpack<T>(v[0][s], zm[0][s], R[0], R[1]);
        hartley_unpack<T>(v[1][s], zm[1][s], R[2], R[3]);
        const int fl = valid ? a.gflags[unit] : 0;
        const bool f0 = fl & 1, f1 = fl & 2;
        const T half = T(0.5);
        int bn[4] = {-1, -1, -1, -1};
        T c[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int sl = 0; sl < 4; ++sl) {
          const T val = half * (pick4(R, sl, f0, false, 0) + pick4(R, sl, false, f1, 0) + R[sl][1] -
                                pick4(R, sl, f0, f1, 1));
          if (valid) put(bsample, row[sl], x, val, sbase ? BV[sl * L + x] : T(0), bn[sl], c[sl]);
        }
        if (bins) add_slots<4, T>(bn, c, whist);
      }
    }
    if (dot) dacc.add(dsum);
    }  // generic epilogue
    // this half is refilled two iterations later (and bstage in the next):
    // the generic-proxy accesses come before the bulk copies' writes
    if constexpr (BULK) fence_proxy_async();
    __syncthreads();
  }
  if constexpr (BULK) {
    if (timed_out && threadIdx.x == 0) {
      note_timeout(a.status);
      // the copies that may still be in flight: those of the last iteration
      // (lt) and the input it issued for the next unit group (at u0)
      const int lt = it - 1;
      mbar_wait(&sbar[lt & 1], (unsigned)(lt >> 1) & 1u);
      if (bstaged) mbar_wait(&sbar[2], (unsigned)lt & 1u);
      if (u0 < a.n_units) mbar_wait(&sbar[it & 1], (unsigned)(it >> 1) & 1u);
    }
  } else {
    cp_wait<0>();
  }
  if (dot) {
    const double tot = dacc.block_sum();
    double* dp = epi.dot + (int64_t)blockIdx.y * kDotStride;
    if (threadIdx.x == 0) dp[blockIdx.x] = tot;
    if (blockIdx.x == 0)
      for (int i = gridDim.x + threadIdx.x; i < kDotStride; i += blockDim.x) dp[i] = 0.0;
  }
  if (bins) {
    __syncthreads();
    if (PM == 1) {
      // one CTA holds every pixel of its sample pairs: complete sums
      for (int i = threadIdx.x; i < 2 * NU * a.nb; i += blockDim.x) {
        const int hs = i / a.nb, bn = i - hs * a.nb;  // hs = 2 (unit) + slot
        const int sample = 2 * (blockIdx.x * NU) + hs;
        double tot;
        if (T8 <= 32) {
          tot = double(hist[i]);
        } else {
          tot = 0.0;
          for (int w = 0; w < WPU; ++w) tot += double(hist[((hs >> 1) * WPU + w) * 2 * a.nb + (hs & 1) * a.nb + bn]);
        }
        if (sample < a.B) (a.epi.gsum ? a.epi.gsum : a.partials)[(int64_t)sample * a.nb + bn] = tot;
      }
    } else {
      fold_bins(a.epi, a.partials, bsample, gridDim.x, blockIdx.x, hist, NW, a.nb, a.nb);
    }
  }
}

// Shared-memory plan of the column kernel (element counts in T).
template <typename T, int L>
struct ColSmem {
  typedef ColShape<L, sizeof(T)> CS;
  static constexpr int XS = L * CS::WP;                              // one staged tile
  static constexpr int LNSZ = CS::NL * rline(L) * 2;                 // exchange lines
  // the exchange lines live in the current tile once it is in registers when
  // they fit (short lines carry relatively more padding and get their own)
  static constexpr bool ALIAS = LNSZ <= XS;
  static size_t bytes(int nb, int nhist_bins) {
    return (size_t)2 * L * sizeof(T) + (size_t)2 * XS * sizeof(T) + (ALIAS ? 0 : (size_t)LNSZ * sizeof(T)) +
           (size_t)(2 * ((nb + 3) / 4 * 4)) * sizeof(T) + (size_t)nhist_bins * sizeof(T);
  }
};

template <typename T, int L, bool MID, int PK, int EK>
__global__ void __launch_bounds__(ColShape<L, sizeof(T)>::NT, col_min_ctas(ColShape<L, sizeof(T)>::NT, sizeof(T)))
    k_col_reg(ColArgs<T> a) {
  typedef typename CplxT<T>::type C;
  typedef ColSmem<T, L> SM;
  constexpr int T8 = L / 8, WP = ColShape<L, sizeof(T)>::WP;
  constexpr int LS = rline(L), CH = 16 / sizeof(T);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  T* xin = reinterpret_cast<T*>(tw + L);      // [2][XS]; the current half is also the output tile
  const int nbp = (a.nb + 3) / 4 * 4;
  C* lines_own = reinterpret_cast<C*>(xin + 2 * SM::XS);  // used when !SM::ALIAS
  T* sA = xin + 2 * SM::XS + (SM::ALIAS ? 0 : SM::LNSZ);
  T* sdA = sA + nbp;
  T* hist = sdA + nbp;  // warp-private per-bin sums in T (FP32: see warp_run_add)
  const bool bins = a.epi.mode == EPI_AMP && a.epi.bins;
  constexpr int NW = ColShape<L, sizeof(T)>::NT / 32;
  T* whist = hist + (threadIdx.x >> 5) * a.nb;
  const int b = blockIdx.y;
  const Pro<T>& pro = a.pro;
  const Epi<T>& epi = a.epi;
  load_twiddles<L>(tw, a.tw, a.log2Lmax - a.log2L);
  bool use_dA = false;
  const bool use_tab = load_tables<T>(pro, epi, b, sA, sdA, a.nb, &use_dA);
  const T* stab = use_tab ? sA : nullptr;
  const T* stdA = use_dA ? sdA : nullptr;
  if (bins)
    for (int i = threadIdx.x; i < NW * a.nb; i += blockDim.x) hist[i] = T(0);
  const int u = threadIdx.x / T8, t = threadIdx.x - u * T8;
  const LineSync<T8> sync{1 + u};
  // W, the chunks per tile row and the tiles per outer index are powers of two:
  // shifts and masks instead of run-time divisions
  const int W = a.W, CPR = W / CH, cpr_sh = __ffs(CPR) - 1;
  const int nblk_sh = __ffsll(a.nblk) - 1;
  const bool lval = 2 * u < W;

  auto tile_base = [&](int64_t unit) -> int64_t {
    const int64_t o = unit >> nblk_sh;
    return o * L * a.inner + (unit & (a.nblk - 1)) * W;
  };
  auto issue = [&](int64_t unit, int buf) {
    const T* src = a.pro.x + b * a.pro.xs + tile_base(unit);
    T* dst = xin + buf * SM::XS;
    for (int c = threadIdx.x; c < L * CPR; c += blockDim.x) {
      const int l = c >> cpr_sh, j = c & (CPR - 1);
      cp_async16(dst + l * WP + j * CH, src + (int64_t)l * a.inner + j * CH);
    }
  };

  int64_t unit = blockIdx.x;
  if (unit < a.n_units) issue(unit, 0);
  cp_commit();
  for (int it = 0; unit < a.n_units; unit += gridDim.x, ++it) {
    const int cur = it & 1;
    if (unit + gridDim.x < a.n_units) issue(unit + gridDim.x, cur ^ 1);
    cp_commit();
    cp_wait<1>();
    __syncthreads();
    const int64_t base = tile_base(unit);
    T* X = xin + cur * SM::XS;
    C v[1][8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int l = t + T8 * s;
      if (lval) {
        const C raw = *reinterpret_cast<const C*>(X + l * WP + 2 * u);
        if constexpr (PK == SK_BUF) {
          v[0][s] = raw;
        } else {
          const int64_t flat = base + (int64_t)l * a.inner + 2 * u;
          v[0][s] = cmake<C>(pro.apply(b, flat, raw.x, stab, stdA), pro.apply(b, flat + 1, raw.y, stab, stdA));
        }
      } else {
        v[0][s] = cmake<C>(T(0), T(0));
      }
    }
    if (SM::ALIAS) __syncthreads();  // the whole tile is in registers: its space becomes the exchange lines
    C* sm[1] = {(SM::ALIAS ? reinterpret_cast<C*>(X) : lines_own) + u * LS};
    C* const* smc = sm;
    reg_fft<C, L, 1>(v, smc, tw, t, sync);
    C zm[1][8];
    if constexpr (MID) {
      reg_mirror<C, L, 1>(v, zm, smc, t, sync);
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        T ha[2], hb[2];
        hartley_unpack<T>(v[0][s], zm[0][s], ha, hb);
        const int64_t flat = base + (int64_t)(t + T8 * s) * a.inner + 2 * u;
        v[0][s] = lval ? a.mid.apply2(b, flat, ha[0], hb[0]) : cmake<C>(T(0), T(0));
      }
      reg_fft<C, L, 1>(v, smc, tw, t, sync);
    }
    reg_mirror<C, L, 1>(v, zm, smc, t, sync);
    __syncthreads();  // every line has read the input tile: reuse it for the output
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      T ha[2], hb[2];
      hartley_unpack<T>(v[0][s], zm[0][s], ha, hb);
      if (lval) *reinterpret_cast<C*>(X + (t + T8 * s) * WP + 2 * u) = cmake<C>(ha[0], hb[0]);
    }
    __syncthreads();
    // write the tile back row by row (CH consecutive columns per thread); the
    // loop is uniform over the block so the warp reductions see full warps
    for (int c0 = 0; c0 < L * CPR; c0 += blockDim.x) {
      const int c = c0 + threadIdx.x;
      const bool act = c < L * CPR;
      const int l = act ? c >> cpr_sh : 0, j = act ? c & (CPR - 1) : 0;
      const int64_t flat = base + (int64_t)l * a.inner + j * CH;
      const T* src = X + l * WP + j * CH;
      if constexpr (EK == SK_BUF) {
        if (act) *reinterpret_cast<uint4*>(epi.y + b * epi.ys + flat) = *reinterpret_cast<const uint4*>(src);
      } else {
#pragma unroll
        for (int e = 0; e < CH; ++e) {
          int bn = -1;
          T cc = T(0);
          if (act)
            epi.store_b(b, flat + e, src[e],
                        (epi.mode == EPI_AMP && epi.base) ? epi.base[b * epi.bs + flat + e] : T(0), bn, cc, stab);
          if (bins) warp_run_add(bn, cc, whist);
        }
      }
    }
    __syncthreads();  // tiles of this half are refilled two iterations later
  }
  cp_wait<0>();
  if (bins) {
    __syncthreads();
    fold_bins(a.epi, a.partials, b, gridDim.x, blockIdx.x, hist, NW, a.nb, a.nb);
  }
}

// Column sweep of FP32 plain buffers (the metric's axis-0 sweep, MID, and the
// 3-D middle-axis sweeps) with its tiles moved by bulk tensor copies.  One
// elected thread loads the next unit's tile (W columns x L rows, boxes of at
// most 256 rows) into the other half of the double buffer, completing on that
// half's mbarrier, and stores each finished output tile from shared memory
// with a bulk tensor store; the threads only transform.  Tiles are dense rows
// of W floats (32 / 64 / 128 bytes) in the copies' swizzled layout, which
// keeps a half-warp's 8-byte column-pair accesses at two wavefronts.  Waits
// are bounded: a wait that runs out (decided for the whole CTA) is counted in
// *status and the CTA stops after waiting, again bounded, for its copies.
// The metric's sweep (MID) also loads the unit's tile of the weights w (same
// boxes and layout, one buffer) when the unit starts; it is first read after
// the forward transform, which hides the copy.
template <int L>
struct ColTma {
  typedef ColShape<L, 4> CS;
  static constexpr int W = CS::W, XS = L * W, RB = L < 256 ? L : 256, NBOX = L / RB;
  static constexpr unsigned SWM = W == 8 ? 0x10u : (W == 16 ? 0x30u : 0x70u);
  static constexpr int SWB = W * 4;  // swizzle span in bytes
  // a buffer holds a tile and, once the tile is in registers, the exchange
  // lines; buffers start at multiples of 1024 bytes (the swizzle's alignment)
  static constexpr int LNSZ = CS::NL * rline(L) * 2;  // floats
  static constexpr int BUFB = ((XS > LNSZ ? XS : LNSZ) * 4 + 1023) / 1024 * 1024;
  // bytes: the two buffers, the weights (MID), the twiddle tables, the three
  // mbarriers; the dynamic shared memory (the kernel's only shared memory)
  // starts on a 1024-byte boundary, which the kernel checks
  static constexpr int TWB = (tw_total(L) * 8 + 15) / 16 * 16;
  static constexpr size_t bytes(bool mid) { return (size_t)2 * BUFB + (mid ? (size_t)XS * 4 : 0) + TWB + 32; }
  // four CTAs per SM (1 KB reserved per CTA, 228 KB per SM) for lines of up to 512 points
  static_assert(L > 512 || 4 * (bytes(true) + 1024) <= 228 * 1024, "column tiles exceed a quarter SM");
  // float index of element (l, col) of a tile
  __device__ __forceinline__ static int at(int l, int col) {
    const unsigned A = (unsigned)(l * W + col) * 4u;
    return (int)((A ^ ((A >> 3) & SWM)) >> 2);
  }
};

template <int L, bool MID>
__global__ void __launch_bounds__(ColShape<L, 4>::NT, col_min_ctas(ColShape<L, 4>::NT, 4))
    k_col_tma(ColArgs<float> a, const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
              const __grid_constant__ CUtensorMap twt, int wb, unsigned* status) {
  typedef float T;
  typedef float2 C;
  typedef ColTma<L> TM;
  constexpr int T8 = L / 8, W = TM::W, XS = TM::XS, RB = TM::RB, NBOX = TM::NBOX, LS = rline(L);
  extern __shared__ __align__(1024) unsigned char smem_tma[];
  unsigned char* bufs = smem_tma;
  // the swizzled tiles need 1024-byte alignment (the layout's assumption; a
  // CTA that finds otherwise does nothing and is counted)
  if ((smem_u32(bufs) & 1023u) != 0) {
    if (threadIdx.x == 0) note_timeout(status);
    return;
  }
  auto tile = [&](int buf) { return reinterpret_cast<T*>(bufs + buf * TM::BUFB); };
  T* WT = reinterpret_cast<T*>(bufs + 2 * TM::BUFB);  // MID: the unit's weights (a multiple of 1024 bytes)
  C* tw = reinterpret_cast<C*>(bufs + 2 * TM::BUFB + (MID ? XS * 4 : 0));
  uint64_t* bar = reinterpret_cast<uint64_t*>(bufs + 2 * TM::BUFB + (MID ? XS * 4 : 0) + TM::TWB);  // halves, weights
  const int b = blockIdx.y;
  load_twiddles<L>(tw, a.tw, a.log2Lmax - a.log2L);
  const int u = threadIdx.x / T8, t = threadIdx.x - u * T8;
  const LineSync<T8> sync{1 + u};
  const int nblk_sh = __ffsll(a.nblk) - 1;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&bar[2], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int64_t unit, int buf) {  // elected thread
    const int z = (int)(unit >> nblk_sh), x = (int)((unit & (a.nblk - 1)) * W);
    mbar_arrive_tx(&bar[buf], (unsigned)(XS * 4));
#pragma unroll
    for (int k = 0; k < NBOX; ++k) tma_load_4d(tile(buf) + k * RB * W, &tin, x, k * RB, z, b, &bar[buf]);
  };
  int64_t unit = blockIdx.x;
  if (threadIdx.x == 0 && unit < a.n_units) issue(unit, 0);
  int it = 0;
  bool timed_out = false;
  for (; unit < a.n_units; unit += gridDim.x, ++it) {
    const int cur = it & 1;
    if (threadIdx.x == 0 && unit + gridDim.x < a.n_units) {
      bulk_wait_read0();  // the store of two units ago has read the other half
      issue(unit + gridDim.x, cur ^ 1);
    }
    if (MID && threadIdx.x == 0) {
      // this unit's weights (the last unit's reads of WT came before the
      // proxy fence and barrier ahead of its store)
      const int z = (int)(unit >> nblk_sh), x = (int)((unit & (a.nblk - 1)) * W);
      mbar_arrive_tx(&bar[2], (unsigned)(XS * 4));
#pragma unroll
      for (int k = 0; k < NBOX; ++k) tma_load_4d(WT + k * RB * W, &twt, x, k * RB, z, wb * b, &bar[2]);
    }
    const bool ok = mbar_wait(&bar[cur], (unsigned)(it >> 1) & 1u);
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      break;
    }
    const int64_t o = unit >> nblk_sh;
    T* X = tile(cur);
    C v[1][8];
#pragma unroll
    for (int s = 0; s < 8; ++s) v[0][s] = *reinterpret_cast<const C*>(X + TM::at(t + T8 * s, 2 * u));
    __syncthreads();  // the whole tile is in registers: its buffer becomes the exchange lines
    C* sm[1] = {reinterpret_cast<C*>(X) + u * LS};
    C* const* smc = sm;
    reg_fft<C, L, 1>(v, smc, tw, t, sync);
    C zm[1][8];
    if constexpr (MID) {
      reg_mirror<C, L, 1>(v, zm, smc, t, sync);
      const bool okw = mbar_wait(&bar[2], (unsigned)it & 1u);
      if (__syncthreads_or(!okw)) {
        timed_out = true;
        break;
      }
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        T ha[2], hb[2];
        hartley_unpack<T>(v[0][s], zm[0][s], ha, hb);
        const C ww = *reinterpret_cast<const C*>(WT + TM::at(t + T8 * s, 2 * u));
        v[0][s] = cmake<C>(ww.x * ha[0], ww.y * hb[0]);
      }
      reg_fft<C, L, 1>(v, smc, tw, t, sync);
    }
    reg_mirror<C, L, 1>(v, zm, smc, t, sync);
    __syncthreads();  // every line has read the input tile: it takes the output
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      T ha[2], hb[2];
      hartley_unpack<T>(v[0][s], zm[0][s], ha, hb);
      *reinterpret_cast<C*>(X + TM::at(t + T8 * s, 2 * u)) = cmake<C>(ha[0], hb[0]);
    }
    fence_proxy_async();  // the generic-proxy writes before the async-proxy store
    __syncthreads();
    if (threadIdx.x == 0) {
      const int z = (int)o, x = (int)((unit & (a.nblk - 1)) * W);
#pragma unroll
      for (int k = 0; k < NBOX; ++k) tma_store_4d(&tout, x, k * RB, z, b, X + k * RB * W);
      bulk_commit();
    }
  }
  if (timed_out && threadIdx.x == 0) {
    note_timeout(status);
    // the loads in flight: the current unit's (and its weights) and the one
    // issued for the next
    mbar_wait(&bar[it & 1], (unsigned)(it >> 1) & 1u);
    if (MID) mbar_wait(&bar[2], (unsigned)it & 1u);
    if (unit + gridDim.x < a.n_units) mbar_wait(&bar[(it + 1) & 1], (unsigned)((it + 1) >> 1) & 1u);
  }
  if (threadIdx.x == 0) bulk_wait0();
}

}  // namespace nre
