// One (dtype, line length) instantiation of the register-resident sweep
// kernels and their launchers.  The build compiles this file once per
// combination with -DNRE_SWEEP_T=float|double -DNRE_SWEEP_L=8..4096; without
// the defines it compiles to nothing.
#include "sweeps_launch.cuh"

#if defined(NRE_SWEEP_T) && defined(NRE_SWEEP_L)

namespace nre {

template <typename K>
static int set_smem(K k, size_t smem) {
  return raise_smem(k, smem);
}

template <typename T, int L, int PM, bool MID, int PK, int EK>
int launch_row_k(const RowArgs<T>& a, dim3 grid, size_t smem, cudaStream_t st) {
  NRE_TRY(set_smem(k_row_reg<T, L, PM, MID, PK, EK>, smem));
  k_row_reg<T, L, PM, MID, PK, EK><<<grid, RowShape<L>::NT, smem, st>>>(a);
  return NRE_OK;
}

template <typename T, int L, int PM>
int launch_row_pm(const RowArgs<T>& a, int pk, int ek, dim3 grid, size_t smem, cudaStream_t st) {
  if (pk == SK_TAB && ek == SK_BUF) return launch_row_k<T, L, PM, false, SK_TAB, SK_BUF>(a, grid, smem, st);
  if (pk == SK_BUF && ek == SK_TAB) return launch_row_k<T, L, PM, false, SK_BUF, SK_TAB>(a, grid, smem, st);
  if (pk == SK_BUF && ek == SK_BUF) return launch_row_k<T, L, PM, false, SK_BUF, SK_BUF>(a, grid, smem, st);
  return launch_row_k<T, L, PM, false, SK_GEN, SK_GEN>(a, grid, smem, st);
}

template <typename T>
int pro_kind(const Pro<T>& p) {
  if (p.mode == PRO_BUF) return SK_BUF;
  // TAB: the metric's prologue (per-pixel bins, the tangent's dA)
  return (p.mode == PRO_AMP && p.av.mode == AMPV_PIX && p.av.bpix != nullptr && p.dA != nullptr) ? SK_TAB : SK_GEN;
}
template <typename T>
int epi_kind(const Epi<T>& e) {
  if (e.mode == EPI_BUF) return SK_BUF;
  // TAB: the metric / MGVI epilogue (per-pixel bins, a base, bin sums)
  return (e.mode == EPI_AMP && e.av.mode == AMPV_PIX && e.av.bpix != nullptr && e.base != nullptr && e.bins)
             ? SK_TAB
             : SK_GEN;
}

template <typename T, int L>
int row_reg_L(RowArgs<T> a, bool mid, dim3 grid, size_t smem, cudaStream_t st, int64_t N) {
  const char* name = row_name(a.pm, mid, sizeof(T));
  // the staged rows (input, and the base rows where they are staged) are
  // copied in 16-byte pieces or whole by bulk copies: rows and samples must
  // start on 16-byte boundaries
  auto al = [](const void* q, int64_t stride) {
    return reinterpret_cast<uintptr_t>(q) % 16 == 0 && (stride * (int64_t)sizeof(T)) % 16 == 0;
  };
  if (!al(a.pro.x, a.pro.xs) || (a.epi.mode == EPI_AMP && a.epi.base != nullptr && !al(a.epi.base, a.epi.bs)))
    return set_error(NRE_EINVAL, "internal: row sweep rows not 16-byte aligned");
  a.status = timeout_word();
  prof_begin(name, sweep_bytes<T>(a.pro, a.epi, &a.mid, mid, a.B, N), st);
  int s;
  if (a.pm == 1) {
    s = mid ? launch_row_k<T, L, 1, true, SK_GEN, SK_GEN>(a, grid, smem, st)
            : launch_row_k<T, L, 1, false, SK_GEN, SK_GEN>(a, grid, smem, st);
  } else {
    const int pk = pro_kind(a.pro), ek = epi_kind(a.epi);
    s = a.pm == 2 ? launch_row_pm<T, L, 2>(a, pk, ek, grid, smem, st)
                  : launch_row_pm<T, L, 3>(a, pk, ek, grid, smem, st);
  }
  prof_end(st);
  NRE_TRY(s);
  NRE_CHECK_LAUNCH();
  return NRE_OK;
}

// CTAs per sample of a persistent sweep: about `resident` in total, at least
// one, at most one per unit group and at most kMaxGridX.
inline int persistent_gx(int64_t groups, int B, int resident) {
  int64_t gx = (resident + B - 1) / B;
  if (gx > groups) gx = groups;
  if (gx > kMaxGridX) gx = kMaxGridX;
  return gx < 1 ? 1 : (int)gx;
}

template <typename T, int L>
int row_reg_plan(RowArgs<T>& a, int B, bool bins, dim3* grid, size_t* smem, int* nparts) {
  constexpr int NU = RowShape<L>::NU;
  const bool sbase = a.epi.mode == EPI_AMP && a.epi.base != nullptr;
  if (a.pm == 1) {
    a.n_units = (B + 1) / 2;
    *grid = dim3((a.n_units + NU - 1) / NU, 1);  // one group per CTA: histograms per sample
    *nparts = 1;
  }
  a.nU = NU;
  const int pm = a.pm;
  const int ek = pm == 1 ? SK_GEN : epi_kind(a.epi);
  const bool bstaged = sbase && !row_direct_base(RowShape<L>::NT, pm, ek, sizeof(T), L);
  const int hreg = RowShape<L>::hist_regions(pm);  // warp-private bin histograms
  *smem = pm == 1   ? RowSmem<T, L, 1>::bytes(bstaged, a.nb, bins ? hreg * a.nb : 0)
          : pm == 2 ? RowSmem<T, L, 2>::bytes(bstaged, a.nb, bins ? hreg * a.nb : 0)
                    : RowSmem<T, L, 3>::bytes(bstaged, a.nb, bins ? hreg * a.nb : 0);
  if (pm != 1) {
    const int gx = persistent_gx((a.n_units + NU - 1) / NU, B,
                                 resident_ctas(row_min_ctas(RowShape<L>::NT, pm, ek, sizeof(T), L), *smem));
    *grid = dim3(gx, B);
    *nparts = gx;
  }
  return *smem <= 200 * 1024 ? NRE_OK : NRE_EINVAL;
}

template <typename T, int L>
int col_reg_L(ColArgs<T> a, bool mid, int B, bool bins, int* nparts, cudaStream_t st, int64_t N) {
  constexpr int NT = ColShape<L, sizeof(T)>::NT;
  const size_t smem = ColSmem<T, L>::bytes(a.nb, bins ? (NT / 32) * a.nb : 0);  // warp-private histograms
  const int gx = persistent_gx(a.n_units, B, resident_ctas(col_min_ctas(NT, sizeof(T)), smem));
  *nparts = gx;
  if (smem > 200 * 1024) return set_error(NRE_EINVAL, "column sweep of length %d needs %zu bytes of shared memory", L, smem);
  const dim3 grid((unsigned)gx, B);
  const char* name = sizeof(T) == 8 ? (mid ? "col_sweep_f64_metric" : "col_sweep_f64")
                                    : (mid ? "col_sweep_f32_metric" : "col_sweep_f32");
  const bool buf = a.pro.mode == PRO_BUF && a.epi.mode == EPI_BUF;
  if (mid && !buf) return set_error(NRE_EINVAL, "internal: the metric's column sweep reads and writes plain buffers");
  prof_begin(name, sweep_bytes<T>(a.pro, a.epi, &a.mid, mid, B, N), st);
  if constexpr (sizeof(T) == 4 && L >= 128 && L <= 1024) {
    // FP32 plain buffers with whole tiles: bulk tensor copies
    auto al = [](const void* q) { return reinterpret_cast<uintptr_t>(q) % 16 == 0; };
    unsigned* status = timeout_word();
    if (buf && a.W == ColShape<L, 4>::W && a.inner % 4 == 0 && a.pro.xs % 4 == 0 && a.epi.ys % 4 == 0 &&
        al(a.pro.x) && al(a.epi.y) && status != nullptr) {
      typedef ColTma<L> TM;
      const int64_t outer = a.n_units / a.nblk;
      const uint64_t dims[4] = {(uint64_t)a.inner, (uint64_t)L, (uint64_t)outer, (uint64_t)B};
      const uint64_t sin[3] = {(uint64_t)a.inner * 4, (uint64_t)L * a.inner * 4, (uint64_t)a.pro.xs * 4};
      const uint64_t sout[3] = {(uint64_t)a.inner * 4, (uint64_t)L * a.inner * 4, (uint64_t)a.epi.ys * 4};
      const uint32_t box[4] = {(uint32_t)TM::W, (uint32_t)TM::RB, 1u, 1u};
      CUtensorMap tin, tout, twt;
      int s = tmap_tiled(&tin, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.pro.x, dims, sin, box, TM::SWB);
      if (s == NRE_OK) s = tmap_tiled(&tout, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.epi.y, dims, sout, box, TM::SWB);
      int wb = 0;  // the weights' sample coordinate per sample: 0 when all samples share w
      if (s == NRE_OK && mid) {
        // the weights w ([N] shared, or [B][N]) in the tiles' geometry
        if (!al(a.mid.w) || a.mid.ws % 4 != 0) {
          s = NRE_EINVAL;
        } else {
          wb = a.mid.ws != 0 ? 1 : 0;
          const uint64_t wd[4] = {dims[0], dims[1], dims[2], (uint64_t)(wb ? B : 1)};
          const uint64_t sw[3] = {sin[0], sin[1], wb ? (uint64_t)a.mid.ws * 4 : sin[1] * (uint64_t)outer};
          s = tmap_tiled(&twt, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.mid.w, wd, sw, box, TM::SWB);
        }
      }
      if (s == NRE_OK) {
        const size_t tsm = TM::bytes(mid);
        // persistent grid for this kernel's own shared memory (no bin sums here)
        const int gxt = persistent_gx(a.n_units, B, resident_ctas(col_min_ctas(NT, 4), tsm));
        *nparts = gxt;
        const dim3 gridt((unsigned)gxt, B);
        if (mid) {
          NRE_TRY(set_smem(k_col_tma<L, true>, tsm));
          k_col_tma<L, true><<<gridt, NT, tsm, st>>>(a, tin, tout, twt, wb, status);
        } else {
          NRE_TRY(set_smem(k_col_tma<L, false>, tsm));
          k_col_tma<L, false><<<gridt, NT, tsm, st>>>(a, tin, tout, tin, 0, status);
        }
        prof_end(st);
        NRE_CHECK_LAUNCH();
        return NRE_OK;
      }
      clear_error();  // fall back to the staged kernel
    }
  }
  if (mid) {
    NRE_TRY(set_smem(k_col_reg<T, L, true, SK_BUF, SK_BUF>, smem));
    k_col_reg<T, L, true, SK_BUF, SK_BUF><<<grid, NT, smem, st>>>(a);
  } else if (buf) {
    NRE_TRY(set_smem(k_col_reg<T, L, false, SK_BUF, SK_BUF>, smem));
    k_col_reg<T, L, false, SK_BUF, SK_BUF><<<grid, NT, smem, st>>>(a);
  } else {
    NRE_TRY(set_smem(k_col_reg<T, L, false, SK_GEN, SK_GEN>, smem));
    k_col_reg<T, L, false, SK_GEN, SK_GEN><<<grid, NT, smem, st>>>(a);
  }
  prof_end(st);
  NRE_CHECK_LAUNCH();
  return NRE_OK;
}

template int row_reg_plan<NRE_SWEEP_T, NRE_SWEEP_L>(RowArgs<NRE_SWEEP_T>&, int, bool, dim3*, size_t*, int*);
template int row_reg_L<NRE_SWEEP_T, NRE_SWEEP_L>(RowArgs<NRE_SWEEP_T>, bool, dim3, size_t, cudaStream_t, int64_t);
template int col_reg_L<NRE_SWEEP_T, NRE_SWEEP_L>(ColArgs<NRE_SWEEP_T>, bool, int, bool, int*, cudaStream_t, int64_t);

}  // namespace nre

#endif
