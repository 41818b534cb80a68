// Launchers of the register-resident sweep kernels.  The kernels are
// instantiated once per (dtype, line length) in sweeps_inst.cu (compiled once
// per combination with -DNRE_SWEEP_T / -DNRE_SWEEP_L) so the build runs in
// parallel; sweeps.cu dispatches on the line length.
#pragma once

#include "sweeps_reg.cuh"

namespace nre {

constexpr int kMaxGridX = 128;      // CTAs per sample of a sweep (bounds the partials buffer)
static_assert(kMaxGridX <= kBinGroup * (kGcntStride - 1), "arrival counters of the in-place bin sums");

// CTAs of a persistent register sweep resident at once: per SM the fewer of
// the kernel's compiled minimum (row_min_ctas / col_min_ctas) and what its
// shared memory admits (1 KB reserved per CTA), times the SMs of the device.
inline int resident_ctas(int min_ctas, size_t smem) {
  static const int2 dev = [] {
    int d = 0, nsm = 152, sm = 228 * 1024;
    cudaGetDevice(&d);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, d);
    cudaDeviceGetAttribute(&sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, d);
    return make_int2(nsm, sm);
  }();
  int per = (int)((size_t)dev.y / (smem + 1024));
  if (per > min_ctas) per = min_ctas;
  if (per < 1) per = 1;
  return per * dev.x;
}

// Algorithmic bytes of a sweep: per-sample arrays count B times, arrays shared
// by the batch (expansion point, weights, fixed spectrum) once.
template <typename T>
double sweep_bytes(const Pro<T>& pro, const Epi<T>& epi, const Mid<T>* mid, bool has_mid, int B,
                   int64_t N) {
  const double e = (double)N * sizeof(T);
  double per = 2.0, shared = 0.0;  // the input x and the output y
  if (pro.mode == PRO_AMP) {
    if (pro.av.mode != AMPV_MODEL) shared += 1.0;
    if (pro.dA) (pro.ps ? per : shared) += 1.0;
  } else if (pro.mode == PRO_SQRTW) {
    shared += 1.0;
  }
  if (epi.mode == EPI_AMP) {
    if (epi.base) per += 1.0;
    if (epi.bins) (epi.ps ? per : shared) += 1.0;
    if (epi.av.mode != AMPV_MODEL && !(pro.mode == PRO_AMP && pro.av.mode != AMPV_MODEL)) shared += 1.0;
  } else if (epi.mode == EPI_WEIGHT && epi.mask) {
    shared += 1.0;
  }
  if (has_mid) shared += 1.0;
  return e * (per * B + shared);
}

inline const char* row_name(int pm, bool mid, int es) {
  static const char* names[2][4] = {
      {"row_sweep_f32_1d", "row_sweep_f32_1d_metric", "row_sweep_f32_2d", "row_sweep_f32_3d"},
      {"row_sweep_f64_1d", "row_sweep_f64_1d_metric", "row_sweep_f64_2d", "row_sweep_f64_3d"}};
  const int t = es == 8 ? 1 : 0;
  return pm == 1 ? names[t][mid ? 1 : 0] : names[t][pm];
}

// Fills the grid, shared-memory size and partial count of a row sweep;
// NRE_EINVAL if the register kernel does not fit (use the generic one).
template <typename T, int L>
int row_reg_plan(RowArgs<T>& a, int B, bool bins, dim3* grid, size_t* smem, int* nparts);
template <typename T, int L>
int row_reg_L(RowArgs<T> a, bool mid, dim3 grid, size_t smem, cudaStream_t st, int64_t N);
template <typename T, int L>
int col_reg_L(ColArgs<T> a, bool mid, int B, bool bins, int* nparts, cudaStream_t st, int64_t N);

#define NRE_DECL_SWEEP(T, L)                                                                   \
  extern template int row_reg_plan<T, L>(RowArgs<T>&, int, bool, dim3*, size_t*, int*);        \
  extern template int row_reg_L<T, L>(RowArgs<T>, bool, dim3, size_t, cudaStream_t, int64_t);  \
  extern template int col_reg_L<T, L>(ColArgs<T>, bool, int, bool, int*, cudaStream_t, int64_t);
#define NRE_DECL_SWEEP_T(T)                                                                     \
  NRE_DECL_SWEEP(T, 8) NRE_DECL_SWEEP(T, 16) NRE_DECL_SWEEP(T, 32) NRE_DECL_SWEEP(T, 64)         \
  NRE_DECL_SWEEP(T, 128) NRE_DECL_SWEEP(T, 256) NRE_DECL_SWEEP(T, 512) NRE_DECL_SWEEP(T, 1024)   \
  NRE_DECL_SWEEP(T, 2048) NRE_DECL_SWEEP(T, 4096)

}  // namespace nre
