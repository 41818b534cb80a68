// The ICR plan shared by the 2-D (icr.cu) and 3-D (icr3.cu) implementations.
#pragma once

#include <vector>

#include "metric_internal.cuh"

struct nre_icr_plan {
  int dtype = NRE_F32;
  int ndim = 2;                  // 2: log-radial chart; 3: spherical log-radial chart (icr3.cu)
  int n0 = 8, n_levels = 7;
  double r_min = 0.1, r_max = 1.0, rho = 0.1, var = 1.0;
  std::vector<int> sizes;        // n_l, l = 0..n_levels
  std::vector<int64_t> offsets;  // latent offset of level l
  int64_t latent = 0, stride = 0, n_out = 0;
  nre::DevBuf L0;                // [n0^2][n0^2] lower (row-major), plan dtype
  nre::DevBuf mats;              // 2-D, per level: [n_l][52]: R (4x9 row-major), L (4x4 row-major);
                                 // 3-D, per level: [n_l][n_l][280]: R (8x27), L (8x8), row-major
  std::vector<int64_t> mat_off;  // element offset of level l in mats
  nre::DevBuf ws_a, ws_b, ws_c;  // per-batch level buffers (3-D: ws_c holds the adjoint's R^T g)
  // 2-D adjoint: stage fine rows with bulk tensor copies; status counts the
  // waits that ran out (nre_wait_timeouts)
  bool use_tma = true;
  unsigned* status = nullptr;
  // second stream of a batch split into two halves (see icr_forward_t)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  nre_icr_plan() = default;
  nre_icr_plan(const nre_icr_plan&) = delete;
  nre_icr_plan& operator=(const nre_icr_plan&) = delete;
  ~nre_icr_plan() {
    if (side) cudaStreamDestroy(side);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
  }
};

namespace nre {
// 3-D chart (icr3.cu): plan set-up after the generic fields are filled, and
// the forward (scale: optional per-output factor [n_out]) / adjoint
// (base: optional [B][stride] added to the result) of a batch.
int icr3_setup(nre_icr_plan* p);
template <typename T>
int icr3_forward_t(nre_icr_plan* p, const T* xi, T* s, int B, const T* scale, cudaStream_t st);
template <typename T>
int icr3_vjp_t(nre_icr_plan* p, const T* ct, int64_t cts, T* g, const T* base, int B, cudaStream_t st);
}  // namespace nre
