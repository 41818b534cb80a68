// Likelihood and metric objects shared by metric.cu, cg.cu and icr.cu.
#pragma once

#include <vector>

#include "cf_internal.cuh"

struct nre_icr_plan;

struct nre_lik {
  int kind = NRE_LIK_GAUSS, response = NRE_RESP_EXP;
  double sig_or_scale = 1.0;
  std::vector<double> mask;  // empty: every pixel observed
  int64_t n_data = 0;
};

struct nre_metric {
  int model_kind = NRE_MODEL_CF;
  nre_cf_plan* cf = nullptr;
  nre_icr_plan* icr = nullptr;
  int dtype = NRE_F32;
  int max_batch = 1;
  int64_t n_data = 0, latent = 0, stride = 0;
  nre_lik lik;
  nre::DevBuf xi_p;     // [stride] copy of the expansion point
  nre::DevBuf w;        // [n_data] Fisher weights at xi_p
  nre::DevBuf mask;     // [n_data] or empty
  nre::DevBuf state;    // amplitude state at xi_p (power model)
  nre::DevBuf apix;     // [n_data] A_full at xi_p per pixel (power model)
  nre::DevBuf bpix;     // [n_data] int16 log-|k| bin per pixel (power model)
  nre::DevBuf dA;       // [max_batch][n_bins]
  nre::DevBuf tmp0, tmp1, part;
  // conjugate-gradient workspace (grown by cg_solve)
  nre::DevBuf cg_r, cg_p, cg_q, cg_sc, cg_part;
  std::vector<double> cg_host;
  // preconditioner (metric_set_precond)
  int precond = 0;
  double pc_c = 0.0;      // N * mean(w)
  int pc_nh = 0;          // hyper-parameters handled by the Schur block
  nre::DevBuf pc_G;       // float [n_hyper][n_bins]: dA_b / dh at xi_p
  nre::DevBuf pc_Sinv;    // float [n_hyper][n_hyper]: inverse Schur complement
  nre::DevBuf cg_z, pc_gz, pc_part;
};

namespace nre {
// Amplitude view of the metric's expansion point: per-pixel tables for the
// power model, the plan's per-pixel spectrum for the fixed kinds.
template <typename T>
AmpView<T> metric_view(const nre_metric* m);
// out = v + J^T (w * J v) for a batch (dtype-dispatched inside).
int metric_apply_impl(nre_metric* m, const void* v, void* out, int batch, cudaStream_t st);
// ICR model hooks (icr.cu).
int icr_metric_setup(nre_metric* m, cudaStream_t st);
int icr_metric_apply(nre_metric* m, const void* v, void* out, int batch, cudaStream_t st);
int icr_mgvi_rhs(nre_metric* m, const void* xi_prime, const void* eta, void* b, int batch,
                 cudaStream_t st);
int icr_layout(const nre_icr_plan* p, int64_t* n_out, int64_t* latent, int64_t* stride, int* dtype);
// Preconditioned CG (pcg.cu), used by cg_solve when m->precond != NRE_PRECOND_NONE.
int pcg_solve_impl(nre_metric* m, const void* b, void* x, int batch, double rtol, int maxiter,
                   int* iters_out, double* relres_out, cudaStream_t st);
}  // namespace nre
