// Likelihood and metric objects shared by metric.cu, cg.cu and icr.cu.
#pragma once

#include <vector>

#include "cf_internal.cuh"

struct nre_icr_plan;
struct nre_kl;

// Model kind of the sample-averaged KL metric (kl.cu); internal: such metric
// objects come from kl_metric and are owned by their KL object.
constexpr int NRE_MODEL_KL = 2;

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
  nre_kl* kl = nullptr;  // NRE_MODEL_KL
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
  // FP32 power model: the amplitude Jacobian at xi_p (see amp_jacobian)
  bool amp_lin = false;
  nre::DevBuf amp_G, amp_Gt, amp_eye, amp_Jt;
  nre::DevBuf gsum;  // [max_batch][n_bins] complete bin sums of the last sweep
  nre::DevBuf gcnt;  // [max_batch][kGcntStride] unsigned arrival counters of those sums (zero between sweeps)
  nre::DevBuf tmp0, tmp1, part;
  // conjugate-gradient workspace (grown by cg_solve)
  nre::DevBuf cg_r, cg_p, cg_q, cg_sc, cg_part;
  nre::DevBuf cg_dot;  // [max batch][kDotStride] fused p.q partials
  nre::DevBuf cg_pn;   // [batch][n_hyper] the current p_h when CG handles the hyper block (cg.cu)
  std::vector<double> cg_host;
  // preconditioner (metric_set_precond)
  int precond = 0;
  int pc_nh = 0;          // hyper-parameters handled by the Schur block
  nre::DevBuf pc_G;       // float [n_hyper][n_bins]: dA_b / dh at xi_p
  nre::DevBuf pc_Sinv;    // float [n_hyper][n_hyper]: inverse Schur complement
  nre::DevBuf cg_z, pc_gz, pc_part;
  nre::DevBuf pc_tmp, pc_eye, pc_dG;  // preconditioner set-up scratch
  nre::DevBuf pc_A, pc_W, pc_T1, pc_Sd;  // FP64 Schur block, its factor, Woodbury product, S^-1
  nre::DevBuf pc_invD, pc_e;          // per pixel: 1 / D and A xi_p / D
  nre::DevBuf pc_Gt;                  // float [n_bins][n_hyper]: G transposed
  nre::DevBuf pc_cdev;                // double: c = N mean(w), on the device
  // residual correction (refine.cu): FP64 metric: residual, product, partials;
  // low precision metric: right-hand side and correction of the inner solve
  nre::DevBuf rf_r, rf_q, rf_part;
  // geoVI update (geovi.cu): p per system, shifted points, VJP output,
  // coordinate residual, Newton step, model values, t(p) and dt(p), partials
  nre::DevBuf gv_pp, gv_pts, gv_u, gv_F, gv_step, gv_cf, gv_tp, gv_part;
  // second stream of a metric product split into two half batches (metric.cu)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  nre_metric() = default;
  nre_metric(const nre_metric&) = delete;
  nre_metric& operator=(const nre_metric&) = delete;
  ~nre_metric() {
    if (side) cudaStreamDestroy(side);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
  }
};

namespace nre {
// Amplitude view of the metric's expansion point: per-pixel tables for the
// power model, the plan's per-pixel spectrum for the fixed kinds.
template <typename T>
AmpView<T> metric_view(const nre_metric* m);
// out = v + J^T (w * J v) for a batch (dtype-dispatched inside).  With `dot`
// (correlated field only) also the inner products v . out as partials
// dot[b * kDotStride + i], whose sum over i is the product of system b.
// hyper_in_cg (FP32 power model with the linearised amplitude, CG only): the
// caller has formed dA for v and zeroed gsum, and forms the hyper part of out
// and of the inner product itself from gsum (see CGHyper in cg.cu); the
// product then covers the field part only.
int metric_apply_impl(nre_metric* m, const void* v, void* out, int batch, cudaStream_t st,
                      double* dot = nullptr, bool hyper_in_cg = false);
// ICR model hooks (icr.cu).
int icr_metric_setup(nre_metric* m, cudaStream_t st);
int icr_metric_apply(nre_metric* m, const void* v, void* out, int batch, cudaStream_t st);
int icr_mgvi_rhs(nre_metric* m, const void* xi_prime, const void* eta, void* b, int batch,
                 cudaStream_t st);
int icr_layout(const nre_icr_plan* p, int64_t* n_out, int64_t* latent, int64_t* stride, int* dtype);
// Residual correction in pieces (refine.cu), enqueue only: with d_lo (the
// low precision correction of the last inner solve, lo->rf_q in cg_solve_refined)
// x += d_lo first and the residual is r = b - M_hi x, else r = b; the sums
// r.r (and with with_bb b.b) per system land in *sums ([B] then [B], device).
// refine_down casts r of the systems flagged in active_host (host int[B]) to
// lo's dtype into lo->rf_r (zeros for the others).
int refine_residual(nre_metric* lo, nre_metric* hi, const double* b, double* x, const void* d_lo, int B,
                    bool with_bb, double** sums, cudaStream_t st);
int refine_down(nre_metric* lo, nre_metric* hi, int B, const int* active_host, void** rlo, cudaStream_t st);
// The KL's sample-averaged metric (kl.cu): out[b] = Mbar v[b].
int kl_metric_apply(nre_kl* k, const void* v, void* out, int batch, cudaStream_t st);
// Preconditioned CG (pcg.cu), used by cg_solve when m->precond != NRE_PRECOND_NONE.
int pcg_solve_impl(nre_metric* m, const void* b, void* x, int batch, double rtol, int maxiter,
                   int* iters_out, double* relres_out, cudaStream_t st);

// CG in pieces (cg.cu / pcg.cu), for callers that advance many solves at once
// without waiting on each: cg_begin enqueues x = 0, r = b and the initial
// scalars; cg_iterate enqueues `iters` iterations; neither synchronises.  The
// per-system scalars live on the device in m->cg_sc, CG_SC_N doubles per
// system, with the entries below (rr = r.r, bb = b.b, active = 1 while the
// system runs, iters = iterations taken).  cg_read_scalars copies them to
// m->cg_host and waits; cg_report turns them into iterations / relres and
// the NRE_ENOTCONV status.
enum { CG_SC_RR = 0, CG_SC_BB = 1, CG_SC_ACTIVE = 4, CG_SC_ITERS = 5, CG_SC_N = 8 };
int cg_begin(nre_metric* m, const void* b, void* x, int batch, double rtol, cudaStream_t st);
int cg_iterate(nre_metric* m, void* x, int batch, int iters, double rtol, cudaStream_t st);
int pcg_begin(nre_metric* m, const void* b, void* x, int batch, double rtol, cudaStream_t st);
int pcg_iterate(nre_metric* m, void* x, int batch, int iters, double rtol, cudaStream_t st);
int cg_read_scalars(nre_metric* m, int batch, cudaStream_t st);
bool cg_any_active(const nre_metric* m, int batch);
int cg_report(const nre_metric* m, int batch, double rtol, int maxiter, int* iters_out, double* relres_out,
              const char* what);
// Recompute the metric's expansion-point data (w, amplitude state, per-pixel
// tables) at a new xi_p (device, [latent]) in the buffers it already owns.
int metric_relinearize(nre_metric* m, const void* xi_p, cudaStream_t st);
}  // namespace nre
