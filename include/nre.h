/*
 * nre.h - C ABI of the GB300 metric-vector-product / CG-sampling library
 * (NIFTy.re hot path, arXiv:2402.16683).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every call returns an int status (NRE_OK = 0 or one of NRE_E*); on error
 *   nre_last_error() returns a thread-local message.  No C++ exception crosses
 *   the ABI.  Invalid arguments are rejected before any work is enqueued.
 * - Array arguments named `xi`, `v`, `s`, ... are DEVICE pointers to contiguous
 *   C-order arrays of the plan's dtype (NRE_F32: float, NRE_F64: double),
 *   16-byte aligned.  Arguments documented as "host" are host pointers.
 * - A batch of latent vectors is [batch][stride] with `stride` from
 *   *_latent_layout(); entries stride[latent_size:] are padding that the library
 *   neither reads nor writes.  A batch of position-space fields is [batch][N].
 * - The caller owns every buffer it passes; the library keeps no caller pointer
 *   after a call returns (serving: until the request is polled complete).
 *   Plans own their device workspaces and constant tables; free them with the
 *   matching *_destroy.
 * - Work is enqueued on the given cudaStream_t (NULL = legacy default stream) in
 *   stream order, without host synchronisation, except where a call documents a
 *   synchronisation (cg_solve's host scalars, serving).
 * - A plan may be used by one host thread at a time.
 */
#ifndef NRE_H
#define NRE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *nre_stream_t; /* == cudaStream_t */

/* ------------------------------------------------------------------ status */
enum {
  NRE_OK = 0,
  NRE_EINVAL = 1,    /* bad argument (null pointer, size, dtype, layout)       */
  NRE_ENOMEM = 2,    /* device or host allocation failed                       */
  NRE_ECUDA = 3,     /* a CUDA call failed (message holds cudaGetErrorString)  */
  NRE_ENOTCONV = 4,  /* cg_solve: some system missed rtol within maxiter       */
  NRE_ETIMEDOUT = 5, /* a bounded device-side wait gave up                     */
  NRE_EBUSY = 6,     /* serving: request can never fit the HBM budget          */
  NRE_EAGAIN = 7     /* serving: request still pending                         */
};

enum { NRE_F32 = 0, NRE_F64 = 1 };

/* Thread-local message of the last failing call on this thread ("" if none). */
const char *nre_last_error(void);
/* Library ABI version (major * 10000 + minor * 100 + patch). */
int nre_version(void);

/* ============================================================ correlated field
 * Sec. "Gaussian Processes": s = FT o sqrt(P) o xi on a regular periodic grid
 * (the example uses unit total volume, distances = 1/d).  Reading used here:
 * FT is the unnormalised multi-dimensional Hartley transform
 *     H[z]_k = sum_x z_x cas(2 pi sum_d k_d x_d / N_d),  cas = cos + sin,
 * and the model (log-field, before any response) is
 *     cf(xi) = offset_mean + H(A_full * xi_field),
 * where A_full[k] = A(|k|) for k != 0 and A_full[0] = offset_std (the zero mode
 * of xi_field is the offset excitation).  k_d = m_d / (N_d dx_d) with the folded
 * index m_d (Nyquist folded to +N_d/2).
 *
 * Amplitude kinds:
 *  NRE_AMP_ARRAY         A_full given per pixel (host array, harmonic C order,
 *                        entry 0 is the zero mode); no hyper-parameters.
 *  NRE_AMP_MATERN_FIXED  A_full[k] = (1 + (|k|/k0)^2)^-gamma for k != 0,
 *                        scaled so that sum_{k!=0} A^2 = variance;
 *                        A_full[0] = zero_mode; no hyper-parameters.
 *  NRE_AMP_POWER_MODEL   the non-parametric power-spectrum model of Sec.
 *                        "Gaussian Processes" (add_fluctuations: fluctuations,
 *                        loglogavgslope, flexibility, asperity; offset (mean,
 *                        std)): log-normal / normal hyper-parameters, an
 *                        integrated Wiener process on n_bins log-|k| bins,
 *                        normalised to total variance theta_fluct^2.  Computed
 *                        in FP64 for both dtypes.
 *  NRE_AMP_MATERN_MODEL  the parametric Matern kernel the same section names
 *                        beside the non-parametric one: on the same n_bins
 *                        log-|k| bins, a_b = (1 + (k_b / theta_cutoff)^2)^
 *                        (theta_slope / 4) at the bin-centre wavenumbers
 *                        k_b = exp(l_b), A_b = theta_scale a_b /
 *                        sqrt(sum_b n_b a_b^2); theta_scale, theta_cutoff
 *                        log-normal with the given (mean, std) of the variable,
 *                        theta_slope (the power spectrum's log-log slope above
 *                        the cutoff) normal; A_full[0] = offset_std.  FP64.
 *
 * Latent layout of one sample (float/double):
 *   [0, N)                         xi_field, harmonic C order
 *   [N, N + n_hyper)               POWER_MODEL: xi_fluct, xi_slope,
 *                                  xi_flex, xi_asp, xi1[n_bins-1], xi2[n_bins-1];
 *                                  MATERN_MODEL: xi_scale, xi_cutoff, xi_slope
 *   [latent_size, stride)          padding (stride is a multiple of 64)
 */
enum { NRE_AMP_ARRAY = 0, NRE_AMP_MATERN_FIXED = 1, NRE_AMP_POWER_MODEL = 2, NRE_AMP_MATERN_MODEL = 3 };

typedef struct {
  int kind;                 /* NRE_AMP_*                                      */
  const double *amp_array;  /* ARRAY: host, N values (copied at create)       */
  double k0, gamma, variance, zero_mode;            /* MATERN_FIXED           */
  double fluct_mean, fluct_std, slope_mean, slope_std;   /* POWER_MODEL       */
  double flex_mean, flex_std, asp_mean, asp_std;         /* POWER_MODEL       */
  double offset_mean;       /* added to cf in position space (all kinds)      */
  double offset_std;        /* POWER_ / MATERN_MODEL: A_full[0]                */
  int n_bins;               /* POWER_ / MATERN_MODEL: log-|k| bins (2..1024)  */
  double scale_mean, scale_std, cutoff_mean, cutoff_std;  /* MATERN_MODEL      */
  double lls_mean, lls_std; /* MATERN_MODEL: log-log slope of the power        */
} nre_cf_amp_params;

typedef struct nre_cf_plan nre_cf_plan;

/* Create a correlated-field plan.  ndim in 1..3; every shape[d] a power of two
 * in [4, 4096] (shapes in [4, 4096]); spacing[d] > 0 with the same total
 * length N_d * spacing[d] on every axis (isotropic |k|).  dtype NRE_F32 or
 * NRE_F64.  Allocates the plan's constant tables on the current device. */
int cf_create(nre_cf_plan **plan, int ndim, const int64_t *shape,
              const double *spacing, const nre_cf_amp_params *amp, int dtype);
int cf_destroy(nre_cf_plan *plan);
/* N (pixels), n_hyper, latent_size = N + n_hyper and the per-sample stride. */
int cf_latent_layout(const nre_cf_plan *plan, int64_t *n_field, int64_t *n_hyper,
                     int64_t *latent_size, int64_t *stride);
/* Back-compatible short form: latent_size only. */
int cf_latent_size(const nre_cf_plan *plan, int64_t *latent_size);

/* s[b] = cf(xi[b]) for b < batch.  xi: [batch][stride], s: [batch][N]. */
int cf_forward(nre_cf_plan *plan, const void *xi, void *s, int batch,
               nre_stream_t stream);
/* jv[b] = (d cf / d xi at xi_p[b]) v[b].  xi_p, v: [batch][stride]; jv: [batch][N]. */
int cf_jvp(nre_cf_plan *plan, const void *xi_p, const void *v, void *jv,
           int batch, nre_stream_t stream);
/* g[b] = (d cf / d xi at xi_p[b])^T ct[b].  ct: [batch][N]; g: [batch][stride]. */
int cf_vjp(nre_cf_plan *plan, const void *xi_p, const void *ct, void *g,
           int batch, nre_stream_t stream);

/* cf_forward without any device allocation (the paper has no counterpart: this
 * is an interface for callers that cannot allocate).  cf_forward may grow the
 * plan's workspaces with cudaMalloc, which can synchronise the device and take
 * unpredictable time, and some host runtimes hand out device memory only
 * through their own pool; this variant instead keeps the transform's
 * intermediates (and the amplitude-model state) in one fixed 16 MiB device
 * array that every GPU loading the library holds until the process exits.
 * Same arguments and results as cf_forward.  Returns NRE_EINVAL, before any
 * work is enqueued, if `batch` needs more than 16 MiB of intermediates (about
 * batch * N * sizeof(dtype) per intermediate: one for 2-D grids, two for 3-D).
 * The first call on a device looks up the array's device address (with that
 * device current), so make that first call before any stream capture.  The
 * address is kept per device ordinal for the life of the process: call from
 * the device's primary context (the runtime API's default), and not after a
 * cudaDeviceReset, which would leave the kept address stale.  All calls share
 * the array: calls that overlap on the GPU (other streams, or unordered host
 * threads) race on it. */
int cf_forward_noalloc(nre_cf_plan *plan, const void *xi, void *s, int batch,
                       nre_stream_t stream);

/* Host-only helper (no GPU needed): log-|k| bin of every harmonic pixel as the
 * POWER_MODEL uses it (-1 at k = 0), C order, into host array out[N]. */
int cf_bin_map(int ndim, const int64_t *shape, const double *spacing,
               int n_bins, int32_t *out);

/* ===================================================================== ICR
 * Sec. "Gaussian Processes", ICR paragraph: iterative charted refinement, a GP
 * on a deformed space refined coarse-to-fine from nearest neighbours.  Reading
 * used here: a 2-D log-radial chart, level l with n_l = n0 2^l points per axis
 * at u = (i+1/2)/n_l, v = (j+1/2)/n_l, r = r_min (r_max/r_min)^u, phi = 2 pi v;
 * Matern-3/2 kernel (rho, var); level 0 is s_0 = chol(K0) xi_0; each coarse
 * pixel's 3x3 neighbourhood (radial window clamped to the chart, angular axis
 * periodic) predicts its 2x2 children with R = K_fc K_cc^-1 and adds
 * chol(K_ff - R K_cf) xi_children.  Matrices are assembled in FP64 on the host.
 * Latent layout: xi_0, ..., xi_L (each n_l x n_l, C order), then padding to
 * `stride`.  Output: the finest level, n_L x n_L.
 */
/* ndim 0 or 2: the 2-D log-radial chart above.  ndim 3: a spherical
 * log-radial chart (a reading of the paper's 3-D setting): level l has
 * n_l = n0 2^l points per axis at (u, v, t) = ((i,j,k) + 1/2) / n_l, radius
 * r = r_min (r_max/r_min)^u, polar angle pi v, azimuth 2 pi t; each coarse
 * voxel's 3x3x3 neighbourhood (radial and polar windows clamped to the chart,
 * azimuth periodic, order 9a + 3b + c) predicts its 2x2x2 children (order
 * 4a + 2b + c) with R = K_fc K_cc^-1 (8 x 27) and chol(K_ff - R K_cf), per
 * (level, radial row, polar row); level 0 is chol(K0) over the n0^3 points.
 * Latent: xi_0, ..., xi_L, each n_l^3 in C order; output the finest level.
 * 3-D limits: n0 in [3, 8], n0 2^n_levels <= 512. */
typedef struct { int n0; double r_min, r_max; int ndim; } icr_chart_params;
typedef struct { double rho, var; } icr_kernel_params;
typedef struct nre_icr_plan nre_icr_plan;

/* n0 even in [4, 64], n_levels in [1, 10] refinements, n0 * 2^n_levels <= 4096. */
int icr_create(nre_icr_plan **plan, const icr_chart_params *chart,
               const icr_kernel_params *kernel, int n_levels, int dtype);
int icr_destroy(nre_icr_plan *plan);
int icr_latent_layout(const nre_icr_plan *plan, int64_t *n_out,
                      int64_t *latent_size, int64_t *stride);
/* s[b] = ICR(xi[b]); xi: [batch][stride], s: [batch][n_L * n_L].  Calls of two
 * or more samples run as two half batches on `stream` and on a second stream
 * the plan creates on first use (never during a stream capture), forked and
 * joined by events: the work stays ordered on `stream`. */
int icr_forward(nre_icr_plan *plan, const void *xi, void *s, int batch,
                nre_stream_t stream);
/* The ICR map is linear: jv = ICR(v) (xi_p is accepted for symmetry, unused). */
int icr_jvp(nre_icr_plan *plan, const void *xi_p, const void *v, void *jv,
            int batch, nre_stream_t stream);
/* g[b] = ICR^T ct[b]; ct: [batch][n_L^2], g: [batch][stride]. */
int icr_vjp(nre_icr_plan *plan, const void *xi_p, const void *ct, void *g,
            int batch, nre_stream_t stream);

/* ============================================================== likelihood
 * Sec. "Building Up Complex Models": Poissonian(data).amend(forward) with
 * forward = exp(cf); Sec. "Performance": N^-1 is the Fisher metric of the
 * likelihood.  Folded Fisher weights w at the expansion point (data never enter
 * the metric):
 *   NRE_LIK_GAUSS, NRE_RESP_EXP:       w = mask * exp(cf_p)^2 / sigma^2
 *   NRE_LIK_GAUSS, NRE_RESP_IDENTITY:  w = mask / sigma^2
 *   NRE_LIK_POISSON (rate = scale * exp(cf)):  w = scale * exp(cf_p)
 */
enum { NRE_LIK_GAUSS = 0, NRE_LIK_POISSON = 1 };
enum { NRE_RESP_EXP = 0, NRE_RESP_IDENTITY = 1 };
typedef struct nre_lik nre_lik;

/* mask_host: NULL (every pixel observed) or host array of n_data values in
 * {0, 1} (copied).  sigma_or_scale: noise std (GAUSS) or rate scale (POISSON). */
int lik_create(nre_lik **lik, int kind, int response, const double *mask_host,
               int64_t n_data, double sigma_or_scale);
int lik_destroy(nre_lik *lik);

/* ================================================================= metric
 * Sec. "Performance": M_p = F_p + 1 with F_p = J^T N^-1 J, the benchmarked
 * operator that dominates a VI minimisation.  metric_create linearises the
 * model at xi_p (one latent vector, device) and precomputes w(p), A(p) and the
 * amplitude linearisation; it owns copies of everything it needs and
 * workspaces for up to max_batch tangents.  model_plan must outlive it.
 */
enum { NRE_MODEL_CF = 0, NRE_MODEL_ICR = 1 };
typedef struct nre_metric nre_metric;

int metric_create(nre_metric **m, int model_kind, void *model_plan,
                  const nre_lik *lik, const void *xi_p, int max_batch,
                  nre_stream_t stream);
int metric_destroy(nre_metric *m);
/* out[b] = v[b] + J^T (w * J v[b]), v and out [batch][stride], batch <= max_batch.
 * out may not alias v.  A product of two or more samples on a 2-D / 3-D grid
 * runs its two half batches on `stream` and on a second stream the metric
 * owns, forked from and joined back into `stream` by events: the call's work
 * stays ordered on `stream` (and is captured whole into a CUDA graph). */
int metric_apply(nre_metric *m, const void *v, void *out, int batch,
                 nre_stream_t stream);

/* Sec. "Variational Inference": MGVI samples N(p, M_p^-1).  Right-hand side
 * with covariance M_p:  b = xi_prime + J^T (sqrt(w) * eta).
 * xi_prime, b: [batch][stride]; eta: [batch][N data].  The sample pair is
 * p +/- M_p^-1 b. */
int mgvi_rhs(nre_metric *m, const void *xi_prime, const void *eta, void *b,
             int batch, nre_stream_t stream);

/* Sec. "Variational Inference" (draw_linear_kwargs, cg_kwargs maxiter): solve
 * M_p x[b] = b[b] for every b < batch by conjugate gradients, x_0 = 0, with
 * FP64 inner products and alpha/beta.  A system stops (its x frozen) once
 * ||r|| <= rtol ||b|| (recursive residual) or after maxiter iterations; rtol = 0
 * runs exactly maxiter iterations unless a residual becomes exactly zero (the
 * system is then solved and stops, as the rtol test would at any rtol).  iters_out[batch], relres_out[batch] are
 * HOST arrays (may be NULL), written after a synchronisation of `stream`.
 * Returns NRE_ENOTCONV if rtol > 0 and some system missed it. */
int cg_solve(nre_metric *m, const void *b, void *x, int batch, double rtol,
             int maxiter, int *iters_out, double *relres_out,
             nre_stream_t stream);

/* Sec. "Variational Inference" (the linear draw's CG tolerance), solved to a
 * TRUE relative residual: x (FP64, [batch][stride]) with
 *     ||b - M_hi x|| <= rtol ||b||  for every system,
 * by residual correction: x_0 = 0; r_k = b - M_hi x_k in FP64; the inner CG of
 * cg_solve on m_lo solves M_lo d = r_k to inner_rtol (recursive residual,
 * inner_maxiter iterations at most, m_lo's preconditioner); x_{k+1} = x_k + d.
 * m_hi is an FP64 metric and m_lo a metric of either dtype, both created at the
 * same expansion point for the same model (same latent layout); the product of
 * m_hi decides the residual, so an FP32 m_lo reaches residuals below its own
 * operator error.  b: FP64 [batch][stride] (device); x: FP64 output.  At most
 * max_outer correction passes (each one FP64 product; the residual of
 * x_0 = 0 is b itself).  Systems that reach rtol are frozen.  HOST outputs
 * (may be NULL): iters_out[batch] = inner CG iterations summed over the
 * passes, relres_out[batch] = final true relative residuals, *outer_out =
 * passes taken.  Synchronises `stream` once per pass.  Returns NRE_ENOTCONV if
 * some system is above rtol after max_outer passes; NRE_EINVAL for a non-FP64
 * m_hi, different layouts, rtol <= 0 or inner_rtol outside (0, 1). */
int cg_solve_refined(nre_metric *m_lo, nre_metric *m_hi, const void *b, void *x,
                     int batch, double rtol, int max_outer, double inner_rtol,
                     int inner_maxiter, int *iters_out, double *relres_out,
                     int *outer_out, nre_stream_t stream);

/* Sec. "Variational Inference": the geoVI nonlinear update of sample
 * residuals (the example's minimiser "SN": xtol, maxiter = 5).  Reading used
 * here: with t the likelihood's standardising transform (Gaussian
 * t = sqrt(mask) R(cf) / sigma, Poisson t = 2 sqrt(lambda)) and J_p the
 * Jacobian of xi -> t(cf(xi)) at the metric's expansion point p, each residual
 * delta[b] solves
 *     F(delta) = delta + J_p^T [t(cf(p + delta)) - t(cf(p))] - b = 0
 * by Newton iterations delta <- delta - M_p^-1 F(delta) (cg_solve on m with its
 * preconditioner, to cg_rtol / cg_maxiter), until mean_i |step_i| <= xtol for
 * every system or maxiter iterations.  delta: [batch][stride], on entry the
 * starting residuals (usually the linear ones, M_p^-1 b), on exit the updated
 * ones; b: [batch][stride] (for the antithetic partner pass -b).  HOST outputs
 * (may be NULL): iters_out[batch] (first iteration whose step met xtol, else
 * the iterations run), step_out[batch] (the last mean |step|).  m must be a
 * correlated-field metric. */
int geovi_update(nre_metric *m, const void *b, void *delta, int batch,
                 double xtol, int maxiter, double cg_rtol, int cg_maxiter,
                 int *iters_out, double *step_out, nre_stream_t stream);

/* ============================================================ KL minimisation
 * Sec. "Variational Inference": MGVI alternates between drawing samples and
 * minimising the KL divergence; the example's KL minimiser "M" is a Newton-CG
 * (kl_kwargs: xtol, maxiter = 35).  Reading used here, for a correlated-field
 * plan, a likelihood and its data:
 *   samples xi_s = xi_bar + delta_s (s < n_samples) with the residual samples
 *   delta_s held fixed (e.g. the antithetic pairs +-M^-1 b of the linear draw);
 *   E(xi_bar) = (1/S) sum_s [NLL(d | cf(xi_s)) + |xi_s|^2 / 2] with
 *     Poisson NLL = sum lambda - d ln lambda (lambda = scale exp(cf)),
 *     Gaussian NLL = sum mask (d - R(cf))^2 / (2 sigma^2);
 *   grad E = (1/S) sum_s [xi_s + J_s^T dNLL/dcf(xi_s)];
 *   Newton curvature: Mbar = I + (1/S) sum_s J_s^T W_s J_s (Fisher weights at
 *   each xi_s);
 *   one Newton-CG step: D = -Mbar^-1 grad E by cg_solve on Mbar, backtracking
 *   line search (alpha = 1, halved while E does not decrease, at most 30
 *   times; no decrease: the position stays and the step is 0), xi_bar +=
 *   alpha D;  kl_minimize stops once mean_i |alpha D_i| <= xtol or after
 *   maxiter steps.
 * Energies are FP64 sums; vectors are in the plan's dtype.
 */
typedef struct nre_kl nre_kl;
/* data: HOST doubles [n_data = N] (counts or observations, harmonic grid order
 * of the model output); deltas: DEVICE [n_samples][stride] in the plan dtype
 * (copied).  The plan and likelihood must outlive the KL object. */
int kl_create(nre_kl **kl, nre_cf_plan *plan, const nre_lik *lik,
              const double *data, int64_t n_data, const void *deltas,
              int n_samples, nre_stream_t stream);
int kl_destroy(nre_kl *kl);
/* Move to xi_bar (device [stride]): the points, their Fisher weights and
 * amplitude states, the energy (*energy, host, may be NULL) and the gradient. */
int kl_set_position(nre_kl *kl, const void *xi_bar, double *energy,
                    nre_stream_t stream);
/* Energy (host) and gradient (device [stride], may be NULL) at the position. */
int kl_energy_gradient(nre_kl *kl, double *energy, void *grad,
                       nre_stream_t stream);
/* Energy (host) at xi (device [stride]); the position does not change. */
int kl_energy_at(nre_kl *kl, const void *xi, double *energy,
                 nre_stream_t stream);
/* Mbar at the position as a metric object for metric_apply / cg_solve
 * (max_batch 1, no preconditioner, no mgvi_rhs).  Owned by the KL object:
 * metric_destroy refuses it. */
int kl_metric(nre_kl *kl, nre_metric **metric);
/* Copy of the position (device [stride]). */
int kl_position(nre_kl *kl, void *xi_bar, nre_stream_t stream);
/* One Newton-CG step (inner CG to cg_rtol / cg_maxiter); host outputs (may be
 * NULL): mean |alpha D|, the new energy, the inner CG iterations. */
int kl_newton_step(nre_kl *kl, double cg_rtol, int cg_maxiter,
                   double *mean_abs_step, double *energy, int *cg_iters,
                   nre_stream_t stream);
/* Newton-CG steps until mean |step| <= xtol or maxiter steps. */
int kl_minimize(nre_kl *kl, double xtol, int maxiter, double cg_rtol,
                int cg_maxiter, int *iters, double *energy,
                nre_stream_t stream);

/* ================================================================ tracing
 * Launch accounting for measurement tools.  nre_launch_count() counts every
 * kernel launch the library has issued in this process.  While tracing is
 * enabled (nre_prof_enable(1)) each launch is also bracketed by CUDA events on
 * its stream and tagged with its algorithmic bytes (unique bytes of its global
 * inputs and outputs); nre_prof_report() synchronises the device and writes a
 * JSON object {"kernel": [launches, total_ms, bytes], ...} of the traced
 * launches into buf[len] (NRE_EINVAL if too small), then clears the record. */
unsigned long long nre_launch_count(void);
int nre_prof_enable(int on);
int nre_prof_report(char *buf, size_t len);

/* Preconditioner of cg_solve on this metric (default NRE_PRECOND_NONE: textbook
 * CG, whose iterates are those of the unpreconditioned method).
 * NRE_PRECOND_HARMONIC (correlated field only): the exact inverse of the metric
 * with the weight w replaced by its mean w_bar, applied in harmonic
 * coordinates.  With c = N w_bar the field block is diag(D), D_k = 1 + c A_k^2,
 * and the power-spectrum hyper-parameters h couple through the amplitude
 * Jacobian G = dA/dh; the preconditioner solves the block system by the Schur
 * complement S = I + c G^T diag(U) G, U_b = sum_{k in b} xi_p[k]^2 / D_k
 * (n_hyper x n_hyper; formed and inverted on the device in FP64, through the
 * Woodbury identity with an n_bins x n_bins matrix when n_hyper > n_bins;
 * applied in FP32).  It changes the CG iterates but not the solution; the
 * stopping test stays on the unpreconditioned residual ||r|| / ||b||.  Setup
 * only enqueues work on `stream` (no host synchronisation).
 * This is an addition for solves to a tolerance: the paper runs plain CG. */
enum { NRE_PRECOND_NONE = 0, NRE_PRECOND_HARMONIC = 1 };
int metric_set_precond(nre_metric *m, int kind, nre_stream_t stream);

/* Device bytes currently held by the library's own allocations (plans,
 * metrics, CG workspaces, servers), summed over all devices. */
int nre_device_bytes(int64_t *bytes);

/* Kernels that stage tiles or rows with bulk copies (TMA tiles of the column
 * sweeps and the ICR adjoint, whole rows of the row sweeps) wait for them on a
 * shared-memory barrier with an iteration limit (about a second); a wait that
 * runs out makes the kernel skip the rest of its work (the row sweeps: after
 * finishing the current unit group with void results) and counts here, as
 * does a column-sweep CTA whose shared memory is not 1024-byte aligned.  Writes
 * the count of the current device to *count and, if reset != 0, clears it;
 * synchronises the device.  A nonzero count means that some output of an
 * earlier call is incomplete. */
int nre_wait_timeouts(unsigned *count, int reset);
/* Test hook of those bounded waits (the paper has no counterpart): one CTA
 * waits, with an iteration limit of `limit` (1 .. 2^20), on a shared-memory
 * barrier that no copy completes; the wait runs out, the CTA counts one
 * timeout (read with nre_wait_timeouts) and returns.  Enqueued on `stream`. */
int nre_wait_selftest(unsigned limit, nre_stream_t stream);

/* ================================================================ serving
 * A request loop for sampling solves: each request is one expansion point of
 * a correlated-field model (Sec. "Variational Inference": MGVI draws each
 * posterior sample by a CG solve of the metric at the current point) with
 * n_samples right-hand sides solved to a relative residual.  Requests of
 * different grids and likelihoods are served at once: a request is admitted
 * when a slot is free and its device footprint fits the HBM budget (first in,
 * first out), its CG state stays on the device until it converges, every
 * admitted request runs on its own CUDA stream (optionally replaying its CG
 * iterations as a CUDA graph), and the convergence of all of them is polled
 * without blocking.  Nothing here is in the paper: it serves the paper's
 * sampling step to many callers.
 *
 * Threads: serve_create starts prep_threads admission / set-up threads, one
 * CG-launch thread and one completion thread.  serve_submit and serve_poll may be called
 * from any thread.  serve_destroy waits for admitted work, fails queued
 * requests with NRE_EBUSY and joins the threads. */
typedef struct nre_server nre_server;

typedef struct {
  uint64_t hbm_budget_bytes; /* device bytes the server may hold; 0: half of
                                the free device memory at create            */
  int max_slots;             /* requests on the device at once (1..256)     */
  int dtype;                 /* NRE_F32 or NRE_F64 for every solve          */
  int chunk_iters;           /* CG iterations between convergence polls
                                (0: 8)                                      */
  int use_graphs;            /* 1: capture each slot's chunk of iterations
                                once as a CUDA graph and replay it          */
  int prep_threads;          /* admission / set-up threads (0: 8)           */
} nre_serve_cfg;

typedef struct {
  int ndim;                  /* 1..3                                        */
  int64_t shape[3];          /* powers of two in [8, 4096]; spacing 1/shape */
  nre_cf_amp_params amp;     /* amplitude model (POWER_MODEL or MATERN_FIXED;
                                copied at submit)                           */
  int lik_kind;              /* NRE_LIK_GAUSS (every pixel observed, sigma)
                                or NRE_LIK_POISSON (rate scale exp(cf))    */
  int response;              /* Gaussian: NRE_RESP_EXP or NRE_RESP_IDENTITY;
                                Poisson: NRE_RESP_EXP                       */
  double sigma_or_scale;
  int precond;               /* NRE_PRECOND_* of the solves                 */
  int n_samples;             /* right-hand sides, 1..64                     */
  double rtol;               /* > 0: stop at ||r|| <= rtol ||b||            */
  int maxiter;               /* >= 1                                        */
  /* HOST arrays in the server's dtype, C order, latent = cf_latent_size of
   * the grid.  They are read after serve_submit returns, up to the moment the
   * request starts, and x_out is written just before it completes: all must
   * stay valid until serve_poll has returned NRE_OK for the request.  Page-
   * locked memory makes the copies asynchronous. */
  const void *xi_p;          /* [latent] expansion point                    */
  const void *b;             /* [n_samples][latent] right-hand sides, or the
                                latent draws xi' when eta is given          */
  const void *eta;           /* NULL, or [n_samples][N] data-space draws:
                                the right-hand sides become the MGVI
                                b = xi' + J^T (sqrt(w) eta)                 */
  void *x_out;               /* [n_samples][latent] solutions (unused, may
                                be NULL, when refine > 0)                   */
  /* Residual correction to a TRUE relative residual (FP32 servers only; see
   * cg_solve_refined): refine > 0 allows that many passes after the first
   * solve.  The slot object then also holds an FP64 plan and metric at the
   * same expansion point; each pass takes the FP64 residual b - M64 x and,
   * while a system is above rtol, solves for its correction with the FP32
   * CG to a relative 1e-2.  x64_out: HOST doubles [n_samples][latent], the
   * FP64 solutions; the result's relres are the true residuals and iters
   * the CG iterations of all passes. */
  int refine;
  void *x64_out;
} nre_serve_req;

typedef struct {
  int status;                /* NRE_OK, NRE_ENOTCONV or the error of the solve */
  int iters[64];             /* CG iterations per sample                    */
  double relres[64];         /* recursive ||r|| / ||b|| per sample (refine:
                                the true FP64 residual)                     */
  double t_submit, t_start, t_done; /* CLOCK_MONOTONIC seconds: submit,
                                admission, result copied to x_out           */
  uint64_t device_bytes;     /* footprint charged against the budget        */
  char error[192];           /* message when status != NRE_OK               */
} nre_serve_result;

typedef struct {
  uint64_t budget, reserved, peak_reserved; /* bytes (reserved includes idle
                                slot objects kept for reuse)                */
  int active, queued, idle_objects;
  uint64_t completed, reused, created, evicted, graph_replays, chunks;
} nre_serve_stats;

int serve_create(nre_server **srv, const nre_serve_cfg *cfg);
/* Queues a request and returns its id.  NRE_EINVAL for a malformed request,
 * NRE_EBUSY if its footprint exceeds the whole budget (it could never run). */
int serve_submit(nre_server *srv, const nre_serve_req *req, uint64_t *id);
/* Waits up to timeout_ms (0: do not wait, < 0: forever) for request id.
 * NRE_OK: done, *res filled and the id released; NRE_EAGAIN: still pending;
 * NRE_EINVAL: unknown or already collected id. */
int serve_poll(nre_server *srv, uint64_t id, nre_serve_result *res, int timeout_ms);
/* Device bytes a request would be charged (its footprint estimate). */
int serve_footprint(const nre_serve_req *req, int dtype, uint64_t *bytes);
int serve_stats(nre_server *srv, nre_serve_stats *st);
int serve_destroy(nre_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* NRE_H */
