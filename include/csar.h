/*
 * csar.h — C ABI of libcsar: compressed-sensing SAR imaging with a chirp-scaling
 * approximated observation, on one NVIDIA GB300 (sm_103a).
 *
 * The library computes the iterative thresholding algorithm of the paper's
 * Algorithm 1 / Eq. (25),
 *
 *     X <- T_sigma( X + mu * M( S . (Y - G(X)) ) ),
 *
 * where M is the chirp-scaling focusing operator (Section III-D: the approximated
 * observation may be built from the inverse of the Chirp-Scaling Algorithm), G is
 * its inverse with conjugate phases in reverse order (Section III-C, Eq. (18)),
 * S is the sub-Nyquist sampling mask (the sampling operators Theta_eta, Theta_tau
 * of Eq. (24) generalised to a 2-D mask) and T_sigma is complex soft or half
 * thresholding at sigma = |b|_(K+1), the (K+1)-th largest magnitude of
 * b = X + mu * Delta X (Section IV-B).
 *
 * Conventions (all entry points):
 *  - Arrays are row-major [n_az][n_rg] complex64 (interleaved float re, im):
 *    rows = pulses (azimuth, slow time), columns = range bins (fast time).
 *    Range bin n_rg/2 is the scene-centre range r0; pulse n_az/2 is azimuth time 0.
 *  - The DFT is unnormalised forward, 1/N inverse, on a circular grid with no
 *    padding: M is exactly unitary and G = M^-1 = M^H (Theorem 1).
 *  - Sampling masks are bit-packed row-major: bit j of 32-bit word w is element
 *    32*w + j; a set bit marks a sampled echo element.
 *  - Pointers named *_dev are device pointers (cudaMalloc'd or equivalent) owned
 *    by the caller; the library never frees them.  Pointers named *_host are host
 *    pointers (pageable or pinned).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Entry points taking device pointers only enqueue work on `stream` and return
 *    without synchronising, unless documented otherwise.
 *  - Every entry point returns a csar_status.  Invalid arguments are rejected on
 *    the host before any launch; the message is available from csar_last_error()
 *    (thread-local).  Errors detected on the device (non-finite data, capacity)
 *    are latched in the plan and reported by csar_plan_check() and by the next
 *    synchronising call.
 *  - A plan is not thread-safe: calls on one plan must be serialised by the
 *    caller (they share the plan's workspace).
 */
#ifndef CSAR_H
#define CSAR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CSAR_OK = 0,
  CSAR_E_INVALID = 1,      /* bad argument (null pointer, size, range)                 */
  CSAR_E_UNSUPPORTED = 2,  /* valid but outside what the kernels cover                  */
  CSAR_E_OOM = 3,          /* device allocation failed                                 */
  CSAR_E_CUDA = 4,         /* a CUDA runtime call failed                                */
  CSAR_E_TIMEOUT = 5,      /* a bounded device-side wait expired                        */
  CSAR_E_NONFINITE = 6,    /* NaN or Inf met in the echo or the iterate                 */
  CSAR_E_INTERNAL = 7      /* internal capacity / consistency check failed              */
} csar_status;

/* System parameters (the paper's Table 2 rows: slant range of scene centre R_c,
 * effective velocity V, centre frequency f0 = c / wavelength, PRF, range FM rate
 * K_r = bandwidth / pulse_len, pulse duration, range sampling rate F_r).
 * Zero squint, zero Doppler centroid. */
typedef struct {
  int32_t n_az;        /* N_a: rows (pulses); power of two, 16 .. 8192              */
  int32_t n_rg;        /* N_r: columns (range bins); power of two, 16 .. 8192       */
  double wavelength;   /* lambda [m]                                                 */
  double velocity;     /* effective radar velocity V [m/s]                           */
  double r0;           /* slant range of the scene centre (bin n_rg/2) = R_ref [m]  */
  double prf;          /* pulse repetition frequency [Hz]                            */
  double bandwidth;    /* chirp bandwidth B [Hz] (up-chirp)                          */
  double pulse_len;    /* pulse duration T_p [s]                                     */
  double fs;           /* range sampling rate [Hz]                                   */
  double antenna_len;  /* La [m]; used only by the echo simulator csar_echo_points       */
  double c;            /* speed of light [m/s]; 0 selects 299792458                  */
} csar_params;

typedef struct csar_plan_s* csar_plan;
typedef struct csar_batch_s* csar_batch;

/* csar_plan_create flags: force the column-pass cluster size (CTAs per column tile,
 * 1..16, power of two; 0 = the autotuned or default choice), and/or column-pass CTAs
 * of 4096 complex values (four per SM, half-width tiles) or of 16384 (one per SM,
 * double-width tiles: wider row segments per memory request) instead of 8192 (two per
 * SM).  A configuration that is not built for n_az gives CSAR_E_UNSUPPORTED, and so do
 * both tile flags together. */
#define CSAR_PLAN_COL_CLUSTER(p) ((uint32_t)(p) << 8)
#define CSAR_PLAN_COL_HALF_TILE ((uint32_t)1 << 16)
#define CSAR_PLAN_COL_WIDE_TILE ((uint32_t)1 << 18)
/* csar_plan_create flags: CSAR_PLAN_COL_PERSIST runs the forward, inverse, residue and
 * selection column passes as persistent clusters that walk the column tiles, each
 * tile's block arriving by 2-D tensor copies into a landing buffer while the previous
 * tile is transformed (alone: clusters of n_az/1024 CTAs of 4096 values, n_az >= 1024;
 * with the cluster / tile flags above: that configuration, if built persistent).
 * CSAR_PLAN_COL_NO_PERSIST keeps the per-tile column kernels whatever the default or
 * the autotuner chose.  Results are the same either way; only speed differs. */
#define CSAR_PLAN_COL_PERSIST ((uint32_t)1 << 19)
#define CSAR_PLAN_COL_NO_PERSIST ((uint32_t)1 << 20)
/* csar_plan_create flag: configure the plan exactly as a member of a batch whose passes
 * run as one launch each (csar_batch_create): column passes on 4096 values per CTA with
 * 1 (n_az <= 1024), 2 (n_az = 2048) or 4 (n_az = 4096) CTAs per tile, the first column
 * pass of the sparse iterate always by the clustered FFT (no direct DFT), the default
 * range-pass schedule.  Only for n_az and n_rg in {512, 1024, 2048, 4096}
 * (CSAR_E_UNSUPPORTED otherwise); not with the other CSAR_PLAN_COL_* flags
 * (CSAR_E_INVALID).  A plan made so computes bit for bit what its batch computes for that
 * patch. */
#define CSAR_PLAN_BATCH_MEMBER ((uint32_t)1 << 21)

/* csar_plan_create flag: csar_G / csar_M use the range-Doppler operator pair of the
 * paper's concrete example (Section III-C, Eqs. (14)-(18)) instead of the chirp-scaling
 * one: M = range compression (range FFT, x exp(j pi f_tau^2 / K_r), range IFFT), azimuth
 * FFT, RCMC C (8-tap truncated-sinc interpolation along range to tau + dr, dr =
 * 2 R0 (1/D - 1) fs / c samples, Eq. (16)), x exp(j 4 pi R0 f0 D / c), azimuth IFFT;
 * G = M^H (conjugate filters, D = C^T, reverse order; Theorem 1).  M G is close to,
 * not exactly, the identity (the truncated interpolation is not unitary).  Range
 * compression commutes with the azimuth transforms, so each operator runs as azimuth
 * FFT, one range pass, azimuth IFFT.  csar_ita_step and csar_solve run Algorithm 1 with
 * this pair (the paper's CS-RDA); autofocus and batch entry points reject such a plan
 * (CSAR_E_UNSUPPORTED), and so does plan creation when a row's migration slope
 * 1/D - 1 exceeds 1/2 (D < 2/3). */
#define CSAR_PLAN_RDA ((uint32_t)1 << 17)

enum { CSAR_MU_FIXED = 0, CSAR_MU_NIHT = 1 };
enum { CSAR_THRESH_SOFT = 0, CSAR_THRESH_HALF = 1, CSAR_THRESH_HARD = 2 };

/* Options of the iterative thresholding algorithm (Algorithm 1, Section IV-B). */
typedef struct {
  int64_t K;          /* sparsity: sigma = (K+1)-th largest |b|; K >= n keeps all      */
  int32_t iters;      /* number of iterations I (csar_solve)                           */
  int32_t mu_mode;    /* CSAR_MU_FIXED or CSAR_MU_NIHT (adaptive step)                 */
  float mu;           /* fixed step (CSAR_MU_FIXED); must be > 0                       */
  int32_t thresh;     /* CSAR_THRESH_SOFT (q = 1), CSAR_THRESH_HALF (q = 1/2) or
                         CSAR_THRESH_HARD (q = 0: b kept where |b| > sigma)           */
} csar_opts;

/* Per-iteration diagnostics, host arrays of length >= opts.iters (any may be NULL). */
typedef struct {
  double* resid_sq;   /* ||S . (Y - G(X^(i)))||^2                                       */
  float* mu;          /* step mu_i                                                      */
  float* sigma;       /* lambda_i mu_i = |b|_(K+1)                                      */
  int64_t* nnz;       /* nonzeros of X^(i+1)                                             */
} csar_stats;

/* Create a plan: validates `params`, builds the FP64 phase-coefficient tables of
 * the chirp-scaling functions H1 (chirp scaling), H2 (range compression, SRC and
 * bulk RCMC) and H3 (azimuth matched filter and residual phase) and uploads them,
 * and allocates the plan's device workspace.  `flags`: 0 (the autotuned or default
 * column configuration), the CSAR_PLAN_COL_* flags above, and CSAR_PLAN_RDA.  The plan uses the
 * current CUDA device.  On error *out is set to NULL.  CSAR_E_UNSUPPORTED if the
 * geometry's phase arguments exceed what the on-the-fly phase evaluation covers
 * (|range-linear term| >= 2^22 cycles). */
csar_status csar_plan_create(const csar_params* params, uint32_t flags, csar_plan* out);

/* Destroy a plan (synchronises the device, frees the workspace).  NULL is a no-op. */
csar_status csar_plan_destroy(csar_plan plan);

/* y_dev = G(x_dev): the approximated observation (Section III-C/D, Eq. (18) with
 * chirp-scaling sub-operations): azimuth FFT, x conj(H3), range FFT, x conj(H2),
 * range IFFT, x conj(H1), azimuth IFFT (on a CSAR_PLAN_RDA plan: azimuth FFT,
 * x conj(P_eta), D = C^T, range compression with the conjugate filter, azimuth IFFT).
 * x_dev, y_dev: n_az*n_rg complex64 device arrays; x_dev == y_dev (in place) is
 * allowed; otherwise they must not overlap. */
csar_status csar_G(csar_plan plan, const void* x_dev, void* y_dev, void* stream);

/* x_dev = M(y_dev) = G^H(y_dev): chirp-scaling focusing (Section III-A Eq. (10),
 * Section III-D): azimuth FFT, x H1, range FFT, x H2, range IFFT, x H3, azimuth
 * IFFT (on a CSAR_PLAN_RDA plan: azimuth FFT, range compression, RCMC C, x P_eta,
 * azimuth IFFT).  Same layout and aliasing rules as csar_G. */
csar_status csar_M(csar_plan plan, const void* y_dev, void* x_dev, void* stream);

/* One iteration of Algorithm 1 (Eq. (25)) on device data:
 *   X_dev <- T_sigma(X + mu M(S . (Y - G(X)))).
 * Y_dev: echo, n complex64 (values where the mask bit is clear are ignored).
 * mask_dev: bit-packed sampling mask, n/32 uint32.  X_dev: in/out, n complex64
 * (any number of nonzeros on input; at most K on output).  sigma_dev: optional
 * device float receiving sigma (NULL to skip).  The step is opts->mu (FIXED) or the
 * NIHT step (NIHT; for an all-zero X the support is the top K of |Delta X|). */
csar_status csar_ita_step(csar_plan plan, const void* Y_dev, const uint32_t* mask_dev,
                          void* X_dev, const csar_opts* opts, float* sigma_dev,
                          void* stream);

/* Algorithm 1 from X^(0) = 0 for opts->iters iterations; the K-sparse iterate stays
 * on the device as a (index, value) list between iterations and X_dev (n complex64,
 * output only) receives X^(I).  Each iteration is one CUDA graph launch.  If
 * `stats` is non-NULL the call synchronises `stream` and fills the host arrays. */
csar_status csar_solve(csar_plan plan, const void* Y_dev, const uint32_t* mask_dev,
                       void* X_dev, const csar_opts* opts, const csar_stats* stats,
                       void* stream);

/* csar_solve from HOST buffers: copies Y_host (n complex64) and mask_host (n/32
 * uint32) into plan-owned device buffers, runs csar_solve, copies X^(I) back into
 * X_host (n complex64), and synchronises `stream` before returning. */
csar_status csar_solve_host(csar_plan plan, const void* Y_host, const uint32_t* mask_host,
                            void* X_host, const csar_opts* opts, const csar_stats* stats,
                            void* stream);

/* csar_solve without graphs, with CUDA events recorded on `stream` around every
 * pass: pass_ms[0..5] receive the summed device time of the passes C1 (sparse
 * azimuth FFT), R1 (range pass of G), C2 (residue), R2 (range pass of M), C3
 * (Delta X, histogram, candidates) and the selection + threshold kernels, over
 * opts->iters iterations.  n_pass must be >= 6.  Synchronises `stream`. */
csar_status csar_solve_profile(csar_plan plan, const void* Y_dev, const uint32_t* mask_dev,
                               void* X_dev, const csar_opts* opts, float* pass_ms,
                               int32_t n_pass, void* stream);

/* Non-chirp pulse (Section III-D, second generalisation: the approximated observation
 * applies to any transmitted pulse once the range matched filter's conjugate P_tau^* is
 * replaced by the recorded pulse).  On a CSAR_PLAN_RDA plan, spectrum_host (2 * n_rg
 * floats: re, im of the transmitted pulse's range spectrum S at every range-frequency
 * bin, FFT order: bin j is frequency j fs / n_rg for j < n_rg/2 and (j - n_rg) fs / n_rg
 * above; the pulse's time origin, where its compressed peak falls, at delay 0) replaces
 * the chirp filter from then on: G multiplies the range spectrum by S, M by conj(S), so
 * G = M^H still holds (Theorem 1), while M G = I only for a unit-modulus S.  NULL
 * restores the chirp filter exp(j pi f^2 / K_r).  The table is copied; the call
 * synchronises the device and drops the plan's captured graphs.  CSAR_E_UNSUPPORTED on
 * a chirp-scaling plan (chirp scaling is defined for linear FM pulses only),
 * CSAR_E_INVALID for a non-finite entry. */
csar_status csar_plan_set_pulse(csar_plan plan, const float* spectrum_host);

/* ---- Differentiable autofocus (per-pulse azimuth phase error theta) ----------------
 * Observation A_theta X = S . (exp(j theta_eta) . G(X)) with one real phase theta_eta
 * per echo row (pulse).  Its ITA is Algorithm 1 on the de-rotated echo
 * exp(-j theta_eta) . Y.  Gradients follow dL = Re<grad, dz> for complex z (the
 * torch convention).  The paper does not differentiate the method: these entry points
 * add autofocus on top of it.  theta_dev: n_az floats (radians) on the device. */

/* X^(I) of the theta-observation ITA (csar_solve on exp(-j theta).Y).  With
 * checkpoint != 0 every iterate X^(i+1) (at most K entries), sigma_i and the
 * (K+1)-th element are kept in the plan for csar_af_backward (soft threshold and
 * fixed step only, else CSAR_E_UNSUPPORTED); memory: iters * K * 12 bytes. */
csar_status csar_af_solve(csar_plan plan, const void* Y_dev, const uint32_t* mask_dev,
                          const float* theta_dev, void* X_dev, const csar_opts* opts,
                          int32_t checkpoint, void* stream);

/* L = ||S . (exp(-j theta).Y - G(X))||^2 into *loss_dev (one double), and optionally
 * grad_X = -2 M(r) (n complex64) and dL/dtheta_eta = 2 sum_tau Im(conj(r) exp(-j theta) Y)
 * (n_az floats), r = S . (exp(-j theta).Y - G(X)).  X_dev: dense n complex64. */
csar_status csar_af_loss(csar_plan plan, const void* Y_dev, const uint32_t* mask_dev,
                         const float* theta_dev, const void* X_dev, double* loss_dev,
                         void* grad_X_dev, float* grad_theta_dev, void* stream);

/* Backward through the checkpointed unroll of the last csar_af_solve on this plan:
 * given Xbar_dev, the adjoint of X^(I) (n complex64), ADDS the theta adjoint into
 * theta_bar_dev (n_az floats) and writes the adjoint of X^(0) into X0bar_dev (n
 * complex64; NULL to skip).  Per iteration: the soft-threshold VJP (with the
 * dependence of sigma = |b|_(K+1) on b), G and M of the adjoint, and a row reduction. */
csar_status csar_af_backward(csar_plan plan, const void* Y_dev, const uint32_t* mask_dev,
                             const float* theta_dev, const void* Xbar_dev,
                             float* theta_bar_dev, void* X0bar_dev, void* stream);

/* y_dev = G(x_dev) without any device allocation, for callers that cannot call
 * cudaMalloc (their device memory is owned and handed out by a host framework, or
 * they must not allocate after start-up).  The paper has no counterpart:
 * it is a deployment variant of csar_G.  Same operator, layout and aliasing rules as
 * csar_G, but no plan: the phase coefficients and FFT twiddles that a plan would keep
 * in allocated memory go into one static device array of the library (about 580 KiB
 * on every GPU that loads it, kept until process exit), sized for n_az <= 8192.
 * The first call on a device looks up that array's device address (make that first
 * call before any stream capture).  Every call rewrites the whole table, so nothing
 * needs clearing, but calls that overlap on the GPU (other streams, other threads)
 * share the array and race: serialise them.  Host-side calls are serialised
 * internally.  Enqueues on `stream` (a pageable host-to-device copy of the tables,
 * then the three passes). */
csar_status csar_G_noalloc(const csar_params* params, const void* x_dev, void* y_dev,
                           void* stream);

/* ---- Scene simulator ----------------------------------------------------------- */

/* Raw stripmap echo of point targets on image pixels from the exact observation model
 * (Section V-A: time-domain echoes from the exact slant range), computed on the GPU in
 * FP64 geometry: target k at pixel (rows[k], cols[k]) has azimuth time
 * (rows[k] - N_a/2)/PRF and closest range R_t = c tau_cols[k] / 2, tau_j =
 * 2 r0/c + (j - N_r/2)/fs; its echo at pulse i, bin j is
 *   a_k rect(delay/T_p) rect((eta_i - eta_k)/T_a) exp(-j 4 pi R / lambda + j pi K_r delay^2),
 *   R = sqrt(R_t^2 + V^2 (eta_i - eta_k)^2), delay = tau_j - 2R/c,
 *   T_a = 0.886 lambda R_t / (La V), K_r = bandwidth / pulse_len, windows closed.
 * rows, cols: host int32 arrays of `count` (0 <= count <= 2^24) pixels on the grid;
 * amp: host float array of 2*count (re, im); echo_dev: device [N_a][N_r] complex64,
 * overwritten (accumulate = 0) or added to.  Needs antenna_len > 0.  No plan; the
 * target list is copied into stream-ordered device memory (cudaMallocAsync) and freed
 * after the launch; the host arrays may be reused as soon as the call returns. */
csar_status csar_echo_points(const csar_params* params, const int32_t* rows, const int32_t* cols,
                             const float* amp, int64_t count, void* echo_dev, int32_t accumulate,
                             void* stream);

/* ---- Batches of independent patches (uneven sizes) -------------------------------- */

/* One plan per patch (params[0..n_patches-1], each as for csar_plan_create with
 * `flags`).  When every patch has n_az and n_rg in {512, 1024, 2048, 4096} and `flags`
 * holds no CSAR_PLAN_COL_* flag, the plans are made as batch members
 * (CSAR_PLAN_BATCH_MEMBER) and the batch builds work tables of all patches' row blocks
 * and column-tile groups (device memory, held until csar_batch_destroy).  Not
 * thread-safe; the batch owns the plans. */
csar_status csar_batch_create(const csar_params* params, int32_t n_patches, uint32_t flags,
                              csar_batch* out);
csar_status csar_batch_destroy(csar_batch batch);

/* Algorithm 1 on every patch together from X = 0: per iteration ONE CUDA graph launch
 * on `stream`.  For a batch of members with the fixed step, the graph holds one kernel
 * launch per pass (and per selection kernel) over the work tables of all patches, each
 * patch with its own K_p, sigma and control block; otherwise (NIHT step, other sizes or
 * flags) its parallel branches are the patches' own pass sequences.  Either way patches
 * of different sizes run concurrently.  Y_dev, mask_dev, X_dev: host arrays of per-patch
 * device pointers (layout as csar_solve); K: per-patch sparsity; opts: shared step,
 * threshold and iteration count (opts->K ignored). */
csar_status csar_solve_batched(csar_batch batch, const void* const* Y_dev,
                               const uint32_t* const* mask_dev, void* const* X_dev,
                               const int64_t* K, const csar_opts* opts, void* stream);

/* csar_plan_check on every patch of the batch. */
csar_status csar_batch_check(csar_batch batch);

/* Autotuner: times `iters` ITA iterations on synthetic data for every column-pass
 * configuration available for (n_az, n_rg) and, for rows of 1024 bins and more, both
 * radix schedules of the range passes (32 values per thread: 8192 = 8 x 32 x 32; 16:
 * 2 x 16 x 16 x 16), keeps the fastest for plans created afterwards in this process (and
 * in the file named by CSAR_TUNE_FILE, if set), and returns the column configuration's
 * cluster size in *chosen_cluster.  Every CTA size (half, full and wide tiles) is tried.
 * Synchronises the device; allocates temporaries. */
csar_status csar_autotune(const csar_params* params, int32_t iters, int32_t* chosen_cluster);

/* Self-test of failure detection: runs the bounded wait of the column-pass cluster
 * exchanges on an mbarrier that nothing arrives at, with a limit of limit_ms (1..10000)
 * milliseconds, on the current device (legacy stream; synchronises).  Returns
 * CSAR_E_TIMEOUT when the wait ran out and the kernel returned normally (the expected
 * outcome; the context stays usable), CSAR_E_INTERNAL if the wait completed.  The paper
 * has no counterpart: it checks that no device-side wait of the library can hang. */
csar_status csar_selftest_wait_timeout(int32_t limit_ms);

/* ---- Test hook of the threshold rule ---------------------------------------------
 * Section IV-B sets sigma = |b|_(K+1); the selection finds it as the (K+1)-th largest
 * of the fp32 keys key(b) = bits(|b|^2) over the union of the support and the
 * candidates.  With the record enabled (capacity > 0 entries; 0 disables and frees it),
 * every ITA iteration on the plan (csar_ita_step, csar_solve, csar_solve_profile)
 * overwrites a device record of that union right after the threshold: each element's
 * flat index, b (float re, im) and key exactly as the selection kernels formed them,
 * the union size and the iteration's sigma^2 key, mu and sigma.  Enabling synchronises
 * the device, drops the plan's captured graphs and allocates 16 bytes per entry.
 * csar_debug_selection_read synchronises and copies min(union size, capacity of the
 * record, `capacity`) entries into the host arrays (any may be NULL; b_host holds
 * 2 floats per entry); *count receives the union size.  CSAR_E_INTERNAL if the union
 * was larger than the record. */
csar_status csar_debug_selection_enable(csar_plan plan, int64_t capacity);
csar_status csar_debug_selection_read(csar_plan plan, uint32_t* idx_host, float* b_host,
                                      uint32_t* key_host, int64_t capacity, int64_t* count,
                                      uint32_t* sigma2_key, float* mu, float* sigma);

/* ---- Test hook of the out-of-memory paths (host-side fault injection) ------------
 * After csar_debug_fail_alloc(n) with n > 0, the n-th device allocation the library
 * makes from then on (plans, workspaces grown on demand, host-buffer staging, records)
 * fails as if the device were out of memory, without allocating: the entry point that
 * made it returns CSAR_E_OOM and frees what it had allocated for the call.  n = 0 turns
 * the injection off.  Process-wide; not thread-safe against concurrent allocations.
 * The paper has no counterpart: it lets tests drive every allocation-failure path
 * without touching the GPU's memory state. */
csar_status csar_debug_fail_alloc(int32_t n);

/* Synchronise the plan's device and report (and clear) any latched device-side
 * error of the plan (CSAR_E_NONFINITE, CSAR_E_INTERNAL, CSAR_E_TIMEOUT, ...). */
csar_status csar_plan_check(csar_plan plan);

/* Thread-local description of the last error on this thread ("" if none). */
const char* csar_last_error(void);

/* Library version, as major*10000 + minor*100 + patch. */
int32_t csar_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CSAR_H */
