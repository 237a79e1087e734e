/*
 * wf.h -- C ABI of the GB300 multi-messenger Wiener-filter library (libwf.so).
 *
 * Method: Huffenberger 2017, "Preconditioner-free Wiener filtering with a
 * dense noise matrix" (arXiv:1704.00865).  The Wiener filter
 *     s = (S^-1 + N^-1)^-1 N^-1 d                           (Sec. 1, eq. wiener)
 * is found by the messenger iteration of Sec. 2 (eqs. 2mess_t1 - 2mess_s),
 * generalised to a noise covariance N = N_1f + N_stripe + N_white that is a
 * sum of parts, each diagonal in its own basis (Sec. 2: "each additional
 * piece ... two additional fields"; Appendix A, eq. 2mess_prob):
 *
 *   part "2DF"  isotropic 1/f noise, diagonal in the 2D DFT of the map;
 *   part "RF"   horizontal stripes, diagonal in the row-wise 1D DFT along x;
 *   part "PX"   white noise, diagonal in pixels; infinite at masked pixels
 *               (Sec. 3.2, Sec. 3.3: a mask is infinite noise variance).
 *
 * The signal covariance S is diagonal in the 2D DFT.  Messenger covariances
 * are T_i = lambda * tau_i * I with tau_i = theta_i * (minimum eigenvalue of
 * part i) (Sec. 2, Appendix A), Nbar_i = N_i - tau_i held fixed while the
 * cooling parameter lambda is lowered to 1 (Sec. 2), by a fixed schedule or
 * by the adaptive rule of Sec. 3.3.
 *
 * Maps are real, row-major [ny][nx] float32 (x fastest).  Spectral inputs are
 * eigenvalues (they do not depend on how the DFT is normalised) in the
 * half-spectrum layout [ny][nx/2+1] of a real 2D DFT: row ky in FFT order
 * (0, 1, ..., ny/2, -ny/2+1, ..., -1), column kx = 0..nx/2.  Columns kx = 0
 * and kx = nx/2 must be symmetric in ky (a real covariance); others need not.
 *
 * Memory: every array argument may be a device pointer or a host pointer;
 * the library asks the CUDA runtime which one it is; device memory must
 * belong to the current device (another GPU's memory gives WF_EINVAL, since
 * without peer access a kernel touching it faults).  Host arrays are copied
 * to the plan's device workspace (and s_out back) on the plan's stream.
 * The caller keeps ownership of every array.  All calls are stream-ordered
 * on the plan's stream; calls that return results (wf_solve, wf_run,
 * wf_residual, wf_get_field, wf_fft2) synchronise that stream before they
 * return.  A plan is not thread-safe: use one plan per host thread.
 *
 * Sizes: nx and ny are each a power of two in [32, 4096] or one of 384, 768,
 * 1536 (3 x 2^k: the transforms then take one radix-3 stage).
 *
 * Errors: every function returns WF_OK (0) or one of the codes below;
 * wf_strerror() gives a message.  On error nothing is written to outputs
 * except where stated.
 */
#ifndef WF_H
#define WF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WF_ABI_VERSION 3

#if defined(__GNUC__)
#define WF_API __attribute__((visibility("default")))
#else
#define WF_API
#endif

enum wf_status {
  WF_OK = 0,
  WF_EINVAL = 1,      /* bad size, NULL, NaN/Inf input, asymmetric spectrum   */
  WF_ENOTPD = 2,      /* a covariance eigenvalue <= 0: C, P1f, Pst, pixel_var  */
  WF_ENOCONV = 3,     /* max_iters reached; s_out still holds the last iterate */
  WF_ETIMEOUT = 4,    /* a bounded device wait gave up                          */
  WF_ECUDA = 5,       /* a CUDA runtime call failed                             */
  WF_ENOMEM = 6,      /* device allocation failed                               */
  WF_EUNSUPPORTED = 7, /* size or option this build does not handle           */
  WF_ESTALL = 8       /* the residual stopped falling above the tolerance (the
                         FP32 floor, see stall_checks); s_out holds the last
                         iterate                                               */
};

/* noise parts present (bit mask); WF_PART_WHITE is required */
enum { WF_PART_WHITE = 1, WF_PART_1F = 2, WF_PART_STRIPE = 4 };

/* cooling schedules */
enum { WF_SCHED_FIXED = 0, WF_SCHED_ADAPTIVE = 1 };

/* fields that wf_get_field can return (in pixel space) */
enum {
  WF_FIELD_S = 0,      /* the signal estimate s (eq. 2mess_s)                  */
  WF_FIELD_T_2DF = 1,  /* messenger of the 1/f part (t_0 in eq. 2mess_t0)     */
  WF_FIELD_D_2DF = 2,  /* data-like field next to it (d_0 in eq. 2mess_d0)    */
  WF_FIELD_T_RF = 3,   /* messenger of the stripe part                         */
  WF_FIELD_D_RF = 4    /* data-like field next to it                           */
};

/*
 * Cooling schedule (Sec. 2: T_i -> lambda T_i with Nbar_i fixed).
 * WF_SCHED_FIXED: level j runs iters[j] iterations at lambda = lam[j]
 *   (host arrays, nlevels <= 256); level changes happen at residual
 *   checkpoints; after the last level lambda = 1 until convergence.
 * WF_SCHED_ADAPTIVE (Sec. 3.3): lambda starts at lam0; at each checkpoint,
 *   if the per-iteration relative change of Delta d^T Delta d is below
 *   ratio, lambda <- lambda^expo, and lambda = 1 once it falls below snap.
 *   The paper's values are lam0 = 5e5, ratio = 1e-2, expo = 0.7.
 */
typedef struct {
  int mode;
  const double* lam;
  const int* iters;
  int nlevels;
  double lam0, ratio, expo, snap;
} wf_schedule;

/*
 * Solver parameters (pass NULL to wf_plan_create for the defaults given).
 *  theta[3]        tau_i = theta_i * min eigenvalue of part i, for the parts
 *                  (2DF, RF, PX); defaults 0.9, 0.9, 1.0.  theta < 1 is
 *                  required for interior parts (2DF, RF): at theta = 1 the
 *                  minimum-eigenvalue mode has Nbar = 0 and never moves.
 *  split_f         fraction of min(P1f) moved from the 1/f part to the stripe
 *                  part (a white floor is diagonal in every basis, so N is
 *                  unchanged); default 0.5.
 *  split_fp        fraction of min(P1f) moved from the 1/f part to the white
 *                  part (raises tau_PX, which sets how fast masked and noisy
 *                  pixels converge); default 0.5.  split_f + split_fp <= 1
 *                  (< 1 for the plain sweep).
 *  split_w         fraction of min(pixel_var) moved from the white part to
 *                  the stripe part; default 0.
 *  tol_u_scale     the stop test asks ||Delta d_u||/||d_u|| <= tol * tol_u_scale
 *                  and ||(S^-1 s)_m|| / ||S^-1 s|| <= tol; default 1.
 *  merge_2df       1: update s, t_2DF and d_2DF jointly given t_RF (the
 *                  1/f part and S share the 2D Fourier basis, Appendix A:
 *                  t_0 is marginalised and s = (S^-1 + N_0^-1)^-1 N_0^-1 d_0);
 *                  the iteration then needs no tau for the 1/f part and
 *                  split_f may be 1.  0: the plain sweep.  Default 1.
 *  refine          defect-correction solves wf_solve adds after the first
 *                  (default 0, at most 32).  Each takes the residual of the
 *                  accumulated s (Sec. 2): Delta d_u = [(I + N S^-1) s - d] on unmasked
 *                  pixels and j = (S^-1 s) on masked pixels, solves the same
 *                  filter with Delta d_u as data and j as a source,
 *                  (S^-1 + N^-1) e = N^-1 Delta d + j, and subtracts e =
 *                  s - s_exact.  Each pass removes most of the error the
 *                  previous solve left (FP32 stagnation and slow modes).
 *                  Only wf_solve refines.
 *  refine_tol_scale the correction solves stop at tol * refine_tol_scale
 *                  (their data is the previous residual, so percent-level
 *                  accuracy already cuts the error by that factor); default
 *                  100.
 *  refine_max_iters iteration cap of each correction solve; 0 (default):
 *                  max_iters.  A correction that reaches a nonzero cap does
 *                  not make wf_solve return WF_ENOCONV.
 *  stall_checks    at lambda = 1, stop the solve (WF_ESTALL) once this many
 *                  residual checkpoints in a row bring no 1% drop of
 *                  ||Delta d_u||^2: an FP32 iteration stalls once its slow
 *                  links move their fields by less than one unit in the last
 *                  place.  With refine > 0 a stalled first solve goes on to
 *                  the corrections, and wf_solve then reports WF_OK when the
 *                  refined s passes the stop test.  0 (default): never.
 *  autotune        1 (default): the first problem a plan loads times both
 *                  compiled shapes of each pass (values per thread) on the
 *                  plan's buffers and keeps the faster, cached per device and
 *                  map shape for the process (see wf_plan_shapes); 0: the
 *                  first shapes; 2: the second shapes, untimed.  The shape
 *                  changes only the rounding order.
 *  refine_extra    further corrections after the refine ones, each run only
 *                  while the refined s fails the stop test (tol > 0): a
 *                  harder map gets the sweeps it needs without raising the
 *                  budget of every map; default 0, at most 32.
 *  refine_lam1_iters with a cap and a fixed schedule, each correction runs
 *                  the schedule's levels (lambda > 1) for at most
 *                  refine_max_iters - refine_lam1_iters sweeps and then
 *                  lambda = 1 to the cap, so that it ends on the unbiased
 *                  fixed point; default 0.
 *  residual_every  R: the residual and the lambda rule run every R
 *                  iterations; default 10.  With a fixed schedule the
 *                  residual is evaluated only where something uses it: at
 *                  lambda = 1 (stop and stall tests) and at the checkpoint
 *                  that reaches max_iters (the values reported); the other
 *                  checkpoints only advance the schedule.
 *  max_iters       default 200000.
 *  check_every     residual checkpoints between host polls of the done flag
 *                  (latency of the stop test versus host round trips);
 *                  default 8.
 *  dft_precision   arithmetic of the radix-16 stages of the column transforms
 *                  in the iteration's column pass and in wf_fft2: 0 (default)
 *                  FP32 on the CUDA cores; 1 on the tensor cores as DFT
 *                  matrix products with both factors split into two TF32
 *                  parts (hi*hi + hi*lo + lo*hi, FP32 accumulation: about
 *                  FP32 accuracy); 2 one TF32 product (relative error about
 *                  2^-11 per stage).  The residual, the stop test and the
 *                  defect corrections keep FP32 transforms and FP64 sums, so
 *                  they judge a solve made with either.  Nonzero values need
 *                  ny in {512, 1024, 2048, 4096} and merge_2df = 1
 *                  (WF_EUNSUPPORTED otherwise); the column shape is then the
 *                  16-value one.
 *  sweep_kernel    how sweeps are launched: 0 (default) a row-pass and a
 *                  column-pass launch per sweep; 1 one cooperative launch
 *                  per residual_every sweeps, the passes separated by grid
 *                  barriers, every CTA keeping the tables and fields of its
 *                  own rows and column tile in shared memory across sweeps
 *                  (1024 x 1024 maps with a stripe part, the merged 2DF block
 *                  or no 1/f part, dft_precision 0, a GPU with at least 128
 *                  SMs; WF_EUNSUPPORTED from wf_plan_create otherwise).  The
 *                  arithmetic is that of the two launches, with 8 values per
 *                  thread in both transforms.  On a GB300 the one-launch
 *                  form measured slower at 1024^2 (its two grid barriers cost
 *                  more than the launch boundaries they replace), so it is
 *                  not the default.
 *  trace           per-checkpoint trace of the iteration (wf_get_trace): 0
 *                  (default) off; 1 lambda and the two residual terms at every
 *                  checkpoint (a fixed schedule then evaluates the residual at
 *                  every checkpoint, not only at lambda = 1); 2 also chi^2_aug
 *                  (wf_chi2_aug) at every checkpoint (merged 2DF block only,
 *                  WF_EUNSUPPORTED otherwise).  Up to 8192 records per problem.
 *  refine_accel    how the defect corrections are combined: 0 each
 *                  correction is subtracted (s <- s - e, iterative
 *                  refinement); m in 1..16 Anderson acceleration with a
 *                  history of m corrections: with f_k = -e_k the k-th
 *                  correction of s_k, the next s is s_k + f_k - sum_j
 *                  gamma_j (Delta s_j + Delta f_j), gamma minimising
 *                  ||f_k - sum_j gamma_j Delta f_j||_2 over the last m
 *                  differences of consecutive s and f (the same Krylov space
 *                  as GMRES on the corrected system, reached without N^-1).
 *                  The FP64 dot products (summed in a fixed order) and the
 *                  least squares run on the device, so a solve still repeats
 *                  bit for bit and a correction needs no host round trip.  Needs refine > 0 to act; the
 *                  plan keeps 2m + 2 more maps.  Default 0.
 */
typedef struct {
  double theta[3];
  double split_f;
  double split_fp;
  double split_w;
  double tol_u_scale;
  int residual_every;
  int max_iters;
  int check_every;
  int merge_2df;
  int refine;
  double refine_tol_scale;
  int refine_max_iters;
  int refine_lam1_iters;
  int stall_checks;
  int autotune;
  int dft_precision;
  int refine_extra;
  int sweep_kernel;
  int trace;
  int refine_accel;
} wf_params;

/* Results of a solve. */
typedef struct {
  int iters;            /* iterations run                                     */
  int checkpoints;      /* residual evaluations                               */
  double lam_final;     /* lambda at exit (1 when converged)                  */
  double rel_rho_u;     /* ||Delta d_unmasked|| / ||d_unmasked|| at exit        */
  double rel_rho_m;     /* ||S^-1 s on masked pixels|| / ||S^-1 s|| at exit    */
  double tau[3];        /* tau_i used (2DF, RF, PX); 0 for absent parts       */
  int status;           /* WF_OK or WF_ENOCONV                                */
  int parts;            /* parts bit mask                                     */
} wf_stats;

typedef struct wf_plan_s* wf_plan_t;

/* Library ABI version (WF_ABI_VERSION). */
WF_API int wf_version(void);

/* Message for a status code (static string). */
WF_API const char* wf_strerror(int status);

/*
 * wf_params_default -- fill *p with the defaults listed at wf_params.
 */
WF_API void wf_params_default(wf_params* p);

/*
 * wf_plan_create -- make a plan for ny x nx maps with the given noise parts.
 *   out     receives the plan handle (unchanged on error)
 *   parts   WF_PART_WHITE | optional WF_PART_1F | optional WF_PART_STRIPE
 *   p       parameters or NULL for defaults
 *   stream  cudaStream_t the plan's work runs on (NULL: the legacy default)
 * Allocates the plan's device workspace (about 12 maps of 4*ny*nx bytes)
 * with cudaMalloc on the current device.
 */
WF_API int wf_plan_create(wf_plan_t* out, int ny, int nx, unsigned parts,
                   const wf_params* p, void* stream);

/* Release a plan and its workspace (NULL is ignored). */
WF_API void wf_plan_destroy(wf_plan_t plan);

/*
 * wf_set_problem -- load one problem into the plan (setup step): copies and
 * validates the inputs, computes tau_i as theta_i x the minimum eigenvalue
 * of each part (Sec. 2) and zeroes the messenger fields (Sec. 2: the
 * iteration starts from s = t0 = d0 = 0).
 *   d          [ny][nx] data; ignored at masked pixels
 *   pixel_var  [ny][nx] white-noise variance (> 0 at unmasked pixels)
 *   mask       [ny][nx] bytes, nonzero = masked; or NULL
 *   C          [ny][nx/2+1] signal eigenvalues (> 0)
 *   P1f        [ny][nx/2+1] 1/f eigenvalues (> 0); NULL iff no WF_PART_1F
 *   Pst        [nx/2+1] stripe eigenvalues per kx (> 0); NULL iff no
 *              WF_PART_STRIPE
 *   stripe_amp2 [ny] per-row factor a(y)^2 (> 0) of the stripe part, or NULL
 *              for 1: the stripe eigenvalue of mode (y, kx) is a(y)^2 Pst[kx]
 * Returns WF_EINVAL / WF_ENOTPD for invalid inputs (checked on the device).
 */
WF_API int wf_set_problem(wf_plan_t plan, const float* d, const float* pixel_var,
                   const uint8_t* mask, const float* C, const float* P1f,
                   const float* Pst, const float* stripe_amp2);

/*
 * wf_run -- run the messenger iteration on the loaded problem until the
 * schedule ends at lambda = 1 and both ||Delta d_u||/||d_u|| <= tol and
 * ||(S^-1 s)_masked|| / ||S^-1 s|| <= tol at a checkpoint (Sec. 2: Delta d =
 * (I + N S^-1) s - d; on masked pixels the residual is S^-1 s), or until
 * max_iters.  tol <= 0 runs exactly max_iters iterations (no stop test).
 * Continues from the current state (call wf_set_problem to restart).
 * Fills *st if not NULL.  Returns WF_OK or WF_ENOCONV.
 */
WF_API int wf_run(wf_plan_t plan, const wf_schedule* sched, double tol, wf_stats* st);

/*
 * wf_iterate -- run exactly n iterations at fixed lambda (no residual, no
 * stop test): one iteration is the sweep t_PX, d_RF, t_RF, d_2DF, t_2DF, s
 * of eqs. (2mess_t1)-(2mess_s) generalised to the present parts.
 */
WF_API int wf_iterate(wf_plan_t plan, double lam, int n);

/*
 * wf_residual -- evaluate the residual of the current iterate: rel_rho_u =
 * ||Delta d_unmasked|| / ||d_unmasked||, rel_rho_m = ||(S^-1 s)_masked|| /
 * ||S^-1 s|| (Sec. 2, reconstructed data).  Either pointer may be NULL.
 */
WF_API int wf_residual(wf_plan_t plan, double* rel_rho_u, double* rel_rho_m);

/*
 * wf_chi2_aug -- the augmented objective of the current iterate (Appendix A,
 * eq. 2mess_prob: the sum over the chain's links of squared differences over
 * their covariances), which every update of the iteration lowers at fixed
 * lambda and which equals chi^2(s) at the fixed point.  The fields the plan
 * does not keep are at their conditional means: s = C/(C + N_0) d_0 and,
 * with a stripe part, the pixel messenger given d_RF and d.  Evaluated at the
 * current lambda, in FP64 from the FP32 fields; *value receives it.
 * WF_EINVAL without a loaded problem (also after wf_solve with refine > 0,
 * whose fields belong to the last correction); WF_EUNSUPPORTED for the plain
 * sweep (merge_2df = 0 with a 1/f part).
 */
WF_API int wf_chi2_aug(wf_plan_t plan, double* value);

/*
 * wf_get_field -- write one field of the current state, in pixel space, to
 * out [ny][nx] (device or host).  Fields absent from the plan's parts give
 * WF_EINVAL (and WF_FIELD_T_2DF with merge_2df, where t_2DF is marginalised).
 */
WF_API int wf_get_field(wf_plan_t plan, int field, float* out);

/*
 * wf_solve -- wf_set_problem + wf_run + wf_get_field(WF_FIELD_S): the whole
 * Wiener filter for one map, followed by params.refine defect-correction
 * solves (see wf_params).  s_out [ny][nx] receives s (also when the return
 * value is WF_ENOCONV).  st may be NULL; with refinement its iters and
 * checkpoints sum over all solves and rel_rho_* are those of the refined s.
 * After a refined solve the plan holds the last correction problem: call
 * wf_set_problem again before wf_run, wf_residual or wf_get_field.
 */
WF_API int wf_solve(wf_plan_t plan, const float* d, const float* pixel_var,
             const uint8_t* mask, const float* C, const float* P1f,
             const float* Pst, const float* stripe_amp2,
             const wf_schedule* sched, double tol, float* s_out,
             wf_stats* st);

/*
 * wf_fft2 -- the plan's transforms on their own (the basis changes of Sec. 2,
 * flat-sky stand-ins for the paper's spherical-harmonic transforms).
 *   inverse = 0: in = real map [ny][nx], out = spectrum [ny][nx/2] complex
 *                (interleaved float pairs), unnormalised forward DFT.
 *   inverse = 1: in = spectrum, out = real map, with the 1/(ny nx) factor.
 * Spectrum layout: column kx (1 <= kx < nx/2) holds X[ky][kx]; column 0
 * holds Z[ky] = A[ky] + i B[ky], where A = X[.][0] and B = X[.][nx/2] (the
 * two real-signal columns packed into one complex column).
 *   rows_only = 1: only the row-wise transform (the stripe basis): in the
 *                same layout, column 0 holds (X[y][0], X[y][nx/2]) as a
 *                real pair per row.
 * The column transforms follow the plan's dft_precision (wf_params).
 */
WF_API int wf_fft2(wf_plan_t plan, const float* in, float* out, int inverse,
            int rows_only);

/*
 * wf_launch_count -- number of CUDA kernels the plan has launched since it
 * was created (measurement aid: launches inside a timed region are the
 * difference of two calls).  Returns -1 for a NULL plan.
 */
WF_API long long wf_launch_count(wf_plan_t plan);

/*
 * wf_plan_shapes -- values per thread of the row pass and of the column pass
 * the plan uses (set by the autotuner when the first problem is loaded).
 * Either pointer may be NULL.
 */
WF_API int wf_plan_shapes(wf_plan_t plan, int* row_values, int* col_values);

/*
 * wf_time_passes -- measurement aid: at fixed lambda, capture n row passes
 * back to back in a CUDA graph and time its replay with CUDA events, then
 * the same for n column passes; return the mean time per launch of each
 * pass in microseconds.  The passes overwrite the state, so the plan must
 * be loaded again (wf_set_problem) before further iteration.
 */
WF_API int wf_time_passes(wf_plan_t plan, double lam, int n, double* us_row,
                          double* us_col);

/*
 * wf_get_trace -- the per-checkpoint trace (wf_params.trace) of every run since
 * the plan last loaded a problem: the first solve and, after wf_solve with
 * refine > 0, its corrections (Sec. 3.3 and Fig. 3 follow the same
 * quantities).  *n_out receives the number of records; min(n, max_records)
 * are written to out (host or device), 6 doubles each: sweeps done in that
 * run, lambda of those sweeps, ||Delta d_u|| / ||d_u||, ||(S^-1 s)_m|| /
 * ||S^-1 s||, chi^2_aug (trace = 2; NaN otherwise), and the run's index (0
 * the first solve, 1, 2, ... its corrections).  The residual terms and
 * chi^2_aug of a correction are those of its own problem (data Delta d_u);
 * its objective also has the masked-pixel source term, which chi^2_aug does
 * not include, so only the first solve's chi^2_aug is monotone within a
 * lambda level.  WF_EINVAL if tracing is off.
 */
WF_API int wf_get_trace(wf_plan_t plan, double* out, int max_records, int* n_out);

/*
 * wf_time_sweeps -- measurement aid: at fixed lambda, capture n sweeps as the
 * plan's iteration launches them (one cooperative launch, or n row-pass /
 * column-pass pairs; see wf_params.sweep_kernel) in a CUDA graph and time its
 * replay with CUDA events; *us_per_sweep receives the mean time per sweep
 * in microseconds and *one_launch (if not NULL) 1 for the one-launch form.
 * The sweeps overwrite the state: load the plan again (wf_set_problem)
 * before further iteration.
 */
WF_API int wf_time_sweeps(wf_plan_t plan, double lam, int n, double* us_per_sweep, int* one_launch);

/*
 * wf_fft2_noalloc -- the forward or inverse 2D transform of wf_fft2 without a
 * plan and without allocating device memory.  The paper has no counterpart:
 * this entry point exists for callers that are not allowed to call
 * cudaMalloc -- a library embedded in a host application whose allocator owns
 * all device memory, or a pipeline that must not allocate once it is running
 * (an allocation can block, fail or synchronise the device at a bad moment).
 *   ny, nx   sizes as for wf_plan_create (powers of two in [32, 4096], or
 *            384, 768, 1536) with ny * nx <= 1048576
 *            (WF_EUNSUPPORTED otherwise)
 *   in, out  device arrays owned by the caller, laid out as for wf_fft2
 *            (host pointers give WF_EINVAL)
 *   inverse  0: real map -> spectrum; 1: spectrum -> real map (1/(ny nx))
 *   stream   cudaStream_t to launch on; the call returns after launching and
 *            the result is ready when that stream reaches it
 * Working memory (the intermediate row-transformed spectrum, up to 4 MiB, and
 * 64 KiB of twiddle tables) is one fixed device array inside the library that
 * every GPU loading the library keeps until the process exits.  The first
 * call on a device looks that array's address up (cudaGetSymbolAddress, with
 * the device current); make that first call before any stream capture.  All
 * calls share the array and nothing in it has to start at zero (each call
 * rewrites what it reads), but calls that overlap on the GPU -- on different
 * streams, or from different threads -- race with each other.
 */
WF_API int wf_fft2_noalloc(int ny, int nx, const float* in, float* out,
                           int inverse, void* stream);

/* ------------------------------------------------------------------------
 * Batched solves: many independent maps of uneven sizes (the parts and
 * parameters shared).  Every map gets its own plan.  With lanes > 0 the maps
 * are spread over `lanes` host worker threads, each driving its maps one
 * after another on its own CUDA stream, so up to `lanes` solves share the GPU
 * at once (small maps fill only a few SMs each); a map's result is then the
 * one wf_solve gives for it alone, bit for bit.  With lanes = 0 the maps'
 * iterations run together in persistent launches (see wf_batch_create); the
 * steps of each map's solve are those of wf_solve, its transforms may take
 * other shapes (rounding order only).
 * ------------------------------------------------------------------------ */

typedef struct wf_batch_s* wf_batch_t;

/* One map of a batch; arrays as for wf_solve (host or device), s_out
 * receives s. */
typedef struct {
  const float* d;
  const float* pixel_var;
  const uint8_t* mask;
  const float* C;
  const float* P1f;
  const float* Pst;
  const float* stripe_amp2;
  float* s_out;
} wf_map;

/*
 * wf_batch_create -- plans for nmaps maps, map i of ny[i] x nx[i] pixels.
 *   nmaps   1 .. 65536
 *   ny, nx  host arrays of nmaps sizes, each as for wf_plan_create
 *   parts   as for wf_plan_create, shared by all maps
 *   p       parameters (NULL: defaults), shared
 *   lanes   concurrent solves (host threads and streams), 1 .. 64; maps go
 *           to lanes largest first, each to the lane with the fewest pixels.
 *           0: persistent mode -- the sweeps of all maps run together in
 *           one persistent cooperative launch per residual checkpoint, with
 *           device work queues over (map, row group) and (map, column group)
 *           items, a grid barrier between the row and column phases and
 *           per-map done flags (each map keeps its own lambda, residual and
 *           stop test); every polling chunk of checkpoints, with each map's
 *           residual and controller kernels, is one CUDA graph.  Maps must
 *           be square with sides 256, 384, 512, 768, 1024, 1536 or 2048,
 *           with a stripe part and the merged 2DF block (or no 1/f part),
 *           dft_precision 0 (WF_EUNSUPPORTED otherwise).  Each size has one
 *           or two compiled shapes of its transforms; wf_params.autotune
 *           picks them as for a plan (1: timed on the first map of the size,
 *           cached per size and device for the process).
 *   stream  the caller's stream: wf_batch_solve starts after the work
 *           already on it and the caller's later work waits for the batch
 * Allocates every plan's workspace up front (about 14 maps of 4 ny nx bytes
 * per map with refine > 0).  Returns WF_EINVAL / WF_EUNSUPPORTED on bad
 * arguments before any CUDA call.
 */
WF_API int wf_batch_create(wf_batch_t* out, int nmaps, const int* ny, const int* nx, unsigned parts,
                           const wf_params* p, int lanes, void* stream);

/* Release a batch and its plans (NULL is ignored). */
WF_API void wf_batch_destroy(wf_batch_t batch);

/*
 * wf_batch_solve -- wf_solve for every map of the batch.
 *   maps    host array of nmaps wf_map (map i has the batch's size i)
 *   sched, tol  as for wf_solve, shared
 *   stats   host array of nmaps wf_stats, or NULL
 * Returns WF_OK when every map converged, WF_ENOCONV or WF_ESTALL (that of the
 * first such map) when some did not (their s_out holds the last iterate), or
 * the first error of any map.
 */
WF_API int wf_batch_solve(wf_batch_t batch, const wf_map* maps, const wf_schedule* sched, double tol,
                          wf_stats* stats);

/* Kernels launched by all plans of the batch since creation. */
WF_API long long wf_batch_launch_count(wf_batch_t batch);

/* ------------------------------------------------------------------------
 * Learned warm start.  The paper has no network: this is an extension that
 * predicts s with a Fourier neural operator (FNO) and starts the messenger
 * iteration from it; the iteration stays the judge of the result.
 *
 * Network for input x [B, 2, n, n] (see wf_fno_features):
 *   h_0 = P x + p;  h_{l+1} = act(W_l h_l + w_l + K_l h_l), l < layers
 *   (act = GELU, identity after the last layer);  y = Q h_layers + q.
 * K_l: truncated real 2D DFT of every channel on k_x in [0, mx), k_y in
 * [0, my) U [n - my, n), one complex width x width matrix per mode, and the
 * truncated inverse (1/n^2, real part).  Parameters are one FP32 vector in
 * the order P [width][2], p [width], per layer W_l [width][width], w_l
 * [width], R_l [width_in][width_out][2 my][mx] as (re, im) pairs, then
 * Q [1][width], q [1].  Matrices are used in FP16 with FP32 accumulation.
 * ------------------------------------------------------------------------ */

typedef struct wf_fno_s* wf_fno_t;

/*
 * wf_fno_create -- a network and its training state for n x n maps and up to
 * `batch` maps per call.
 *   n        power of two in [16, 1024];  batch 1 .. 64
 *   width    even, 2 .. 64;  mx 1 .. min(32, n/2);  my 1 .. min(32, n/2)
 *   layers   1 .. 8
 *   params   initial parameters (host or device, FP32, in the order above)
 *   stream   cudaStream_t for every later call on this network
 * Adam moments start at zero.
 */
WF_API int wf_fno_create(wf_fno_t* out, int n, int batch, int width, int mx, int my, int layers,
                         const float* params, void* stream);
WF_API void wf_fno_destroy(wf_fno_t fno);

/* Number of parameters (floats), or -1 for NULL. */
WF_API long long wf_fno_num_params(wf_fno_t fno);

/* y [nb, n, n] = network(x [nb, 2, n, n]); device arrays; nb <= batch. */
WF_API int wf_fno_forward(wf_fno_t fno, const float* x, float* y, int nb);

/*
 * wf_fno_gradient -- loss = mean_b ||y_b - t_b||^2 / ||t_b||^2 over nb maps,
 * and its gradient with respect to the parameters (as the forward pass uses
 * them, FP16-rounded matrices) into grad (host or device, num_params floats;
 * NULL to skip).  x, t device arrays.  Nothing is updated.
 */
WF_API int wf_fno_gradient(wf_fno_t fno, const float* x, const float* t, int nb, float* grad, double* loss);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on the FP32 parameters. */
WF_API int wf_fno_train_step(wf_fno_t fno, const float* x, const float* t, int nb, double lr, double* loss);

/* Copy the parameters out (host or device): rounded = 0 the FP32 master
 * values, 1 the values the forward pass uses (FP16-rounded matrices). */
WF_API int wf_fno_get_params(wf_fno_t fno, float* out, int rounded);

/*
 * wf_fno_features -- network input of one map: x[0] = d / sigma (0 where
 * masked), x[1] = log(sigma^2 / pixel_var) (log 1e-6 where masked), with
 * sigma^2 the mean pixel variance over unmasked pixels, written to
 * sigma_out (device float).  All pointers device; launched on `stream`.
 */
WF_API int wf_fno_features(int ny, int nx, const float* d, const float* pixel_var, const uint8_t* mask,
                           float* x_out, float* sigma_out, void* stream);

/*
 * wf_inverse_noise -- approximately inverse-noise-weighted map N^-1 d (with a
 * mask: zero on masked pixels, (P N P^T)^-1 d on the others), computed as a
 * Wiener filter with the signal covariance set to S = alpha I (Sec. 4):
 * N^-1 d ~ alpha^-1 [alpha (alpha I + N)^-1 d], relative error of order
 * alpha / (smallest eigenvalue of N).  alpha > 0 (for example 1e-3 times the
 * smallest pixel variance).  Arguments as for wf_solve without C; out (host
 * or device, [ny][nx]) receives the weighted map; tol is the stop test of
 * that filter.  Uses the plan's host-staging buffers for C and for s.
 */
WF_API int wf_inverse_noise(wf_plan_t plan, const float* d, const float* pixel_var, const uint8_t* mask,
                            const float* P1f, const float* Pst, const float* stripe_amp2, double alpha,
                            const wf_schedule* sched, double tol, float* out, wf_stats* stats);

/*
 * wf_solve_warm -- wf_solve started from an estimate s_init of s (host or
 * device [ny][nx]) instead of zero: the messenger fields are set to s_init
 * in their own bases (t_RF = d_RF = s_init row-transformed; the signal-side
 * field d_2DF = (C + N_0)/C s_init, so that the implicit s equals s_init)
 * before the schedule runs.  Everything else as wf_solve.
 */
WF_API int wf_solve_warm(wf_plan_t plan, const float* d, const float* pixel_var, const uint8_t* mask,
                         const float* C, const float* P1f, const float* Pst, const float* stripe_amp2,
                         const float* s_init, const wf_schedule* sched, double tol, float* s_out,
                         wf_stats* stats);

#ifdef __cplusplus
}
#endif

#endif /* WF_H */
