/*
 * plc.h -- C ABI of libplc, the GB300 (sm_103a) Poisson-lognormal MAP solver.
 *
 * The library finds the maximum a posteriori log-density s = ln(1 + delta) on a
 * periodic cubic grid of n^3 cells, given galaxy counts N, a completeness w,
 * the mean count nbar, a constant prior mean mu and a tabulated power spectrum
 * P(k) (Kitaura, Jasche & Metcalf, "Recovering the nonlinear density field
 * from the galaxy distribution with a Poisson-Lognormal filter"):
 *
 *   -ln P(s|N) = 1/2 (s - mu)^T S^-1 (s - mu) + sum_i [ w_i nbar e^{s_i} - N_i s_i ]
 *
 * (lognormal prior of Sec. 2.3 times the Poisson likelihood of Sec. 2.1, unity
 * bias, constants dropped), whose stationarity condition is Eq. (MAPLNUB).
 *
 * Conventions shared by every call
 *   - Fields are caller-owned DEVICE pointers, C order [z][y][x] (x fastest),
 *     n^3 elements, 16-byte aligned.  Counts N are int32.  The element type
 *     of a field argument is stated per call: "real" means double for a
 *     context created with PLC_FP64 and float for PLC_MIXED.
 *   - w may be NULL, meaning w = 1 everywhere.
 *   - The prior: S is a convolution, diagonal under the unnormalised forward
 *     DFT (Sec. 2.2) with eigenvalue lambda_k = P(|k|) n^3 / L^3,
 *     |k| = (2 pi / L) |m|, m in [-n/2, n/2) per axis; P is interpolated
 *     linearly in (ln k, ln P) between table points.  The DC mode carries an
 *     explicit inverse eigenvalue (0 = flat prior on the mean).
 *   - Work is enqueued on the context's stream.  Calls that return host
 *     scalars synchronise that stream before returning.
 *   - No call throws.  Invalid arguments return PLC_ERR_INVALID_ARG with
 *     nothing launched; plc_last_error() describes the last failure.
 *   - A context is not thread-safe; use one context per host thread.
 *   - The library allocates device scratch only in plc_create/plc_set_prior
 *     and on the first use of a call that needs solver work fields.
 */
#ifndef PLC_H
#define PLC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PLC_OK = 0,
  PLC_ERR_INVALID_ARG = 1,   /* bad size, NULL pointer, bad table, no prior set */
  PLC_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  PLC_ERR_NOT_CONVERGED = 3, /* iteration cap reached; outputs hold the last iterate */
  PLC_ERR_NONFINITE = 4,     /* NaN or Inf in the objective or gradient */
  PLC_ERR_CG_BREAKDOWN = 5,  /* p^T H p <= 0 on the first CG step */
  PLC_ERR_OOM = 6            /* device allocation failed */
} plc_status;

typedef enum {
  PLC_FP64 = 0,  /* every field and FFT in double */
  PLC_MIXED = 1  /* FP32 FFTs and pointwise work, FP64 reductions and scalars;
                    the Newton solve keeps an FP64 master copy of s and takes
                    its stopping gradient in FP64 */
} plc_precision;

typedef struct plc_ctx plc_ctx;

/* Create a context for an n^3 grid in a periodic box of side `box` (Mpc/h).
 * n must be even, 4 <= n <= 512, with no prime factor other than 2 and 3.
 * `cuda_stream` is a cudaStream_t (NULL = legacy default stream).
 * Allocates the FFT scratch (two half-spectra of the widest type). */
plc_status plc_create(plc_ctx** ctx, int n, double box, int precision,
                      void* cuda_stream);

/* Destroy a context and free its device memory.  NULL is accepted. */
plc_status plc_destroy(plc_ctx* ctx);

/* Set the prior (Sec. 2.2-2.3): host arrays k[nk] (h/Mpc, strictly
 * ascending, > 0) and P[nk] ((Mpc/h)^3, > 0), nk >= 2, covering every
 * non-zero mode of the grid: k[0] <= 2 pi / L and k[nk-1] >= sqrt(3) pi n / L.
 * mu is the constant prior mean (Sec. 2.3, Eq. mu); inv_lambda_dc the inverse
 * eigenvalue of the DC mode (>= 0; 0 = flat prior on the mean).  The table is
 * copied; the per-mode inverse eigenvalues are built on the device. */
plc_status plc_set_prior(plc_ctx* ctx, const double* k, const double* P,
                         int nk, double mu, double inv_lambda_dc);

/* y = S^-1 x (Sec. 2.2): forward 3D real FFT, division by lambda_k,
 * inverse FFT.  x, y: real fields (may alias). */
plc_status plc_prior_apply(plc_ctx* ctx, const void* x, void* y);

/* Negative log posterior and its gradient at s (Sec. 3.1.2):
 *   g = S^-1 (s - mu) + nbar w e^s - N.
 * s, w, grad: real fields; N: int32 field.  *neg_logpost (host, FP64,
 * reduced in FP64) receives -ln P(s|N) without its s-independent
 * constants.  Either output may be NULL.  Synchronises the stream when
 * neg_logpost is not NULL. */
plc_status plc_logpost_grad(plc_ctx* ctx, const void* s, const int32_t* N,
                            const void* w, double nbar, double* neg_logpost,
                            void* grad);

/* Hessian-vector product at s (Sec. 3.1.2):
 *   Hv = S^-1 v + nbar w e^s v.
 * s, w, v, Hv: real fields (Hv may alias v). */
plc_status plc_hessvec(plc_ctx* ctx, const void* s, const void* w,
                       double nbar, const void* v, void* Hv);

typedef struct {
  double tol;          /* stop when ||g|| / ||g0|| < tol (default 1e-6) */
  int max_newton;      /* outer iteration cap (default 200) */
  int max_cg;          /* CG iterations per Newton step (default 1000) */
  int precond;         /* 0 none, 1 Jacobi diag(H) (default 1) */
  double g0_norm;      /* > 0: use as ||g0|| (resume); 0: ||g(s_in)|| */
  double step_cap;     /* max |tau xi| per Newton step (default 2) */
  double eta_max;      /* CG forcing term cap (default 0.5); the CG stops at
                          eta = min(eta_max, max(sqrt(rel), 0.3 tol / rel)) */
  int cg_chunk;        /* CG iterations enqueued between host checks (default 8) */
  double mixed_switch; /* PLC_MIXED: gradients in FP32 while ||g|| / ||g0|| is at or
                          above this and above tol, in FP64 below it (default 1e-6;
                          >= 1 means FP64 throughout).  The switch also happens when
                          an FP32 Newton step below 1e-3 fails to halve ||g||.  The
                          stopping test is always taken on an FP64 gradient. */
  int device_driven;   /* 1: the solve's decisions are taken on the device and the
                          whole solve is one CUDA graph launch (conditional nodes;
                          captured on the first call and reused while N, w, nbar,
                          s_inout, the prior and the options stay the same); 0: a
                          host loop reads the device scalars after each gradient,
                          CG chunk and trial.  Same iteration either way
                          (default 1). */
  int start;           /* plc_newton_krylov_map and plc_gauss_map: 1 (default)
                          iterate from the per-cell MAP of the same posterior
                          with the prior replaced by its diagonal (the prior
                          variance per cell; the Lambert-W solution of
                          Eq. MAPLNUB, resp. the domain root of the quadratic of
                          Eq. MAPG, cell by cell), 0 from the caller's start
                          itself.  ||g0|| of the stopping test is taken at the
                          caller's start either way.  2: as 1 with the caller's
                          start taken to be the prior mean (mu, resp.
                          delta = 0) without reading it: s_inout / delta_inout
                          is output only, its contents on entry are ignored
                          (the same iterates and result as 1 with the array
                          filled with the mean, one field read and the fill
                          saved).  plc_bias_map ignores it. */
} plc_opts;

typedef struct {
  int newton_iters;    /* outer iterations taken */
  int cg_iters;        /* total CG iterations */
  int hv_count;        /* Hessian-vector products applied */
  int grad_evals;      /* gradient evaluations, line-search trials included */
  int grad_ffts;       /* of which evaluated through the FFT (the others carry
                          S^-1 (s - mu) forward from the CG) */
  int grad_ffts_fp64;  /* of those, with FP64 transforms */
  double grad_rel;     /* final ||g|| / ||g0|| */
  double g0_norm;      /* ||g0|| used */
  double neg_logpost;  /* final -ln P(s|N) (constants dropped) */
  double ms;           /* wall time of the call, milliseconds */
  long long kernels;   /* kernels launched by the solve (device-driven solves) */
} plc_stats;

/* Fill *opts with the defaults above. */
plc_status plc_default_opts(plc_opts* opts);

/* MAP by inexact Newton-Krylov (Sec. 3.1): s <- s + tau xi with tau from
 * Eq. (New5), xi from preconditioned CG on H xi = -g, a step cap and an
 * Armijo backtracking line search.  The prior term S^-1 (s - mu) is taken
 * through the FFT at the start (and, for PLC_MIXED, once when the state moves
 * from FP32 to FP64) and otherwise carried forward with S^-1 xi from the CG.  s_inout (double, device) holds the start
 * point on entry (e.g. filled with mu; not read with opts->start = 2) and
 * the MAP on exit.  N: int32 field;
 * w: double field or NULL (double in both precisions).  opts NULL = defaults;
 * stats may be NULL.  Returns PLC_ERR_NOT_CONVERGED with s_inout holding the
 * last iterate when max_newton is reached.  Synchronises the stream. */
plc_status plc_newton_krylov_map(plc_ctx* ctx, const int32_t* N, const void* w,
                                 double nbar, double* s_inout,
                                 const plc_opts* opts, plc_stats* stats);

/* MAP of the Gaussian-prior Poisson model with unity bias (Sec. 2.2.2,
 * Eq. MAPG; gradient and Hessian of Sec. 3.1.1 without the factor S): the
 * overdensity delta minimising
 *   1/2 delta^T S^-1 delta + sum_i [ nbar w_i (1 + delta_i) - N_i ln(1 + delta_i) ]
 * over 1 + delta_i > 0 where N_i > 0 (cells with N_i = 0 may go below -1).
 * The same inexact Newton-Krylov iteration and precision scheme as
 * plc_newton_krylov_map (host-driven; opts->device_driven is not used), with
 * the step kept inside the domain by the fraction to the boundary,
 * tau <= 0.99 / max(-xi_i / (1 + delta_i)) over cells with N_i > 0, instead
 * of opts->step_cap.  S is the context's prior (mu is not used: the prior
 * of delta has mean 0).  delta_inout (double, device): start point on entry
 * (0 = the prior mean; it must satisfy 1 + delta > 0 where N > 0), MAP on
 * exit.  N: int32 field; w: double field or NULL.  Synchronises the stream. */
plc_status plc_gauss_map(plc_ctx* ctx, const int32_t* N, const void* w, double nbar,
                         double* delta_inout, const plc_opts* opts, plc_stats* stats);

/* LSQ-Wiener filter with unity bias (Sec. 4.1.1, Eq. WF; Table 1, Gaussian
 * prior and Gaussian likelihood): the linear estimate of the overdensity
 *   delta = (S^-1 + diag(nbar w))^-1 (N - nbar w),
 * from the data vector N / nbar - w (Eq. datamodel) with noise covariance
 * diag(w / nbar) (Eq. noiseav).  S is the context's prior (its mean mu is
 * not used: the prior of delta has mean 0).  Solved by Jacobi-preconditioned
 * CG from delta = 0 to relative residual opts->tol (the CG runs in FP32 for
 * a PLC_MIXED context, so about 1e-6 at best), on the context's stream; the
 * other options are not used.  N: int32 field; w: double field or NULL;
 * delta_out: double field.  stats: cg_iters, hv_count, grad_rel (the final
 * relative residual), g0_norm (||N - nbar w||), ms.  Returns
 * PLC_ERR_NOT_CONVERGED (delta_out holding the last iterate) when max_cg is
 * reached.  Synchronises the stream. */
plc_status plc_wiener_lsq(plc_ctx* ctx, const int32_t* N, const void* w, double nbar,
                          double* delta_out, const plc_opts* opts, plc_stats* stats);

/* Linear bias of the galaxy field (Sec. 2.4.1, with Sec. 2.2.1): the
 * expected counts become nbar w (1 + B delta_M), B the convolution whose
 * Fourier multiplier is the bias b(|k|) (b = sqrt(P_g / P_M) for the galaxy
 * and matter spectra).  k, b: HOST arrays of nb >= 2 points, k > 0 strictly
 * ascending, b > 0, covering [2 pi / L, sqrt(3) pi n / L] like the P(k)
 * table of plc_set_prior; b is linear in (ln k, ln b) between table points.
 * b_dc > 0: the multiplier of the DC mode.  Replaces an earlier table; the
 * context copies what it needs.  Synchronises the stream. */
plc_status plc_set_bias(plc_ctx* ctx, const double* k, const double* b, int nb, double b_dc);

/* -ln P of the lognormal-prior Poisson model with linear bias (Sec. 2.4.1)
 * at s = ln(1 + delta_M):
 *   L(s) = 1/2 (s - mu)^T S^-1 (s - mu) + sum_i [ nbar w_i u_i - N_i ln u_i ],
 *   u = 1 + B(e^s - 1),
 * +inf where u_i <= 0 in a cell with N_i > 0, and its gradient (the MAP
 * equation of Sec. 2.4.1)
 *   g = S^-1 (s - mu) + e^s . B(nbar w - N / u).
 * Needs plc_set_prior and plc_set_bias.  s, grad: fields of the context's
 * precision (grad may be NULL); N: int32 field; w: double field or NULL;
 * neg_logpost: host double or NULL (PLC_ERR_NONFINITE when it is not
 * finite).  Synchronises the stream when neg_logpost is given. */
plc_status plc_bias_logpost_grad(plc_ctx* ctx, const void* s, const int32_t* N, const void* w,
                                 double nbar, double* neg_logpost, void* grad);

/* The exact Hessian of that L applied to v:
 *   H v = S^-1 v + d1 . v + e^s . B((N / u^2) . B(e^s . v)),
 *   d1 = e^s . B(nbar w - N / u).
 * H need not be positive definite.  s, v, Hv: fields of the context's
 * precision; N: int32 field; w: double field or NULL. */
plc_status plc_bias_hessvec(plc_ctx* ctx, const void* s, const int32_t* N, const void* w,
                            double nbar, const void* v, void* Hv);

/* MAP of that L: the inexact Newton-Krylov iteration of
 * plc_newton_krylov_map (host-driven; opts->device_driven and opts->start are
 * not used) with the exact Hessian above.  The CG stops at non-positive
 * curvature and keeps its iterate (the preconditioned gradient step when
 * that happens on its first direction); tau = 1 when xi^T H xi <= 0; trial
 * points outside the domain count as L = +inf and are halved.  The prior
 * term is carried forward with S^-1 xi, one FFT pipeline per Newton step.
 * s_inout (double, device): start point on entry (0, i.e. delta_M = 0, is
 * inside the domain for any b), MAP on exit.  PLC_MIXED: FP32 state and CG
 * until max(mixed_switch, tol) or FP32 stagnation, then FP64 state (FP64
 * transforms) with the FP32 CG; the stop test is passed on an FP64 gradient.
 * Returns PLC_ERR_NONFINITE when the start point is outside the domain.
 * Synchronises the stream. */
plc_status plc_bias_map(plc_ctx* ctx, const int32_t* N, const void* w, double nbar,
                        double* s_inout, const plc_opts* opts, plc_stats* stats);

/* Implicit adjoint of the MAP (implicit-function theorem on g(s*) = 0; the
 * paper has no counterpart).  For a cotangent u (double field), solves
 * H lam = u by CG at s_map and returns
 *   vjp_N   = lam                               (d s* / d N is H^-1)
 *   vjp_lnA = lam^T S^-1_{k != 0} (s_map - mu)  (d s* / d ln A, A scaling
 *                                                every non-DC lambda_k).
 * s_map, u, vjp_N: double fields; w: double field or NULL.  The CG stops at
 * relative residual opts->tol (MIXED: FP32 CG, so about 1e-6 at best).
 * Synchronises the stream. */
plc_status plc_map_vjp(plc_ctx* ctx, const double* s_map, const void* w,
                       double nbar, const double* u, double* vjp_N,
                       double* vjp_lnA, const plc_opts* opts, plc_stats* stats);

/* Quality measures of a reconstruction (Sec. 4.1.2; the paper compares
 * estimates with the true matter field by these): the correlation
 * coefficient r = sum a b / (sqrt(sum a^2) sqrt(sum b^2)) and the Euclidean
 * distance D_Euc = sqrt(mean((a - b)^2)) of two double fields, reduced in
 * FP64 (either output may be NULL, not both).  Synchronises the stream. */
plc_status plc_compare(plc_ctx* ctx, const double* a, const double* b, double* r,
                       double* d_euc);

/* Gaussian smoothing on the periodic grid (Sec. 4.3.3 smooths with radii of
 * 5 and 10 Mpc/h before the matter statistics): y = x convolved with a
 * normalised Gaussian of radius `radius` (Mpc/h, >= 0), i.e. every Fourier
 * mode multiplied by exp(-|k|^2 radius^2 / 2), |k| as for the prior.  x, y:
 * double fields (may alias).  Transforms in float-float (about 48 bits) for
 * lengths with a four-step schedule, FP64 otherwise; uses the solver work
 * fields as scratch.  Needs no prior.  Synchronises the stream. */
plc_status plc_smooth(plc_ctx* ctx, const double* x, double* y, double radius);

/* Matter statistics of x = ln(1 + delta) (Sec. 4.3.3): counts[j] (host,
 * nbins entries, 1 <= nbins <= 4096) of cells with x in
 * [lo + j width, lo + (j+1) width) (bin index floor((x - lo) / width) in
 * FP64), outside[3] = {below lo, at or above lo + nbins width, cells with
 * 1 + delta <= 0}, and moments[4] = {mean, variance (population), skewness
 * m3 / m2^(3/2), excess kurtosis m4 / m2^2 - 3} of x over the cells with
 * 1 + delta > 0 (the paper defers these formulas to earlier work; these are
 * the standard ones).  delta: double field.  The device-side counts live in
 * a buffer of 4099 entries that the context allocates on the first call
 * (any nbins in range fits, whatever the grid size).  nbins outside
 * 1..4096, a non-finite lo, a width <= 0 or a NULL output give
 * PLC_ERR_INVALID_ARG with nothing launched.  Synchronises the stream. */
plc_status plc_log_stats(plc_ctx* ctx, const double* delta, double lo, double width, int nbins,
                         long long* counts, long long* outside, double* moments);

/* FFT schedule of the FP32 transforms (PLC_MIXED contexts; an aid to
 * performance, the paper has no counterpart).  A length n = f1 f2 with a
 * register four-step form can run it with the factors (f1, f2) or with the
 * shared-memory Stockham stages (f1 = f2 = 0); every schedule computes the
 * same transform.  plc_set_fft_schedule selects one (INVALID_ARG if (f1, f2)
 * is not offered for this n).  plc_autotune times `reps` (1..1000)
 * Hessian-vector products with each schedule offered for n, keeps the
 * fastest and returns it (f1, f2 and its time per Hv in microseconds, any
 * output may be NULL); it uses the solver work fields as scratch (and
 * allocates them on first use) and synchronises the stream.  On a PLC_FP64
 * context (Stockham only) it times nothing and returns the current
 * schedule with *us_per_hv = 0. */
plc_status plc_set_fft_schedule(plc_ctx* ctx, int f1, int f2);
plc_status plc_autotune(plc_ctx* ctx, int reps, int* f1, int* f2, double* us_per_hv);

/* A batch of independent MAP solves (many mocks, each with its own grid
 * size, prior, counts and selection; the paper has no counterpart): every
 * context's device-driven solve is captured as its own chain of one CUDA
 * graph, so the whole batch is one graph launch whose chains run
 * concurrently.  plc_batch_create takes `count` contexts (each with its
 * prior set; the batch does not own them, and they must outlive it and not
 * be used concurrently with it). */
typedef struct plc_batch plc_batch;

plc_status plc_batch_create(plc_batch** batch, plc_ctx* const* ctxs, int count);

/* Solve all: N[i] (int32), w[i] (double or NULL; w itself may be NULL for
 * w = 1 everywhere), nbar[i] (host), s_inout[i] (double: start point in,
 * MAP out) are context i's fields.  opts (NULL = defaults) applies to every
 * solve; stats (NULL or count entries) receives each solve's statistics,
 * ms being the wall time of the whole batch.  The graph is captured on the
 * first call and relaunched while the pointers and options stay the same.
 * Launched on cuda_stream (NULL = legacy default stream); synchronises it.
 * Returns the first non-OK status of the solves, PLC_OK if all converged. */
plc_status plc_batch_map(plc_batch* batch, const int32_t* const* N, const double* const* w,
                         const double* nbar, double* const* s_inout, const plc_opts* opts,
                         plc_stats* stats, void* cuda_stream);

plc_status plc_batch_destroy(plc_batch* batch);

/* Per-kernel launch counters and device time (an aid to profiling; the
 * paper has no counterpart).  Launch counts are always kept.  on != 0 also
 * brackets every launch with a pair of CUDA events on the context's stream
 * (a small host cost per launch).  Either call resets the counters. */
typedef struct {
  char name[24];        /* kernel kind, e.g. "z_f32" (pass Z, FP32) */
  long long launches;   /* launches since the last reset */
  long long timed;      /* launches timed with events */
  double total_ms;      /* summed event time of the timed launches */
} plc_kernel_time;

plc_status plc_profile_enable(plc_ctx* ctx, int on);

/* Copy up to cap records into out (cap may be 0 to query *count, the number
 * of kernel kinds).  Synchronises the stream. */
plc_status plc_profile_read(plc_ctx* ctx, plc_kernel_time* out, int cap, int* count);

/* Hessian-vector product that allocates no device memory (the paper has no
 * counterpart; this is a service for callers that cannot call cudaMalloc --
 * programs whose device memory is reserved up front by an allocator they do
 * not own, real-time or certified code that forbids allocation after
 * start-up, plug-ins that may not create allocations of their own).
 * Computes the same Hv = S^-1 v + nbar w e^s v as plc_hessvec on a PLC_FP64
 * context, without a context: the prior is given by HOST arrays k, P
 * (plc_set_prior's rules, 2 <= nk <= 1024) and inv_lambda_dc; s, w (NULL =
 * 1), v, Hv are double DEVICE fields of n^3 cells, 16-byte aligned.
 * Limit: n <= 64 (even, prime factors 2 and 3); larger n returns
 * PLC_ERR_INVALID_ARG with a message in plc_last_error(NULL).
 * Scratch: one file-scope device array of about 4.2 MiB that every GPU
 * which loads the library holds until the process exits.  The first call on
 * a device looks up that array's device address (cudaGetSymbolAddress, with
 * the device current) and caches it; make that first call before any stream
 * capture.  All calls on a device share the array and it keeps the last
 * call's contents (each call rewrites everything it reads, so nothing needs
 * clearing); two calls whose work overlaps on the same GPU, e.g. from
 * different streams, race on it: serialise them.  The cached address dies
 * with the device's primary context: after a cudaDeviceReset, unload and
 * reload the library before calling this again on that device.  If a CUDA
 * error from an earlier, unrelated call is pending on entry, nothing is
 * launched, PLC_ERR_CUDA is returned and the pending error is left in place
 * for its owner.  Enqueued on cuda_stream (NULL = legacy default stream);
 * returns after enqueue. */
plc_status plc_hessvec_noalloc(int n, double box, const double* k, const double* P,
                               int nk, double inv_lambda_dc, const double* s,
                               const double* w, double nbar, const double* v,
                               double* Hv, void* cuda_stream);

/* Message of the last failure on this context ("" if none). */
const char* plc_last_error(const plc_ctx* ctx);

/* Static name of a status code. */
const char* plc_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* PLC_H */
