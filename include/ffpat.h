/*
 * ffpat.h -- C ABI of the GB300 (sm_103a) library for one-step full-field
 * photoacoustic tomography with a variable sound speed (Haltmeier, Zangerl,
 * Nuster, Nguyen, "Photoacoustic image reconstruction from full field data in
 * heterogeneous media", 2019).
 *
 * Model (Sec. 2.1, eq. (1)-(3)): p_tt = c(x)^2 Delta p on [-1,1]^3,
 * p(.,0) = h, p_t(.,0) = 0; W h = p(., T).  Data (eq. (4), Problem 1 with full
 * data): g = P W h, where P takes line integrals in every horizontal plane
 * z = const over the directions theta_j = pi j / n_angles, j < n_angles.
 *
 * Discretisation (fixed by this library):
 *   grid     N^3 cell-centred points, x_i = -1 + (i + 1/2) dx, dx = 2/N;
 *            volumes are [z][y][x] with x fastest, N^3 elements;
 *   time     Nt = ceil(T c_max / (cfl dx) (1 - 1e-12)), dt = T / Nt,
 *            kappa = (c dt / dx)^2; p^1 = p^0 + kappa L4 p^0 / 2 and
 *            p^{n+1} = 2 p^n - p^{n-1} + kappa L4 p^n, L4 the fourth-order
 *            central Laplacian with zero ghost values outside the box;
 *   rays     detector xi_k = -1 + (k + 1/2) dx, k < N; samples
 *            s_m = (m + 1/2 - Ns/2) dx, m < Ns = 2 ceil(N / sqrt 2), each
 *            sampled bilinearly (zero outside the grid) at
 *            xi_k theta + s_m theta_perp, theta_perp = (-sin, cos);
 *   data     g[j][l][k] = dx sum_m B(p[l]; ...), layout [theta][z][xi],
 *            n_angles * N * N elements.
 *   padding  pad > 0 runs the wave on a larger grid than the source box: Nw =
 *            N + 2 pad points per axis with the same dx, spanning [-L, L]^3,
 *            L = Nw / N (the V_T of the wave model, Sec. 2.1, and the enlarged
 *            computational domain of the paper's experiments, Sec. 5), so that
 *            waves travel past the box instead of reflecting at its faces.
 *            The source h, the image-domain results and the support are N^3
 *            on the box; W zero-extends h to the wave grid and steps there;
 *            P projects the whole wave grid: Nw planes of Nw detectors
 *            xi_k = -L + (k + 1/2) dx, Ns = 2 ceil(Nw / sqrt 2) samples, so
 *            the data are n_angles Nw^2 values.  The sound speed c is given
 *            on the wave grid, Nw^3 elements, and Nt uses its maximum.  With
 *            pad = 0, Nw = N and L = 1 throughout.
 * The adjoint entry points apply the exact matrix transposes of these
 * discrete operators, so <A h, g> = <h, A^T g> up to rounding.
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers owned by the caller, of element type
 *     double when problem.precision == FFPAT_FP64 and float otherwise.  The
 *     library keeps no reference to them after the call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is queued on it; unless stated otherwise an entry point
 *     returns once the work is queued, and the caller synchronises the stream.
 *   - `ws` is caller-owned device scratch of at least
 *     ffpat_workspace_bytes(problem) bytes, 256-byte aligned; its contents on
 *     entry do not matter.  Two calls that run concurrently need two
 *     workspaces.  For FP32 grids up to 128^3 the wave time loop is one
 *     cooperative launch that occupies every SM while it runs, so such loops
 *     issued on several streams run one after another rather than side by
 *     side (the results do not depend on it).
 *   - Return value: FFPAT_OK (0) or a negative ffpat_status.  On error,
 *     ffpat_last_error() (per host thread) describes it.  No call aborts the
 *     process and no C++ exception crosses this boundary.
 */
#ifndef FFPAT_H
#define FFPAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FFPAT_OK = 0,
  FFPAT_EINVAL = -1,    /* invalid argument (sizes, c <= 0 or not finite, CFL > 1/2, ...) */
  FFPAT_ENOMEM = -2,    /* workspace too small or allocation refused */
  FFPAT_ECUDA = -3,     /* a CUDA runtime call failed */
  FFPAT_EBUSY = -4,     /* server queue full */
  FFPAT_ETIMEDOUT = -5, /* a bounded wait ran out */
  FFPAT_ECANCELED = -6, /* server request cancelled */
  FFPAT_PENDING = 1     /* server request not finished yet */
} ffpat_status;

typedef enum {
  FFPAT_FP64 = 0,      /* double everywhere */
  FFPAT_FP32 = 1,      /* float wavefields, three-term leapfrog */
  FFPAT_FP32_KAHAN = 2 /* float wavefields, increment form with a Kahan-compensated position update */
} ffpat_precision;

typedef enum {
  FFPAT_PRECOND_NONE = 0, /* Lambda = I (Algorithm 7 / 8 without preconditioning) */
  FFPAT_PRECOND_RAMP = 1  /* Lambda: F Lambda Phi = |omega| / (4 pi) F Phi along xi (Sec. 3.1) */
} ffpat_precond;

typedef enum {
  FFPAT_REG_L1_POS = 0, /* R = ||h||_1 + indicator(h >= 0): h+ = max(f - s lambda, 0) */
  FFPAT_REG_GRAD2 = 1   /* R = 1/2 |grad h|^2 (the paper's experiments, Sec. 5): see ffpat_prox_grad */
} ffpat_regulariser;

/* Problem statement (Problem 1 of Sec. 2.1 with full data). */
typedef struct {
  int32_t n;         /* grid points per axis N (1..2048) of the source box; N^3 volume */
  double T;          /* final time T > 0 */
  double cfl;        /* dt <= cfl dx / c_max; 0 < cfl <= 0.5 (stability of L4 leapfrog) */
  int32_t n_angles;  /* number of projection directions, >= 1 */
  int32_t precision; /* ffpat_precision */
  int32_t precond;   /* ffpat_precond (used by ffpat_fb_solve and ffpat_opnorm) */
  int32_t pad;       /* cells of padding on every side of the wave grid (0..2048; see below) */
} ffpat_problem;

/* Per-solve summary of Algorithm 8.  objective = 1/2 <Lambda r, r> + lambda ||h_k||_1
 * and resid_norm = ||r||_2 with r = A h_k - g, both for the last iteration's
 * input h_k; rel_change = ||h_{k+1} - h_k|| / max(||h_k||, 1e-300). */
typedef struct {
  int32_t iters_done;
  double objective;
  double resid_norm;
  double rel_change;
  double step;      /* step size s actually used */
  double opnorm_sq; /* power-iteration estimate of ||Lambda^1/2 A||^2 (0 if not run) */
} ffpat_fb_stats;

/* Description of the last error on this host thread ("" if none). */
const char *ffpat_last_error(void);

/* Library version string. */
const char *ffpat_version(void);

/* Workspace bytes needed by every entry point below for this problem
 * (0 if the problem is invalid; see ffpat_last_error). */
size_t ffpat_workspace_bytes(const ffpat_problem *problem);

/* Host-only: time discretisation for a given c_max (the wave model of Sec. 2.1):
 * writes Nt, dt and Ns (ray samples).  Any output pointer may be NULL. */
int ffpat_problem_info(const ffpat_problem *problem, double c_max, int32_t *nt, double *dt,
                       int32_t *n_samples);

/* Host-only: the angle table theta_j = pi j / n_angles as cos_sin[2 j] = cos,
 * cos_sin[2 j + 1] = sin (host libm, double), n_angles entries. */
int ffpat_debug_tables(const ffpat_problem *problem, double *cos_sin);

/* Device: index arithmetic of `count` ray samples (j, k, m) given as int32
 * triples in jkm (device); writes the lower-left bilinear corner (i0, j0) to
 * ij and the fractions (fx, fy) to f (device, double).  This is the very
 * device function the projection of an FP64 problem uses. */
int ffpat_debug_samples(const ffpat_problem *problem, int32_t count, const int32_t *jkm,
                        int32_t *ij, double *f, void *stream);

/* g = P W h  (eq. (4) composed with W of eq. (3)).  c: Nw^3, h: N^3; g: n_angles Nw^2. */
int ffpat_forward(const ffpat_problem *problem, const void *c, const void *h, void *g, void *ws,
                  size_t ws_bytes, void *stream);

/* h = W^T P^T g: the exact transpose of ffpat_forward (the discrete form of
 * W_T^* X^* of Sec. 3.1, with the sound speed inside the Laplacian). */
int ffpat_adjoint(const ffpat_problem *problem, const void *c, const void *g, void *h, void *ws,
                  size_t ws_bytes, void *stream);

/* out = W in (transpose = 0; in: N^3 box source, out: Nw^3 field) or
 * out = W^T in (transpose = 1; in: Nw^3, out: N^3), eq. (3).  out may be in
 * itself (in place). */
int ffpat_wave(const ffpat_problem *problem, const void *c, const void *in, void *out,
               int32_t transpose, void *ws, size_t ws_bytes, void *stream);

/* g = P p (eq. (4)) on the data grid; p: Nw^3, g: n_angles Nw^2.  No workspace. */
int ffpat_project(const ffpat_problem *problem, const void *p, void *g, void *stream);

/* h = P^T g, the exact transpose of ffpat_project (backprojection X^* of Sec. 3.1). */
int ffpat_backproject(const ffpat_problem *problem, const void *g, void *h, void *stream);

/* out = Lambda r along every detector row (Sec. 3.1): linear convolution with
 * t_0 = 1/(8 dxi), t_d = -1/(2 pi^2 d^2 dxi) for odd d, 0 for even d != 0. */
int ffpat_ramp(const ffpat_problem *problem, const void *r, void *out, void *stream);

/* out = prox of the gradient regulariser, (I + a D^T D)^{-1} f with
 * a = s lambda / dx^2 (N^3 each; in place allowed): the minimiser of
 * 1/2 ||h - f||^2 + s lambda R(h), R(h) = 1/2 <D h, D h> / dx^2, where D takes
 * the forward differences between neighbouring cells of the box along each
 * axis and none across its faces (h lives on the box: zero-flux faces).
 * Solved exactly by the orthonormal DCT-II along x, y, z (eigenvalues
 * 4 sin^2(pi k / 2N) per axis).  a >= 0.  Uses the workspace. */
int ffpat_prox_grad(const ffpat_problem *problem, double a, const void *f, void *out, void *ws,
                    size_t ws_bytes, void *stream);

/* Power iteration v <- A^T Lambda A v / ||.|| from v0 (device, N^3) for `iters`
 * steps; *opnorm_sq = the estimate of the largest eigenvalue of A^T Lambda A.
 * Synchronises the stream. */
int ffpat_opnorm(const ffpat_problem *problem, const void *c, const void *v0, int32_t iters,
                 double *opnorm_sq, void *ws, size_t ws_bytes, void *stream);

/* Algorithm 8 (Sec. 3.2) with R = ||h||_1 + indicator(h >= 0):
 *   r_k = A^T Lambda (A h_k - g),  h_{k+1} = max(h_k - s r_k - s lambda, 0).
 * h_inout: h_0 on entry (zeros per Algorithm 8), the last iterate on return.
 * step <= 0: s = 1 / L with L from 20 power iterations from a fixed
 * pseudo-random start.  tol > 0 stops once rel_change < tol (one 8-byte
 * device-to-host read per iteration); tol = 0 runs max_iters with no host
 * round trip inside the loop.  history (host, nullable): 4 doubles per
 * iteration (objective, resid_norm, rel_change, ||h_{k+1}||).
 * Synchronises the stream before returning. */
int ffpat_fb_solve(const ffpat_problem *problem, const void *c, const void *g, double lambda,
                   double step, int32_t max_iters, double tol, void *h_inout,
                   ffpat_fb_stats *stats, double *history, void *ws, size_t ws_bytes,
                   void *stream);

/* ---- The two-step method (Algorithm 9, Sec. 4.1), the paper's comparison:
 * first g = X^{-1} G plane by plane, then FB on 1/2 ||W h - g||^2 + lambda R. */

/* out (Nw^3) = X^{-1} G = X^* Lambda G (Sec. 3.1: filtered backprojection in
 * every plane z = const), discretised as (2 pi / (n_angles dx)) P^T Lambda G:
 * 2 pi / n_angles is the angle weight of the backprojection over S^1 (the data
 * over [0, pi) count twice) and 1/dx undoes the sample length of P^T. */
int ffpat_fbp(const ffpat_problem *problem, const void *G, void *out, void *ws, size_t ws_bytes,
              void *stream);

/* Algorithm 9 with R = ||h||_1 + indicator(h >= 0): g = X^{-1} G, then
 * h_{k+1} = max(h_k - s W^T (W h_k - g) - s lambda, 0).  Arguments, step rule
 * (power iteration on W^T W when step <= 0), tol and history as in
 * ffpat_fb_solve; the objective is 1/2 ||W h_k - g||^2 + lambda ||h_k||_1. */
int ffpat_fb_two_step(const ffpat_problem *problem, const void *c, const void *G, double lambda,
                      double step, int32_t max_iters, double tol, void *h_inout,
                      ffpat_fb_stats *stats, double *history, void *ws, size_t ws_bytes,
                      void *stream);

/* Algorithm 8 for limited data and a bounded source (Problem 1 with
 * M_theta != R^2; the source support V of the wave model, Sec. 2.1):
 *   r_k = A^T chi_M Lambda chi_M (A h_k - g),
 *   h_{k+1} = chi_V max(h_k - s r_k - s lambda, 0),
 * i.e. FB on 1/2 <Lambda chi_M (A h - g), chi_M (A h - g)> + lambda (||h||_1
 * + indicator(h >= 0) + indicator(supp h in V)).  mask (n_angles Nw^2) and
 * support (N^3) are device arrays of 0/1 values of the problem's element
 * type, or NULL for full data / the whole grid (then this is
 * ffpat_fb_solve).  The power-iteration step uses the masked operator.
 * regulariser (ffpat_regulariser): FFPAT_REG_GRAD2 replaces the shrinkage by
 * h_{k+1} = prox_{s lambda R}(h_k - s r_k) with R = 1/2 |grad h|^2
 * (ffpat_prox_grad), the objective then carrying lambda R(h_k); it takes no
 * support (EINVAL). */
int ffpat_fb_solve_ex(const ffpat_problem *problem, const void *c, const void *g,
                      const void *mask, const void *support, int32_t regulariser, double lambda,
                      double step, int32_t max_iters, double tol, void *h_inout,
                      ffpat_fb_stats *stats, double *history, void *ws, size_t ws_bytes,
                      void *stream);

/* Algorithm 9 with the choice of regulariser (ffpat_fb_two_step is
 * FFPAT_REG_L1_POS): with FFPAT_REG_GRAD2,
 * h_{k+1} = prox_{s lambda R}(h_k - s W^T (W h_k - g)), R = 1/2 |grad h|^2,
 * the method of the paper's experiments (lambda = 0.5, s = 0.2 there). */
int ffpat_fb_two_step_ex(const ffpat_problem *problem, const void *c, const void *G,
                         int32_t regulariser, double lambda, double step, int32_t max_iters,
                         double tol, void *h_inout, ffpat_fb_stats *stats, double *history,
                         void *ws, size_t ws_bytes, void *stream);

/* Instrumentation.  While enabled, every wave time loop records CUDA events on
 * its stream around its leapfrog launches; ffpat_profile_read synchronises
 * those events and returns the leapfrog launches and steps timed, their total
 * milliseconds, and the algorithmic HBM bytes they move: one pass of the state
 * per launch (16 B FP32, 28 B FP32-Kahan, 32 B FP64 per grid point), where a
 * two-step FP32-Kahan launch advances two steps in its one pass.  Reading
 * resets. */
typedef struct {
  int64_t step_launches;
  double step_ms;
  double step_bytes;
  int64_t kernel_launches; /* all kernels this library launched since the last reset */
  int64_t steps;           /* leapfrog steps inside the timed launches */
} ffpat_profile;
int ffpat_profile_enable(int32_t on);
int ffpat_profile_read(ffpat_profile *out);

/* Total kernels launched by this library since load (monotone counter). */
int64_t ffpat_launch_count(void);

/* Choice of leapfrog kernel (process-wide): 0 = automatic (the TMA-fed kernels
 * when N % 4 == 0 for float or N % 2 == 0 for double and all arrays are
 * 16-byte aligned -- for FP32 and FP32-Kahan the whole time loop in one
 * cooperative launch where its work items fit the GPU at once (N <= 128 on
 * GB300) and the stream is not capturing, else two steps per pass for
 * 128 <= N <= 1624 -- else the plain 2.5D kernel), 1 = always the plain
 * kernel, 2 = the single-step TMA kernel, 3 = the two-step TMA kernels for
 * FP32 and FP32-Kahan (N <= 1624; single steps for FP64), 4 = the resident
 * time loop (FP32, FP32-Kahan);
 * 2, 3 and 4 fail with FFPAT_EINVAL where their kernel cannot be used.  All
 * compute the same steps bit for bit (FP32, FP32-Kahan) or up to rounding
 * order (FP64 plain against TMA); this exists for testing and measurement. */
int ffpat_set_stencil_path(int32_t path);

/* Device status word of the library's kernels: 0, or the negative status of
 * the first device-side failure since the last clear (a bounded wait that ran
 * out sets FFPAT_ETIMEDOUT).  Synchronises the device; clear != 0 resets it. */
int ffpat_device_status(int32_t clear);

/* Failure-detection check: launch a one-CTA kernel that waits on an mbarrier
 * nothing will complete, with the same bounded wait as the stencil kernels
 * (`microseconds` of SM clock, at most 2 s); the wait runs out and the kernel
 * records FFPAT_ETIMEDOUT in the device status word and returns, so the CUDA
 * context stays usable.  Synchronises the stream. */
int ffpat_debug_wait_timeout(int32_t microseconds, void *stream);

/* Arithmetic throughput probe (not part of the method; the paper has no
 * counterpart): the fused multiply-add rate of one pipe of the current
 * device, kind 0 = FP64 (fma), 1 = FP32 (fmaf), 2 = packed two-lane FP32
 * (fma.rn.f32x2, the form the FP32 stencils use), measured with CUDA events
 * on `stream` over a grid that fills every SM with eight independent FMA
 * chains per thread; *flops_per_s receives the best of three launches
 * (2 operations per FMA and lane).  Kernels that are bound by arithmetic
 * rather than memory report their fraction of this measured rate.
 * Synchronises the stream; FFPAT_EINVAL for another kind or a null output. */
int ffpat_debug_fma_rate(int32_t kind, double *flops_per_s, void *stream);

/* ---- Differentiation of g = P W(c) h with respect to h and the sound speed c.
 * The forward pass runs the three-term leapfrog (FFPAT_FP32_KAHAN problems
 * take FP32 three-term steps on this path) and saves (p^{sk}, p^{sk+1}) every
 * k = `every` steps into the caller's checkpoint buffer; the backward pass
 * runs the transposed recurrence from P^T grad_g, recomputing each k-step
 * segment from its checkpoint, and returns grad_h = A^T grad_g and
 * grad_c = d<grad_g, A(c) h>/dc with dt held fixed (Nt is piecewise constant
 * in c).  The paper differentiates only in h (Sec. 3.1); the c-gradient is the
 * same discrete adjoint carried through kappa = (c dt / dx)^2. */

/* The differentiated operator needs pad = 0 (the box is the wave grid). */

/* Checkpoint buffer bytes for Nt steps (ffpat_problem_info) and interval
 * `every`: (2 ceil(Nt / every) + every + 2) volumes; 0 if invalid. */
size_t ffpat_ckpt_bytes(const ffpat_problem *problem, int32_t nt, int32_t every);

/* g = P W h with checkpoints (device buffers as for ffpat_forward; ckpt is
 * caller-owned device memory of ffpat_ckpt_bytes bytes, 256-byte aligned). */
int ffpat_forward_ckpt(const ffpat_problem *problem, const void *c, const void *h, void *g,
                       int32_t every, void *ckpt, size_t ckpt_bytes, void *ws, size_t ws_bytes,
                       void *stream);

/* Backward pass after ffpat_forward_ckpt with the same problem, c, `every`
 * and checkpoint buffer: grad_h (N^3, nullable) = A^T grad_g and grad_c (N^3,
 * nullable) = d<grad_g, A(c) h>/dc. */
int ffpat_backward(const ffpat_problem *problem, const void *c, const void *grad_g, void *grad_h,
                   void *grad_c, int32_t every, void *ckpt, size_t ckpt_bytes, void *ws,
                   size_t ws_bytes, void *stream);

/* ---- Serving: many Algorithm-8 solves in flight on one GPU (continuous batching).
 * A server owns a worker thread and a CUDA stream on the device that is
 * current at creation.  Requests (FFPAT_FP32_KAHAN problems with N % 4 == 0
 * and pad = 0; any N, angle count, T) wait in a FIFO queue and are admitted while a slot is
 * free and their device memory fits the HBM budget; every launch of the
 * leapfrog kernel advances all admitted requests that are inside a wave phase
 * by one step, and requests that arrive while others run join at the next
 * step.  Each request runs exactly the kernels of ffpat_fb_solve, so its
 * result does not depend on the other requests.  The paper has no serving
 * layer; this is the deployment side of Algorithm 8. */
typedef struct ffpat_server ffpat_server;

typedef struct {
  int64_t completed, failed, cancelled;
  double p50_ms, p99_ms, mean_ms, max_ms; /* submit-to-completion latency */
  double point_steps;                     /* leapfrog point-steps of completed requests */
  int64_t ticks;                          /* batched leapfrog launches so far */
  int32_t active, queued;
  size_t hbm_in_use;                      /* bytes held by admitted requests */
} ffpat_serving_stats;

/* Create a server: hbm_budget_bytes bounds the device memory of admitted
 * requests (each needs ffpat_workspace_bytes + 8 N^3 + 4 n_angles N^2 bytes);
 * max_slots (1..28) bounds how many run at once. */
int ffpat_server_create(size_t hbm_budget_bytes, int32_t max_slots, ffpat_server **out);

/* Queue a reconstruction: c_host (N^3 float) and g_host (n_angles N^2 float)
 * are HOST arrays, copied before the call returns; h_0 = 0; `iters` FB
 * iterations with the given lambda; step <= 0 runs 20 power iterations first
 * (as ffpat_fb_solve does).  Returns a ticket.  FFPAT_EBUSY if the queue holds
 * 4096 requests; FFPAT_EINVAL if the request can never fit the budget. */
int ffpat_submit(ffpat_server *server, const ffpat_problem *problem, const void *c_host,
                 const void *g_host, double lambda, double step, int32_t iters, uint64_t *ticket);

/* Non-blocking: FFPAT_PENDING while the request runs; FFPAT_OK once done (the
 * iterate is copied to h_out_host, N^3 float, and *stats filled; the ticket is
 * then released); FFPAT_ECANCELED or another error if it failed. */
int ffpat_poll(ffpat_server *server, uint64_t ticket, void *h_out_host, ffpat_fb_stats *stats);

/* Cancel a queued or running request (only that request is affected). */
int ffpat_cancel(ffpat_server *server, uint64_t ticket);

/* Latency percentiles and throughput counters; returns the worker's fatal
 * error code (0 if none). */
int ffpat_server_stats(ffpat_server *server, ffpat_serving_stats *out);

/* Stop the worker (queued and running requests are cancelled) and free all. */
int ffpat_server_destroy(ffpat_server *server);

/* g = P W h like ffpat_forward, for callers that cannot allocate device
 * memory or pass a workspace (code inside an application that owns all device
 * memory, fixed-budget or real-time pipelines that must not enter an
 * allocator).  The paper has no counterpart; this is a deployment variant.
 * Its scratch is a 32 MiB file-scope device array, committed when the
 * library's device code is loaded on a device and held until exit; under
 * CUDA's lazy module loading (the default) that load happens during the first
 * call on each device, which may allocate once; later calls allocate nothing.
 * Problems whose ffpat_workspace_bytes exceeds 32 MiB fail with FFPAT_EINVAL
 * (a wave grid N + 2 pad <= 64 with up to 180 angles fits every precision;
 * without padding that is N <= 64); a device index >= 64 fails with
 * FFPAT_EINVAL.  The first call on a device looks up the array's device
 * address (with that device current); make it before any stream capture.
 * All calls on a device share the array: calls that overlap on the GPU race
 * and must be serialised by the caller.  Nothing in the array needs to start
 * at zero; it keeps the last call's contents. */
int ffpat_forward_noalloc(const ffpat_problem *problem, const void *c, const void *h, void *g,
                          void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FFPAT_H */
