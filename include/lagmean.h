/*
 * lagmean.h -- C ABI of the GB300 library for on-the-fly Lagrangian means of a
 * doubly periodic pseudospectral rotating shallow-water flow.
 *
 * Method: Kafiabad & Vanneste, "Computing Lagrangian means" (JFM 2023,
 * arXiv 2208.02682).  The library advances the shallow-water equations
 * (Sec. 4.2, Eq. (sw_eqs_dimless), with f0 = 1/Ro, c2 = gH = 1/Fr^2 and a
 * hyperviscosity -nu8 |k|^8 in place of the Laplacian) together with the
 * Lagrangian-mean PDEs of one averaging interval [tau, tau + T]:
 *   Strategy 1 (Sec. 3.1, 4.1): Eq. (gtilde-evol), (d_t + u.grad) g = f with
 *     g = (t - tau) f~, and the mean positions Xi^{-1} of Eq. (Xi-1evol)
 *     carried as the periodic displacement D = (t - tau)(x - Xi^{-1});
 *   Strategy 2 (Sec. 3.2, 4.2): Eqs. (xi_evol), (barf_xi) for the displacement
 *     xi = Xi - x and g = (t - tau) fbar, with u and f interpolated bilinearly
 *     at x + xi;
 *   Eulerian means, Eq. (ave).
 * Intervals are computed one after another, each from its own zero state
 * (Sec. 2: tau_n = n T).  Time stepping is classical RK4 with an integrating
 * factor for the hyperviscosity; all fields share the RK stages.
 *
 * Conventions
 *  - Grid: N x N points on [0, 2 pi)^2, N a power of two in [16, 2048];
 *    x_i = 2 pi i / N.  Physical arrays are row-major with y the slow index:
 *    a[j * N + i] is the value at (x_i, y_j).
 *  - Every call returns an int status (SW_OK = 0).  No C++ exception crosses
 *    the ABI.  sw_last_error() gives a message for the last failing call on a
 *    handle.  A NULL handle argument gives SW_EINVAL (sw_destroy: no-op).
 *  - Device work is issued asynchronously on the stream given to sw_create
 *    (a cudaStream_t passed as void*; NULL = the legacy default stream).
 *    Calls that return data to host memory synchronise that stream.
 *  - One host thread at a time per handle.  The library owns all device
 *    memory of a handle; sw_destroy releases it.
 *  - Precision: SW_PREC_FP64 runs every step in FP64.  SW_PREC_FP32 runs the
 *    transforms, products and advection in FP32 with compensated (Kahan)
 *    summation of the Lagrangian-mean and Eulerian accumulators; the
 *    end-of-interval division, mean-position recovery, initial transform and
 *    invariant reductions are FP64 in both modes.
 */
#ifndef LAGMEAN_H
#define LAGMEAN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define SW_OK 0
#define SW_EINVAL 1   /* invalid argument (value given in sw_last_error)      */
#define SW_ENOMEM 2   /* device or host allocation failed                      */
#define SW_EBUSY 3    /* sw_step while an averaging interval is open           */
#define SW_ERANGE 4   /* more steps than remain in the open interval           */
#define SW_ESTATE 5   /* call not valid in the handle's current state          */
#define SW_ETIMEOUT 6 /* a bounded device wait gave up                         */
#define SW_ECUDA 7    /* a CUDA runtime call failed (message in sw_last_error) */

/* ---- enumerations ------------------------------------------------------- */
#define SW_PREC_FP64 0
#define SW_PREC_FP32 1

#define SW_MODEL_SW 0        /* rotating shallow water, Eq. (sw_eqs_dimless) */
#define SW_MODEL_KINEMATIC 1 /* test model: the state is passively advected
                                by the constant velocity (adv_x, adv_y), and
                                the Lagrangian-mean equations see u = adv   */
#define SW_MODEL_EULER2D 2   /* two-dimensional incompressible flow, the test
                                flow of Sec. 4.1: d_t zeta + div(u zeta) = 0
                                with u = -d_y psi, v = d_x psi, lap psi = zeta.
                                The third field of an initial condition or of
                                sw_get_fields is zeta (no depth); the u, v
                                planes of an initial condition are ignored
                                (derived from zeta).  Lagrangian means of
                                zeta, u and v only; sw_diag is SW_EINVAL.
                                f0, c2 are unused.                            */

/* Lagrangian-mean field mask (lm_params.fields) */
#define LM_ZETA 1 /* relative vorticity zeta = d_x v - d_y u              */
#define LM_H 2    /* depth h                                             */
#define LM_U 4    /* velocity u                                          */
#define LM_V 8    /* velocity v                                          */
#define LM_Q 16   /* potential vorticity q = (f0 + zeta)/h (Sec. 4.2.1)  */
#define LM_POS 32 /* mean positions (always on for Strategy 2)            */

typedef struct sw_handle sw_handle;

/* Model and discretisation parameters (sw_create). */
/* Time steppers, all with the diagonal integrating factor exp(-nu |k|^2p dt)
 * of the viscous term:
 *   SW_STEP_RK4    classical four-stage Runge-Kutta (the default);
 *   SW_STEP_HEUN   Heun's method, the paper's stepper in Sec. 4.1:
 *                  y1 = E^2 (y + dt a), y' = E^2 y + dt/2 (E^2 a + b);
 *   SW_STEP_EULER  forward Euler, the paper's stepper in Sec. 4.2.1:
 *                  y' = E^2 (y + dt a);
 * (a, b: right-hand sides at the stages, E = exp(-nu |k|^2p dt/2)).  The
 * Lagrangian-mean fields share the stages with the dynamics.
 * Viscosity: SW_VISC_HYPER8 -nu |k|^8 (the default), SW_VISC_LAPLACE
 * -nu |k|^2 (the paper's Laplacian, Eq. (sw_momentum_dimless)), with
 * nu = nu8 on u, v, h and lm_nu8 on the Lagrangian-mean fields. */
#define SW_STEP_RK4 0
#define SW_STEP_HEUN 1
#define SW_STEP_EULER 2
#define SW_VISC_HYPER8 0
#define SW_VISC_LAPLACE 1

typedef struct sw_params {
  int32_t N;         /* grid points per side: power of two, 16..2048        */
  int32_t precision; /* SW_PREC_FP64 or SW_PREC_FP32                        */
  int32_t model;     /* SW_MODEL_SW or SW_MODEL_KINEMATIC                    */
  int32_t stepper;   /* SW_STEP_RK4 (0), SW_STEP_HEUN or SW_STEP_EULER       */
  double dt;         /* time step, > 0                                      */
  double f0;         /* Coriolis parameter (1/Ro)                           */
  double c2;         /* squared gravity-wave speed g H (1/Fr^2), >= 0        */
  double nu8;        /* viscosity coefficient on u, v, h (see visc), >= 0    */
  double lm_nu8;     /* viscosity coefficient on the Lagrangian-mean fields  */
  double adv_x;      /* advection velocity of SW_MODEL_KINEMATIC            */
  double adv_y;
  int32_t visc;      /* SW_VISC_HYPER8 (0) or SW_VISC_LAPLACE               */
  int32_t reserved;  /* must be 0                                           */
} sw_params;

/* Discretisation of the mean equations (lm_params.scheme):
 *   LM_SCHEME_COUPLED   the mean fields share every stage of the dynamics'
 *                       stepper (the default);
 *   LM_SCHEME_XI_FIRST  the paper's scheme for Strategy 2 (Sec. 4.2: xi is
 *                       updated first and the updated xi is used for gbar;
 *                       Sec. 4.2.1: forward Euler, the mean equations'
 *                       step twice the dynamics' step): step 2m advances xi
 *                       by 2 dt from the flow at t_2m, step 2m+1 advances
 *                       gbar by 2 dt with xi_{m+1} (advecting velocity
 *                       xi_{m+1}/s_{m+1}) and the flow at t_2m+1; Eulerian
 *                       means step with dt.  Needs strategy 2,
 *                       SW_STEP_EULER and an even n_steps (else SW_EINVAL). */
#define LM_SCHEME_COUPLED 0
#define LM_SCHEME_XI_FIRST 1

/* One averaging interval (lmean_begin). */
typedef struct lm_params {
  int32_t strategy; /* 1 or 2                                               */
  int32_t fields;   /* LM_* mask; at least one of ZETA,H,U,V,Q or POS       */
  int32_t eulerian; /* nonzero: also accumulate Eulerian means of `fields`   */
  int32_t scheme;   /* LM_SCHEME_COUPLED (0) or LM_SCHEME_XI_FIRST            */
  int64_t n_steps;  /* interval length T = n_steps * dt, >= 1               */
} lm_params;

/* Outputs of lmean_end: FP64 physical N x N arrays, caller-owned.  A NULL
 * pointer skips that output.  Fields not in the interval's mask must be NULL.
 * Strategy 1: zeta..q = f~^L = g(tau+T)/T indexed by the end position x,
 *   pos = Xi^{-1}(x, tau+T) = x - D/T (the mean position of the particle
 *   that is at x at tau+T); Strategy 2: zeta..q = fbar^L indexed by the mean
 *   position x, pos = Xi(x, tau+T) = x + xi.  e_* = Eulerian means E/T. */
typedef struct lm_result {
  double *zeta, *h, *u, *v, *q;
  double *pos_x, *pos_y;
  double *e_zeta, *e_h, *e_u, *e_v, *e_q;
  int32_t on_device; /* 1: all pointers are device memory; 0: host memory */
  int32_t reserved;
} lm_result;

/* Create a handle from a physical initial condition.
 * The state is the shallow-water system of Sec. 4.2, Eq. (sw_eqs_dimless)
 * (momentum Eq. (sw_momentum_dimless), mass Eq. (sw_mass_dimless)), in the
 * paper's pseudospectral discretisation with 2/3 dealiasing (Sec. 4.1,
 * 4.2.1): the state is the truncated spectrum of u, v and the depth.
 * ic_uvh: 3*N*N doubles (u, then v, then h), host memory if ic_on_device == 0
 * else device memory; copied, not retained.  The fields are transformed and
 * truncated to the 2/3 box |kx|, |ky| <= floor((N-1)/3).
 * stream: cudaStream_t for all device work of this handle (NULL: default).
 * Errors: SW_EINVAL (bad parameter), SW_ENOMEM, SW_ECUDA.  On error *out is
 * set to NULL and nothing is leaked. */
int sw_create(const sw_params* p, const double* ic_uvh, int ic_on_device,
              void* stream, sw_handle** out);

/* Release all memory of a handle (synchronises its stream).  NULL: no-op.
 * (Sec. 2: each averaging interval is computed independently, so a handle
 * holds no state beyond the current dynamics and its open interval; an open
 * interval is discarded.) */
void sw_destroy(sw_handle* h);

/* Advance the shallow-water state only, Eq. (sw_eqs_dimless), by nsteps >= 0
 * steps of the handle's stepper (sw_params.stepper: RK4, or the paper's Heun
 * of Sec. 4.1 or forward Euler of Sec. 4.2.1, each with the integrating
 * factor of the viscous term).  SW_EBUSY while an averaging interval is
 * open.  Asynchronous. */
int sw_step(sw_handle* h, int64_t nsteps);

/* Open an averaging interval at tau = current time: zero the Lagrangian-mean
 * state (g = D = 0, or xi = g = 0, Sec. 3.1-3.2 initial conditions; Eulerian
 * accumulators = 0).  SW_ESTATE if an interval is already open. */
int lmean_begin(sw_handle* h, const lm_params* lp);

/* Advance the dynamics and the open interval together by nsteps >= 0 steps
 * of the handle's stepper (on-the-fly computation, Sec. 5): Strategy 1,
 * Eq. (gtilde-evol) and the displacement form of Eq. (Xi-1evol); Strategy 2,
 * Eqs. (xi_evol), (barf_xi); Eulerian accumulators, Eq. (ave).  SW_ERANGE if nsteps exceeds the
 * steps remaining, SW_ESTATE if no interval is open.  Asynchronous: the
 * steps are replays of a captured CUDA graph on the handle's stream. */
int lmean_step(sw_handle* h, int64_t nsteps);

/* Close a completed interval (remaining steps == 0, else SW_ESTATE) and write
 * the means (see lm_result) in FP64: Strategy 1, f~^L = g(tau+T)/T (Sec.
 * 4.1, the division that follows Eq. (gtilde-evol)) and the mean positions
 * Xi^{-1}(x, tau+T) = x - D/T (Sec. 3.1, Eq. (Xi-1evol)); Strategy 2,
 * fbar^L = g/T and the lift map Xi = x + xi (Sec. 3.2, Eq. (Xievol); Sec.
 * 4.2, Eqs. (xi_evol), (barf_xi)); Eulerian means E/T, Eq. (ave).  With host outputs it synchronises the
 * handle's stream; with device outputs (on_device = 1) it returns once the
 * work is enqueued on that stream. */
int lmean_end(sw_handle* h, const lm_result* out);

/* Steps remaining in the open interval (0 if none) and steps done. */
int lmean_progress(sw_handle* h, int64_t* done, int64_t* remaining);

/* Physical FP64 u, v, h of the current state into uvh (3*N*N doubles, host
 * if on_device == 0).  Synchronises. */
int sw_get_fields(sw_handle* h, double* uvh, int on_device);

/* Replace the shallow-water state by a physical initial condition (as in
 * sw_create).  SW_EBUSY while an interval is open. */
int sw_set_fields(sw_handle* h, const double* uvh, int on_device);

/* Invariants in FP64 with a deterministic reduction order:
 * out[0] = mass <h> (the k = 0 depth coefficient),
 * out[1] = energy <h |u|^2/2 + c2 h^2/2>,
 * out[2] = potential enstrophy <h q^2/2>, q = (f0 + zeta)/h.
 * Means over the N x N grid.  Synchronises. */
int sw_diag(sw_handle* h, double out[3]);

/* Checkpoint of the complete state (dynamics, open interval, compensation
 * terms, step counters) as an opaque blob.  Call with blob == NULL to get
 * the size in *size; then with a buffer of at least that size.  Restoring
 * with sw_set_state on a handle created with the same sw_params continues
 * bit-for-bit as if uninterrupted.  SW_EINVAL on a size or parameter
 * mismatch. */
int sw_get_state(sw_handle* h, void* blob, size_t* size);
int sw_set_state(sw_handle* h, const void* blob, size_t size);

/* Model time of the current state (dt * steps taken since creation). */
int sw_time(sw_handle* h, double* t);

/* Kernel classes reported by sw_kernel_times. */
#define SW_K_COL_INV 0  /* column pass: spectral -> mixed (derivatives, inverse y-FFT) */
#define SW_K_ROW_INV 1  /* row pass: mixed -> physical base fields (u, v, h, zeta, xi) */
#define SW_K_ROW_PROD 2 /* row pass: inverse x-FFT, products, forward x-FFT        */
#define SW_K_COL_FWD 3  /* column pass: forward y-FFT and 2/3 mask                  */
#define SW_K_UPDATE 4   /* right-hand sides and RK4 integrating-factor update       */
#define SW_K_PHYS_Q 5   /* potential vorticity in the gather buffer (Strategy 2)    */
#define SW_K_COUNT 8

/* Per-kernel device times of the stepping kernels.  Runs nsteps >= 1 RK4
 * steps of the current configuration (dynamics only, or the open interval,
 * whose remaining steps must allow it), advancing the state exactly as
 * sw_step / lmean_step do, but with each kernel launched on its own and
 * bracketed by CUDA events on the handle's stream.  For each class k:
 * ms[k] = summed device milliseconds, launches[k] = launches, bytes[k] =
 * summed algorithmic bytes (the distinct inputs each launch must read and the
 * outputs it must write; L2 hits are not subtracted).  Synchronises. */
int sw_kernel_times(sw_handle* h, int64_t nsteps, double ms[SW_K_COUNT],
                    int64_t launches[SW_K_COUNT], double bytes[SW_K_COUNT]);

/* Number of CUDA kernels this handle has launched since creation (graph
 * replays count each kernel node). */
int sw_launch_count(sw_handle* h, int64_t* count);

/* ---- batches: many runs in the same launches ---------------------------------
 * A batch steps several handles together: every kernel of an RK stage is one
 * launch over all members (a device table of per-run descriptors maps each
 * block to its run), and the steps replay from captured CUDA graphs.  Members
 * may differ in grid size, strategy, field set and interval state; each
 * member's arithmetic is the same as when it steps alone, so its results are
 * bit-for-bit the same alone and in the batch.  A batch does not own its
 * members: destroy the batch before any member.  Members must share the
 * precision and the stream they were created with; grids of different sizes
 * must all lie in 64..512 (larger grids batch only with their own size).
 * Calls on member handles (lmean_begin, lmean_end, sw_get_fields, ...)
 * remain valid between batch steps; the batch re-reads changed members
 * before its next step. */
typedef struct sw_batch sw_batch;

/* Errors: SW_EINVAL (empty, NULL or repeated handle, mixed precision or
 * stream, incompatible block shapes), SW_ENOMEM, SW_ECUDA.  The message of
 * a failing create is given by sw_last_error(NULL). */
int sw_batch_create(sw_handle* const* handles, int n, sw_batch** out);

/* Advance every member by nsteps >= 0 steps of the members' common stepper
 * (its dynamics, and its open interval if it has one).  SW_ERANGE if nsteps exceeds the steps remaining
 * in a member's open interval (nothing is stepped then).  Asynchronous. */
int sw_batch_step(sw_batch* b, int64_t nsteps);

/* Autotuner: times the row-pass launch shapes (points per block 256, 512,
 * 1024 or 2048, as long as every member fits; product pairs per block 1, 2, 3
 * or all; choice = 4 * points index + pairs index) on trial_steps >= 1
 * replayed steps each (after as many untimed ones), keeps the fastest for all members and returns its
 * index in *choice (may be NULL).  The members' states are saved before the trials and
 * restored after them (temporary device copies).  Synchronises. */
int sw_batch_tune(sw_batch* b, int trial_steps, int* choice);

/* Set the row-pass launch shape that sw_batch_tune would pick as `choice`
 * (4 * points index + pairs index, as above) without timing anything: for
 * callers that replay a shape tuned earlier, and for tests that must cover
 * every shape.  The members' arithmetic and results do not depend on it.
 * SW_EINVAL if choice is outside 0..15 or its points per block are fewer
 * than the largest member's N. */
int sw_batch_set_shape(sw_batch* b, int choice);

/* Kernels launched by the batch since its creation. */
int sw_batch_launch_count(sw_batch* b, int64_t* count);

/* Message for the last failing call on b. */
const char* sw_batch_last_error(sw_batch* b);

/* Release the batch (not its members; synchronises).  NULL: no-op. */
void sw_batch_destroy(sw_batch* b);

/* ---- serving: a continuous-batching request loop on one GPU -------------------
 * A server owns a host thread that admits Lagrangian-mean jobs (one averaging
 * interval each, any grid size, window, strategy and field set) in arrival
 * order while the job-state memory stays within hbm_budget bytes and the
 * active jobs within max_active; it keeps each admitted job's state resident
 * on the device, steps all active jobs together in batched launches
 * (sw_batch, grouped by compatible block shapes) in rounds of at most
 * chunk_steps steps, and completes each job as its interval ends (lmean_end
 * into the job's host buffers, then the job's device memory is released).
 * Jobs that arrive while others run join the next round.  A job's result is
 * the same as that of the same job run alone. */
typedef struct sw_server sw_server;

typedef struct sw_server_params {
  int32_t precision;   /* SW_PREC_FP32 or SW_PREC_FP64 for every job        */
  int32_t max_active;  /* concurrent jobs on the device, >= 1               */
  int32_t chunk_steps; /* RK4 steps per round, >= 1                          */
  int32_t reserved;    /* must be 0                                         */
  int64_t hbm_budget;  /* bytes of device memory for job state, > 0         */
  void* stream;        /* cudaStream_t for all job work; NULL: one private
                          stream per group, so that groups overlap          */
} sw_server_params;

typedef struct sw_job {
  sw_params params;      /* the job's grid and model (precision must match)   */
  lm_params lm;          /* its averaging interval                             */
  const double* ic_uvh;  /* host, 3*N*N doubles; read at admission            */
  lm_result out;         /* host output buffers (on_device = 0); written at
                            completion; must stay valid until then            */
  int64_t tag;           /* caller's identifier, returned with the job        */
} sw_job;

typedef struct sw_job_done {
  int64_t tag;
  int32_t status;        /* SW_OK, or the error that ended the job            */
  int32_t reserved;
  double t_submit;       /* seconds on the server clock (sw_server_clock)     */
  double t_admit;
  double t_done;
  int64_t bytes;         /* device bytes the job held                          */
} sw_job_done;

typedef struct sw_server_stats {
  int64_t submitted, completed, failed, active, queued;
  int64_t grid_point_steps; /* sum of N^2 * steps over completed jobs          */
  int64_t bytes_in_use, peak_bytes;
  int64_t rounds;           /* batched step rounds                             */
} sw_server_stats;

/* Start a server (its thread uses the calling thread's current device).
 * Errors: SW_EINVAL, SW_ENOMEM, SW_ECUDA (message via sw_last_error(NULL)). */
int sw_server_create(const sw_server_params* p, sw_server** out);

/* Queue a job (thread-safe; the descriptor is copied).  SW_EINVAL for an
 * invalid job or one whose state alone exceeds the budget, SW_ESTATE after
 * shutdown began. */
int sw_server_submit(sw_server* s, const sw_job* job);

/* Collect up to max finished jobs into done[0..*n); waits up to wait_ms
 * milliseconds for at least one if none is ready (0: do not wait). */
int sw_server_poll(sw_server* s, sw_job_done* done, int max, int* n, int wait_ms);

/* Counters (thread-safe). */
int sw_server_stats_get(sw_server* s, sw_server_stats* st);

/* Seconds since the server was created (monotonic). */
double sw_server_clock(sw_server* s);

/* Stop the loop: jobs still queued are dropped (their results are not
 * written), active jobs are released; then free the server.  NULL: no-op. */
void sw_server_destroy(sw_server* s);

/* Device bytes a handle with these parameters holds (the unit of the
 * server's HBM budget); 0 for invalid parameters. */
int64_t sw_state_bytes(const sw_params* p);

/* ---- allocation-free projection --------------------------------------------
 * The paper has no counterpart to this call; it is a library convenience.
 * Some callers cannot allocate device memory: code running where a
 * framework's caching allocator owns the GPU memory and no other allocation
 * is allowed, or latency-critical loops in which cudaMalloc/cudaFree (which
 * may synchronise the device) are not acceptable.  sw_project_static serves
 * them: it projects one physical field onto the 2/3-dealiased spectral box
 * (forward 2D FFT, keep |kx|, |ky| <= floor((N-1)/3), inverse 2D FFT), in
 * FP64, the same operation as sw_create followed by sw_get_fields, and it
 * allocates nothing.  Its scratch (mixed and spectral intermediates and the
 * twiddle table) is a file-scope static device array of
 * SW_PROJECT_STATIC_BYTES bytes that every GPU loading the library holds
 * until the process exits.
 *   in, out: device pointers to N*N doubles (row-major, y slow); they may
 *            be the same buffer.  The caller owns both.
 *   N:       power of two in [16, SW_PROJECT_STATIC_MAX_N]; larger N is
 *            rejected with SW_EINVAL (message via sw_last_error(NULL)).
 *   stream:  cudaStream_t (NULL: legacy default stream); the call is
 *            asynchronous on it.
 * The first call on a device resolves the device address of the static
 * array (cudaGetSymbolAddress) and sets kernel attributes, once per device;
 * make that first call before any stream capture.  Every call on a device
 * shares the one array, which keeps the last call's contents (each call
 * overwrites all it reads), so calls that overlap on the GPU (different
 * streams, or host threads) race and must be serialised by the caller.
 * Errors: SW_EINVAL, SW_ECUDA. */
#define SW_PROJECT_STATIC_MAX_N 512
#define SW_PROJECT_STATIC_BYTES (3u << 20)
int sw_project_static(const double* in, double* out, int N, void* stream);

/* ---- Strategy-1 remap to the mean-position grid ---------------------------
 * Sec. 3.1, Eq. (remap-strat1): f~^L(x, tau) = fbar^L(Xi^{-1}(x, tau+T), tau).
 * Strategy 1 (lmean_end with strategy 1) yields f~^L and the mean positions
 * Xi^{-1}(x, tau+T) on the grid x, i.e. fbar^L at scattered points.  This
 * call returns fbar^L on the grid y of mean positions by evaluating
 * f~^L at Xi(y), Xi = (Xi^{-1})^{-1} the lift map of Eq. (Xi-def): with the
 * periodic displacement d = x - Xi^{-1}(x), Xi(y) = y + xi(y) where xi is the
 * fixed point of xi = d(y + xi), iterated `iters` times from xi = 0, and
 * off-grid values of d and f~^L are bilinear interpolants (cell index
 * i + floor(xi/dx), periodic; the rule of the Strategy-2 solver, Sec.
 * 4.2.1).  The paper does not fix the interpolation; the fixed point
 * converges while Xi^{-1} stays invertible (|grad d| < 1), and `resid`
 * reports the last update so callers can see where it does not (the mean
 * positions cluster, Sec. 5).  FP64; every arithmetic step is rounded
 * separately (no fused multiply-add), so results are reproducible bit for bit.
 *   N:            power of two in [16, 4096].
 *   pos_x, pos_y: device, N*N doubles each (row-major, y slow): Xi^{-1} at the
 *                 grid points, as lmean_end reports it (unwrapped).
 *   nfields:      0..LM_REMAP_MAX_FIELDS.
 *   ftilde:       HOST array of nfields device pointers, N*N doubles each
 *                 (f~^L on the grid x).
 *   fbar:         HOST array of nfields device pointers, N*N doubles each,
 *                 written with fbar^L on the grid y.  Must not alias any
 *                 input (the gathers read neighbouring points).
 *   iters:        fixed-point iterations, 1..10000 (20 is ample for
 *                 |grad d| < 0.25).
 *   xi_x, xi_y:   device N*N doubles or NULL: Xi(y) = y + xi (unwrapped).
 *   resid:        device N*N doubles or NULL: max(|dxi_x|, |dxi_y|) of the last
 *                 iteration at each point.
 *   stream:       cudaStream_t (NULL: legacy default stream); asynchronous.
 * The caller owns every buffer.  Errors: SW_EINVAL (message via
 * sw_last_error(NULL)), SW_ECUDA. */
#define LM_REMAP_MAX_FIELDS 16
int lmean_remap(int N, const double* pos_x, const double* pos_y, int nfields, const double* const* ftilde,
                double* const* fbar, int iters, double* xi_x, double* xi_y, double* resid, void* stream);

/* ---- diagnostics ------------------------------------------------------------
 * Fields at given positions: out_k(y) = f_k(pos(y)) for every grid point y,
 * by the periodic bilinear rule of the Strategy-2 solver (Sec. 4.2.1; cell
 * index i + floor((pos - y)/dx), weight the remainder), every FP64 operation
 * separately rounded.  With pos = Xi, the lift map that lmean_end returns
 * for Strategy 2 (Sec. 3.2), this gives f(x + xi(x, tau+T), tau+T): the
 * Lagrangian perturbation of Sec. 4.2.2 is fbar^L minus the lifted
 * instantaneous field, and Sec. 4.2.1's rearrangement qbar^L(x) = q(Xi(x))
 * compares the lifted PV with its Lagrangian mean.
 *   N:            power of two in [16, 4096].
 *   pos_x, pos_y: device, N*N doubles each (row-major, y slow), absolute
 *                 (unwrapped) positions.
 *   nfields:      1..LM_REMAP_MAX_FIELDS.
 *   f, out:       HOST arrays of nfields device pointers, N*N doubles each;
 *                 no output may alias an input or another output.
 *   stream:       cudaStream_t (NULL: legacy default stream); asynchronous.
 * Errors: SW_EINVAL (message via sw_last_error(NULL)), SW_ECUDA. */
int lmean_lift(int N, const double* pos_x, const double* pos_y, int nfields, const double* const* f,
               double* const* out, void* stream);

/* Shell spectrum of a real N*N field on the handle's 2/3 box (Sec. 4.2.2
 * plots enstrophy spectra: pass the vorticity).  With F = FFT(f)/N^2 kept for
 * |kx|, |ky| <= K, shell n = round(|k|) receives sum |F(k)|^2/2 over the
 * whole plane, so the shells sum to half the mean square of the box-limited
 * field.  Uses the handle's FP64 staging buffers and stream (the dynamic and
 * Lagrangian-mean state is not touched); synchronises.
 *   field:     N*N doubles, host (on_device = 0) or device (on_device = 1).
 *   spectrum:  HOST array of nshell doubles; nshell >= round(sqrt(2) K) + 1
 *              (K = floor((N-1)/3)); entries past that count are set to 0.
 * Errors: SW_EINVAL, SW_ECUDA (message via sw_last_error(h)). */
int sw_spectrum(sw_handle* h, const double* field, int on_device, double* spectrum, int nshell);

/* ---- semi-Lagrangian Strategy 1 (App. B) ---------------------------------
 * The grid-based Lagrangian average as a semi-Lagrangian discretisation of
 * Eqs. (gtilde-evol) and (Xi-1evol) (App. B): after every RK4 step of the
 * handle's dynamics, at each grid point X with departure point
 * Y = X - dt u(X, t_{n+1}),
 *   SL_EULER      g(X) = g_I(Y) + dt f(X, t_{n+1})              Eq. (sdiscrete_gtilde)
 *   SL_TRAPEZOID  g(X) = g_I(Y) + dt [f_I(Y, t_n) + f(X, t_{n+1})]/2
 *                                                    Eq. (sdiscrete_gtilde_trapez)
 * for g = (t - tau) f~, and the mean positions by the same rule applied to
 * f = x (Eq. (sdiscrete_Xi-1) for the trapezoid), carried as the periodic
 * displacement D = (t - tau)(x - Xi^{-1}).  _I: interpolation at Y,
 * SL_LINEAR (bilinear) or SL_CUBIC (tensor-product 4-point Lagrange; the
 * paper does not name its cubic scheme).  u is the flow velocity (the
 * constant adv for the kinematic model).  FP64 on physical grid fields,
 * whatever the handle's precision.  Results: f~^L = g/T and
 * Xi^{-1}(x, tau+T) = x - D/T (feed them to lmean_remap for fbar^L). */
#define SL_EULER 0
#define SL_TRAPEZOID 1
#define SL_LINEAR 0
#define SL_CUBIC 1
typedef struct sl_params {
  int32_t fields;   /* LM_ZETA | LM_H | LM_U | LM_V | LM_Q | LM_POS (nonzero) */
  int32_t scheme;   /* SL_EULER or SL_TRAPEZOID */
  int32_t interp;   /* SL_LINEAR or SL_CUBIC */
  int32_t reserved; /* must be 0 */
  int64_t n_steps;  /* T = n_steps * dt, >= 1 */
} sl_params;
typedef struct sl_interval sl_interval;

/* Open an interval at the handle's current time.  The handle must have no
 * open lmean interval; while the SL interval lives, step the handle only
 * through sw_sl_step and do not destroy it.  Allocates the interval's device
 * buffers (about 2 (2 nf + 2) N*N doubles for nf averaged fields) and
 * synchronises.  Errors: SW_EINVAL, SW_EBUSY, SW_ENOMEM, SW_ECUDA (message
 * via sw_last_error(h), or sw_last_error(NULL) when h is NULL). */
int sw_sl_create(sw_handle* h, const sl_params* p, sl_interval** out);

/* Advance the dynamics and the interval by nsteps >= 0 steps (one sw_step
 * and one update each); SW_ERANGE if more than remain.  Asynchronous. */
int sw_sl_step(sl_interval* s, int64_t nsteps);

/* Requires the interval complete (SW_ESTATE otherwise).  Writes f~^L into
 * the zeta/h/u/v/q pointers of out and Xi^{-1} into pos_x/pos_y for the
 * requested fields (N*N doubles each; e_* ignored; host or device per
 * out->on_device), then frees the interval.  Synchronises. */
int sw_sl_end(sl_interval* s, const lm_result* out);

/* Free an interval without results.  NULL: no-op. */
void sw_sl_destroy(sl_interval* s);

/* ---- measurement ------------------------------------------------------------
 * Fused-multiply-add rate of this GPU's CUDA cores in TFLOP/s (2 flops per
 * FMA), for the arithmetic roofline of the transform kernels: the FP64 path
 * is bound by its FP64 arithmetic, which runs on these cores.  Runs
 * 8 x (multiprocessors) blocks of 256 threads, each with 8 independent FMA
 * chains of 16 x trips FMAs, and reports the best of five timed launches
 * (CUDA events on `stream`, after one warm-up launch).  Allocates a small
 * scratch buffer; synchronises.  The paper has no counterpart.
 *   precision: SW_PREC_FP64 or SW_PREC_FP32; trips: 1..2^20 (4096 is ample).
 * Errors: SW_EINVAL, SW_ECUDA (message via sw_last_error(NULL)). */
int sw_fma_peak(int precision, int trips, double* tflops, void* stream);

/* Wait for all device work of the handle. */
int sw_sync(sw_handle* h);

/* Message for the last failing call on h ("" if none); valid until the next
 * call on h.  With h == NULL, the message of the last failing sw_create,
 * sw_project_static, lmean_remap or lmean_lift on the calling thread. */
const char* sw_last_error(sw_handle* h);

/* Library version string. */
const char* sw_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LAGMEAN_H */
