/*
 * jd.h -- C ABI of the GB300 (sm_103a) library for adjoint-based optimal control of
 * jump-diffusion processes, after "Adjoint-based optimal control of jump-diffusion
 * processes" (arXiv 2505.04328).
 *
 * The library evaluates, for a time-dependent control u = (u_0, ..., u_{Nt-1}),
 * u_k in R^du constant on [t_k, t_{k+1}) (Sec. 3 eq:piecewise_constant_control),
 *
 *   J(u) = (1/M) sum_m sum_{k=1..Nt} dt l(X_k^m, t_k) + (nu/2) dt sum_k |u_k|^2
 *          (Sec. 3 eq:discrete_functional),  l(x,t) = 1/2 sum_i q_i (x_i - xd_i(t))^2,
 *
 * where each path X^m solves the controlled SDE dX = f(X,u) dt + diag(sigma) dB + dY
 * (Sec. 1 eq:SDE_general, Sec. 2 eq:compact_forward) with drift
 * f(x,u) = A x + C (x*x*x) + B u (Sec. 5.4 eq:coefficients: H <-> A, h <-> C x^3) and
 * additive compound-Poisson jumps Y of intensity lambda, discretized by Euler-Maruyama
 * on the jump-adapted grid (Sec. 3 eq:Deterministic_timestep; Algorithms 5.1, 5.2);
 * and its exact discrete gradient by the backward adjoint sweep (Sec. 4
 * eq:AdjointModel, eq:definition_Gradient; Sec. 5.5 eq:adjoint_eq_approximation).
 *
 * Random numbers: counter-based Philox4x32-10 (Salmon et al., SC'11).  Key = seed
 * (low word, high word).  Step k of path m draws its Poisson count and sub-step-0
 * normals from the blocks with counter (k, m, b, epoch), b = 0, 1, ...; jump slot i
 * (i = 1..n) draws from counter (k, m, 1<<24 | i<<16 | b, epoch).  A result therefore
 * depends only on (seed, epoch, path index, step index), never on launch geometry.
 *
 * Conventions for every function:
 *   - returns a jd_status; no exception or abort crosses the ABI; a message for the
 *     last failure of the calling thread is available from jd_last_error();
 *   - the caller owns every buffer passed in; jd_problem_create deep-copies the
 *     descriptor's arrays, so they may be freed after it returns;
 *   - arrays are row-major float64.  A pointer tagged JD_MEM_DEVICE is a CUDA device
 *     pointer read or written on the problem's stream; JD_MEM_HOST is host memory;
 *   - calls that write host memory synchronize the problem's stream before
 *     returning; calls whose outputs are all device pointers return without
 *     synchronizing (results are ready in stream order).
 *   - a problem object is not thread-safe: calls on one problem must not overlap.
 */
#ifndef JD_H
#define JD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  JD_OK = 0,
  JD_ERR_INVALID_ARG = 1,  /* bad size, NULL where required, non-finite input */
  JD_ERR_OOM = 2,          /* device allocation failed or the plan exceeds the memory budget */
  JD_ERR_CUDA = 3,         /* a CUDA runtime call failed (message in jd_last_error) */
  JD_ERR_NONFINITE = 4,    /* the cost or gradient came out NaN or Inf */
  JD_ERR_LINESEARCH = 5,   /* Armijo backtracking exhausted max_backtracks */
  JD_ERR_TIMEOUT = 6,      /* a bounded device-side wait (tensor-core completion) gave up */
  JD_ERR_UNSUPPORTED = 7,  /* valid request this build does not implement (e.g. d > 32) */
  JD_ERR_BUSY = 8          /* serving: result not ready yet */
} jd_status;

typedef enum { JD_DRIFT_LINEAR = 0, JD_DRIFT_CUBIC = 1 } jd_drift;
typedef enum { JD_JUMP_NONE = 0, JD_JUMP_NORMAL = 1, JD_JUMP_UNIFORM = 2, JD_JUMP_KS = 3 } jd_jump_law;
typedef enum { JD_FP32 = 0, JD_FP64 = 1 } jd_precision;
typedef enum { JD_ADJ_AUTO = 0, JD_ADJ_STORED = 1, JD_ADJ_RECOMPUTE = 2 } jd_adjoint_mode;
typedef enum { JD_MEM_HOST = 0, JD_MEM_DEVICE = 1 } jd_memspace;

/* Problem descriptor (Sec. 3 eq:OCP_fully_discrete with the additive jump map).
 *   d, du        state and control dimensions, 1 <= d <= 32, 1 <= du <= 4; for
 *                8 < d <= 32 the build has FP32 paths, LINEAR drift and the stored
 *                adjoint (no parameter gradients)
 *   T, Nt, M     horizon, uniform steps (dt = T/Nt), Monte Carlo paths (M < 2^32)
 *   drift        LINEAR (C ignored) or CUBIC
 *   A, C         d*d; B d*du; dA d*d direction for the drift-coefficient gradient
 *                (A(theta) = A + theta dA), NULL if not needed
 *   sigma        d, diagonal additive diffusion
 *   lambda       jump intensity; jump_law NONE/NORMAL (N(0, jump_scale^2) per
 *                component) / UNIFORM (U[-jump_scale, jump_scale] per component) /
 *                KS, the Keilson-Storer velocity reset of Sec. 5.3 Eq. jump_law: the
 *                state is z = (x, v) with v the components c >= d/2, and a jump sets
 *                v_c <- jump_gain v_c + jump_scale xi_c, xi_c ~ N(0, 1), leaving x;
 *                the paper's kernel has jump_scale = 1/sqrt(2 beta) and intensity
 *                sqrt(beta/pi).  KS is built for d <= 8 (UNSUPPORTED above) and is
 *                not taken by jd_cost_noalloc
 *   x0           d, deterministic initial state
 *   q            d, diagonal tracking weights; xd (Nt+1)*d, target xd(t_k)
 *   nu           control weight (the paper's alpha); u_min, u_max box bounds
 *   seed, epoch  Philox key and the counter's fourth word (resampling mode)
 *   prec         JD_FP32: path arithmetic in FP32, reductions in FP64;
 *                JD_FP64: everything in FP64
 *   mode         adjoint variant: STORED keeps X_k in device memory; RECOMPUTE keeps
 *                checkpoints every S steps and regenerates each segment from the
 *                counter-based streams (exact, same result); AUTO picks STORED when it
 *                fits mem_budget_bytes
 *   use_tensor_cores  8 < d <= 32 only: the drift contraction A x (and A^T lambda in the
 *                adjoint) of each 128-path tile as one tcgen05 MMA per step: 1 = BF16
 *                inputs, FP32 accumulation; 2 = BF16 high + low parts, three products
 *                (about 16 mantissa bits); 3 = the forward on the CUDA cores in FP32 and
 *                the adjoint's A^T lambda as in 2 (the forward is bound by its draws,
 *                the adjoint by the contraction); 0 = FP32 on the CUDA cores
 *   mem_budget_bytes  device bytes this problem may allocate, 0 = library default
 *                (half of the free device memory at creation)
 *   cuda_stream  cudaStream_t for all work of this problem; NULL = the library
 *                creates its own stream
 *   jump_gain    KS only: the velocity gain gamma (finite; the paper takes 0 <= gamma
 *                < 1); ignored by the additive laws
 *   m_offset     global index of the problem's first path: the problem is paths
 *                [m_offset, m_offset + M) of a larger Monte Carlo sample (one shard of
 *                a problem whose paths are split over several GPUs; every draw is
 *                keyed by the global path index).  0 for a whole problem;
 *                m_offset + M <= 2^32.  J and the gradient of such a problem are the
 *                means over its own M paths; jd_gradient_units gives the sums that
 *                combine into the whole problem's result.
 */
typedef struct {
  int d, du;
  double T;
  int Nt;
  int64_t M;
  jd_drift drift;
  const double *A, *C, *B, *dA;
  const double *sigma;
  double lambda;
  jd_jump_law jump_law;
  double jump_scale;
  const double *x0;
  const double *q;
  const double *xd;
  double nu, u_min, u_max;
  uint64_t seed;
  uint32_t epoch;
  jd_precision prec;
  jd_adjoint_mode mode;
  int use_tensor_cores;
  size_t mem_budget_bytes;
  void *cuda_stream;
  double jump_gain;
  int64_t m_offset;
} jd_problem_desc;

typedef struct jd_problem jd_problem;

/* Validate and copy a descriptor; upload coefficients; no path memory is allocated
 * yet.  Errors: INVALID_ARG (sizes, NULL arrays, non-finite values, u_min > u_max),
 * UNSUPPORTED (d > 32, du > 4, use_tensor_cores with d != 32 or CUBIC), CUDA. */
jd_status jd_problem_create(const jd_problem_desc *desc, jd_problem **out);
jd_status jd_problem_destroy(jd_problem *p);

/* J(u) (eq:discrete_functional): forward sweep and cross-path reduction.
 * u: Nt*du in memory space us.  J: host double.  Errors: INVALID_ARG, NONFINITE, CUDA. */
jd_status jd_cost(jd_problem *p, const double *u, jd_memspace us, double *J);

/* J(u) and the Euclidean gradient grad_k = dJ/du_k = nu dt u_k + (1/M) sum_m G_k^m,
 * G_k^m = sum over the sub-steps i of step k of delta_i B^T lambda'_i (exact discrete
 * adjoint; eq:definition_Gradient).  J: host double, may be NULL.  grad: Nt*du in
 * memory space gs, may be NULL.  grad_theta: host, d+2 doubles or NULL:
 * [dJ/dtheta along dA, dJ/dsigma_0 .. dJ/dsigma_{d-1}, dJ/djump_scale].
 * Errors: INVALID_ARG, OOM (plan does not fit), NONFINITE, CUDA. */
jd_status jd_gradient(jd_problem *p, const double *u, jd_memspace us, double *J, double *grad,
                      jd_memspace gs, double *grad_theta);

/* jd_gradient split in two halves, for reverse-mode differentiation frameworks (the
 * forward pass keeps what the backward pass needs, like an autograd graph).
 *
 * jd_forward: J(u) by the forward sweep in the problem's adjoint plan: STORED keeps X_k
 *   and the post-jump states in device memory; RECOMPUTE keeps only the states at every
 *   S-th step (S = 32 for d <= 2, 16 for d <= 8: about sqrt(Nt) checkpointing for
 *   Nt ~ 10^3).  u: Nt*du in memory space us.  J: one double in memory space js, may be
 *   NULL; with js = JD_MEM_DEVICE the call does not synchronize.
 * jd_backward: the adjoint sweep and reductions for the u and coefficients of the last
 *   jd_forward (or jd_gradient) on this problem: grad (Nt*du) and grad_theta (d+2
 *   doubles, layout as in jd_gradient, may be NULL), both in memory space gs; bitwise
 *   equal to jd_gradient's results.  With gs = JD_MEM_DEVICE the call does not
 *   synchronize and non-finite results are not reported (check the outputs).
 *   It may be called more than once after one forward.  Any other call on the problem
 *   in between (jd_cost, jd_optimize, jd_sample_paths, jd_problem_update) discards the
 *   forward; jd_backward then fails with INVALID_ARG.
 * Errors: as jd_gradient. */
jd_status jd_forward(jd_problem *p, const double *u, jd_memspace us, double *J, jd_memspace js);
jd_status jd_backward(jd_problem *p, double *grad, jd_memspace gs, double *grad_theta);

/* Replace the coefficients of a problem without reallocating its device buffers: A, C,
 * B, dA, sigma, lambda, jump_law, jump_scale, x0, q, xd, nu, u_min, u_max, seed and
 * epoch are taken from desc (host arrays, copied; validated as in jd_problem_create).
 * d, du, T, Nt, M, drift, prec, mode and use_tensor_cores must equal the problem's
 * (else INVALID_ARG); mem_budget_bytes and cuda_stream are ignored.  Used to move a
 * parameter (drift coefficient, sigma, jump scale) between autograd evaluations, or
 * the epoch word between resampled iterations (Sec. 5.6).  Synchronizes the stream
 * only when the target xd changes.  Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
jd_status jd_problem_update(jd_problem *p, const jd_problem_desc *desc);

/* Trajectories of paths m0 .. m0+count-1 (host outputs, any may be NULL):
 * X (count, Nt+1, d) states on the uniform grid; lam (count, Nt+1, d) adjoint states
 * lambda_k = d(path cost)/dX_k; cost (count) per-path running cost.  Uses the same
 * kernels and streams as jd_gradient.  Errors: INVALID_ARG, OOM, CUDA. */
jd_status jd_sample_paths(jd_problem *p, const double *u, jd_memspace us, int64_t m0,
                          int64_t count, double *X, double *lam, double *cost);

/* Projected gradient descent with the Armijo rule (Algorithm 5.4, eq:Stochastic_Armijo).
 * Each iteration evaluates the gradient at u^n, searches the step and updates; no
 * gradient is evaluated after the last update.  With g = grad/dt (the L2
 * representative) the trial point is u+ = clip(u - zeta g, u_min, u_max), accepted when
 * J(u+) <= J(u) + c <g, u+ - u>_{L2}; zeta starts at zeta0, is doubled (capped at
 * zeta_max) at the start of every later iteration and halved on rejection.  Stops when
 * |P(u - g) - u|_{L2} <= tol_rel_grad |P(u0 - g0) - u0|_{L2} (checked when a gradient
 * is evaluated), when |u+ - u|_{L2} < tol_step, or after max_iter updates.  The Armijo
 * test and every FP64 reduction run on the device; the host only reads the accept flag.
 * r->iters = updates done, r->evals = gradient + cost evaluations, r->zeta = last
 * accepted step (pass 2*zeta as zeta0 to continue an interrupted run).
 * Paired trials: for an iteration's first trial (unless the last two iterations took
 * their first point) the trial point zeta and its backtrack zeta/2 are evaluated in
 * one forward sweep on the same
 * random data (both controls share the draws; each state's arithmetic is that of a
 * sweep of its control alone) and tested in backtracking order, so iterates, J values,
 * zeta and r->evals are those of one trial per sweep; r->sweeps counts the forward
 * sweeps run (a pair counts one).  Needs a second set of the plan's path buffers within
 * the memory budget (else one trial per sweep); not with the block-wise stored plan
 * nor for d > 4 (where a pair costs more than two single sweeps or saves nothing). */
typedef struct {
  int max_iter;
  double tol_rel_grad, tol_step, armijo_c, zeta0, zeta_max;
  int max_backtracks;
  int resample;   /* 0: one fixed sample (sample average approximation).  1: the stochastic
                     descent of Sec. 5.6 / Algorithm 5.4 with fresh random data every
                     iteration: iteration n evaluates its gradient and its Armijo trials on
                     epoch desc.epoch + n; J_hist[n] is J(u^n) on sample n, the last entry
                     the accepted trial's cost on the last iteration's sample; the problem's
                     epoch is restored when the call returns */
  int one_trial_per_sweep;   /* 0: paired trials where available (above); 1: never */
} jd_opt_params;

typedef struct {
  int iters, evals;
  double J, rel_grad_norm, zeta;
  jd_status status;
  int sweeps;   /* forward sweeps run (gradients with their own forward, trials, pairs) */
} jd_opt_result;

/* u_inout: Nt*du in memory space us, updated in place.  J_hist: host, max_iter+1
 * doubles or NULL (J of every iterate).  Errors: INVALID_ARG, LINESEARCH, NONFINITE,
 * OOM, CUDA. */
jd_status jd_optimize(jd_problem *p, double *u_inout, jd_memspace us, const jd_opt_params *o,
                      jd_opt_result *r, double *J_hist);

/* Device bytes the plan of this problem uses (after the first evaluation) and the
 * adjoint variant in use (JD_ADJ_STORED or JD_ADJ_RECOMPUTE; JD_ADJ_AUTO before the
 * first evaluation). */
jd_status jd_problem_info(const jd_problem *p, size_t *device_bytes, jd_adjoint_mode *mode);

/* Device bytes a problem with this descriptor allocates under the given adjoint plan
 * (JD_ADJ_STORED or JD_ADJ_RECOMPUTE): the buffers of jd_problem_create plus the plan's
 * state storage.  Host arithmetic only; no device is touched.  Used for admission by
 * HBM footprint.  Errors: INVALID_ARG (as jd_problem_create, or another plan),
 * UNSUPPORTED (RECOMPUTE with d > 8). */
jd_status jd_problem_footprint(const jd_problem_desc *desc, jd_adjoint_mode plan, size_t *bytes);

/* Serving: a request loop that solves many optimal-control problems concurrently on
 * the current device (the paper's method, Algorithm 5.4, once per request).
 *
 * jd_server_create: hbm_budget = device bytes the server may hold for admitted
 *   requests (0 = 80% of the free memory); max_slots = requests in flight at most
 *   (1..256).  One worker thread owns the device work; every slot has its own stream.
 * jd_server_submit: copies the descriptor (host arrays) and the optimizer parameters
 *   and queues the request; returns at once with a ticket.  The control starts at
 *   u = 0 projected into [u_min, u_max]; cuda_stream and mem_budget_bytes are ignored
 *   (the server assigns them); mode AUTO lets the server pick the plan.  Validation
 *   errors are returned here (as jd_problem_create).
 * Admission: in arrival order, a request starts when a slot is free and its footprint
 *   (jd_problem_footprint) fits the free budget; AUTO picks STORED when that plan fits
 *   a quarter of the budget, else RECOMPUTE (d <= 8).  A request that cannot fit even
 *   an empty server finishes with status OOM; later requests may overtake one that is
 *   waiting for memory.
 * Execution: each request runs jd_optimize's arithmetic and host decisions on its own
 *   buffers, so its result is bitwise the same as a solo jd_optimize with u0 = 0,
 *   whatever else runs; the kernels of all active requests overlap.  Large requests run
 *   on their own stream.  Small ones (d <= 2, du = 1, the stored plan, M at most the
 *   batching limit) share launches (the paper's Algorithm 5.4 per request, its gradient
 *   evaluations batched): the pending optimizer phases (gradient or line-search trial)
 *   of up to 16 such requests with the same precision and dimension are one launch
 *   sequence -- forward sweeps (single and paired) and one adjoint sweep over all their
 *   paths, one launch per reduction and per optimizer step -- in which every problem's
 *   blocks compute what its own launches would.
 * jd_server_poll: JD_ERR_BUSY while the request runs; then JD_OK with r (the request's
 *   own status in r->status) and, if u_out is not NULL, the final control (Nt*du host
 *   doubles), which is handed out once (a second poll with u_out fails with INVALID_ARG).
 * jd_server_wait: blocks until the request is done or timeout_s seconds pass (BUSY).
 * jd_server_info: times in seconds since the server was created (admit_s, done_s are
 *   -1 until they happen), bytes and plan of the admitted request, its gradient
 *   path-steps (M*Nt per gradient evaluation: forward + adjoint sweep) and its sweep
 *   path-steps (M*Nt per sweep over the paths actually run: forward sweeps of gradients
 *   and line-search trials, a paired trial counting one, plus the adjoint sweeps).  A request's footprint includes the second buffer set of paired
 *   trials when that keeps it within a quarter of the budget and what is free.
 * jd_server_set_batching: the batching limit, in paths, for requests admitted after the
 *   call (default JD_SERVER_BATCH_PATHS; 0 = every request runs its own launches).
 *   INVALID_ARG for a negative limit.
 * jd_server_batch_stats: batched launch sequences so far, and the request phases they
 *   ran (phases / launches = the mean batch size).  Either pointer may be NULL.
 * jd_server_destroy: cancels requests not yet admitted (status INVALID_ARG), waits for
 *   the running ones, frees everything. */
#define JD_SERVER_BATCH_PATHS 65536
typedef struct jd_server jd_server;
typedef struct {
  double submit_s, admit_s, done_s;
  size_t device_bytes;
  jd_adjoint_mode plan;
  int done;
  int64_t path_steps, sweep_steps;
} jd_request_info;
jd_status jd_server_create(size_t hbm_budget, int max_slots, jd_server **s);
jd_status jd_server_submit(jd_server *s, const jd_problem_desc *d, const jd_opt_params *o, uint64_t *ticket);
jd_status jd_server_poll(jd_server *s, uint64_t ticket, double *u_out, jd_opt_result *r);
jd_status jd_server_wait(jd_server *s, uint64_t ticket, double timeout_s);
jd_status jd_server_info(jd_server *s, uint64_t ticket, jd_request_info *info);
jd_status jd_server_set_batching(jd_server *s, int64_t max_paths);
jd_status jd_server_batch_stats(jd_server *s, int64_t *launches, int64_t *phases);
jd_status jd_server_destroy(jd_server *s);

/* Number of kernels this library has launched in this process (monotone counter). */
uint64_t jd_kernel_launch_count(void);

/* Kernel timing (tracing).  jd_profile_enable(1) clears the record and brackets every
 * later launch with a CUDA event pair on the launching stream; jd_profile_enable(0)
 * stops recording.  jd_profile_read waits for the recorded events and fills up to
 * max_entries per-class totals (classes: fwd_cost, fwd_store, fwd_ckpt, adj_stored,
 * adj_recompute, finalize, prep_u, opt_step); returns the number filled.  name points
 * to static storage. */
typedef struct {
  const char *name;
  uint64_t launches;
  double total_ms;
} jd_kernel_stat;
void jd_profile_enable(int on);
int jd_profile_read(jd_kernel_stat *out, int max_entries);

/* ---------------------------------------------------------------------------
 * Path sharding: one problem's M paths split over several GPUs (or processes).
 *
 * The Monte Carlo mean of Sec. 3 is a sum over paths, and every draw is keyed by the
 * global path index, so a problem splits into shards of consecutive paths (m_offset,
 * M of each shard's descriptor) that run independently.  The reduction over paths is
 * defined on units of JD_UNIT_PATHS consecutive paths: within a unit a fixed tree over
 * its per-warp partials, across units a plain sum in unit order.  A shard that starts at
 * a unit boundary therefore produces exactly the unit sums the whole problem would, and
 * jd_combine_units over all shards' units (in path order) gives J and the gradient of
 * jd_gradient on the whole problem bit for bit, for every split.  jd_gradient and
 * jd_cost use the same unit reduction.
 *
 * jd_gradient_units / jd_cost_units: run the problem's paths at u and write its units,
 *   units[nu][ne], nu = ceil(M / JD_UNIT_PATHS), ne = 1 + Nt du (gradient) or 1 (cost):
 *   units[i][0] = sum of the unit's path costs sum_k dt l(X_k, t_k) (eq:discrete_functional
 *   without the control term), units[i][1 + k du + l] = sum over the unit's paths of the
 *   step's sensitivity delta B^T lambda' (eq:definition_Gradient without the nu term and
 *   the 1/M).  u as in jd_gradient; units in memory space os (host: synchronizes; device:
 *   stream ordered).  INVALID_ARG unless m_offset is a multiple of JD_UNIT_PATHS.
 * jd_combine_units: host arithmetic, no GPU.  M_total: paths of the whole problem; u:
 *   host, Nt du doubles (the control term nu dt/2 sum |u_k|^2 and nu dt u_k); units: all
 *   shards' units in path order, nunits = ceil(M_total / JD_UNIT_PATHS) rows of ne;
 *   grad: Nt du doubles or NULL when ne = 1.  Returns J and grad as jd_gradient would.
 */
#define JD_UNIT_PATHS 16384
jd_status jd_gradient_units(jd_problem *p, const double *u, jd_memspace us, double *units, jd_memspace os);
jd_status jd_cost_units(jd_problem *p, const double *u, jd_memspace us, double *units, jd_memspace os);
jd_status jd_combine_units(int64_t M_total, int Nt, int du, double T, double nu, const double *u,
                           const double *units, int64_t nunits, int ne, double *J, double *grad);

/* J(u) for callers that cannot allocate device memory once they are running: a
 * real-time control loop (cudaMalloc can take milliseconds and synchronizes the
 * device) or an application whose memory pool owns the whole GPU.  The paper has no
 * counterpart; this is a deployment variant of jd_cost.
 *
 * It runs the same forward cost kernel as jd_cost, but allocates nothing, on the
 * device or on the host: its scratch is one fixed 4 MiB file-scope device array that
 * every GPU loading this library holds until the process exits.
 *   desc   problem descriptor: host arrays; A, B, C, sigma, x0, q are read during the
 *          call, xd is copied into the scratch by cudaMemcpyAsync on desc->cuda_stream,
 *          so xd (pageable or page-locked host memory, not device memory) must stay
 *          unchanged until the stream has reached the call; d <= 2, du == 1, FP32 or
 *          FP64, the additive jump laws; mode, mem_budget_bytes and use_tensor_cores
 *          are ignored (use_tensor_cores must be 0)
 *   u      device pointer, Nt doubles
 *   J      device pointer, one double, written in stream order on desc->cuda_stream
 *          (NULL = the legacy default stream); the call does not synchronize
 * The scratch holds, each rounded up to 256 bytes, the FP64 target ((Nt+1) d doubles),
 * the padded target ((Nt+1) d values) and the control (Nt values) in kernel precision,
 * and one FP64 partial per 128 paths; a problem whose total exceeds 4 MiB is rejected
 * with JD_ERR_OOM (for d = 2, Nt = 1000 in FP32 the fixed part takes 28,416 bytes,
 * which leaves room for 520,736 partials: M up to about 66.6 million paths; M is also
 * limited to 2^32 - 1).  Every entry read is written earlier in the same call, so
 * nothing needs clearing between calls.  All calls on a device share the one array:
 * calls that overlap on the GPU (other streams, other host threads) race and must be
 * serialized by the caller.
 * The first call on each device is a warm-up: it takes the array's device address
 * with cudaGetSymbolAddress (with that device current) and the cost kernels'
 * per-thread stack needs, and its launches may load the kernels' code (the CUDA
 * runtime loads modules lazily, which allocates).  Make that first call before any
 * stream capture and before the point from which nothing may allocate; later calls
 * allocate nothing.  Errors are reported by status only (jd_last_error is not updated,
 * since that would allocate): INVALID_ARG, UNSUPPORTED (d > 2, du != 1, or a
 * per-thread stack limit below what the cost kernel needs: the call does not raise
 * it), OOM (beyond the scratch), CUDA. */
jd_status jd_cost_noalloc(const jd_problem_desc *desc, const double *u, double *J);

/* ---------------------------------------------------------------------------
 * Feedback control (Sec. 2 eq:control_structure; Sec. 5.1-5.2; Sec. 5.5; Sec. 6).
 *
 * On a problem with d = 2, du = 1, read as the phase space z = (x, v), the control is
 * the state feedback u(z, t) = sum_{i,l} mu_k[i][l] phi(x - x^i) phi(v - v^l) for t in
 * [t_k, t_{k+1}), with the bump phi(r) = exp(-1/(1 - (eps r)^2)) on |r| < 1/eps
 * (Sec. 5.2 eq:Gaussian_RBF) centred on the cell centres x^i = (i + 1/2) 2 x_max/nx -
 * x_max, v^l = (l + 1/2) 2 v_max/nv - v_max (Sec. 5.1; i, l from 0).  B u(z) enters the
 * drift, evaluated at the left end of every sub-step of the jump-adapted grid.  The
 * cost is J(mu) = (1/M) sum_m [ sum_{k=1..Nt} dt l(X_k, t_k) + sum over sub-steps
 * (alpha/2) delta u(Y)^2 ], alpha = the descriptor's nu, with l the quadratic term
 * (1/2) sum q_c (z_c - xd_c)^2, the Gaussian -exp(-sum q_c (z_c - xd_c)^2 / (2 sigma_J^2))
 * of Sec. 6 eq:tracking_cost, or the ellipse term of Sec. 6.4.  u_min and u_max do not apply.  The gradient is the exact
 * derivative of J in mu (eq:definition_Gradient with the adjoint of
 * eq:adjoint_eq_approximation, u_x and u_v included).  Every jump law is accepted.
 * --------------------------------------------------------------------------- */
typedef enum { JD_TRACK_QUADRATIC = 0, JD_TRACK_GAUSS = 1, JD_TRACK_ELLIPSE = 2 } jd_track;
typedef enum { JD_FB_EXACT = 0, JD_FB_SURROGATE = 1 } jd_fb_adjoint;

typedef struct {
  int nx, nv;            /* centres per axis, 1..16; L = nx nv weights per step */
  double x_max, v_max;   /* half-widths of the computational domain, > 0 */
  double eps;            /* bump shape parameter eps_phi, > 0 */
  jd_track track;        /* tracking term l */
  double sigma_J;        /* Gaussian width, > 0 for JD_TRACK_GAUSS */
  jd_fb_adjoint adjoint; /* EXACT: the discrete adjoint along the forward's states.
                            SURROGATE (Sec. 6.5): the costates run backwards along states
                            drawn around the target, zs_k = xd(t_k) + sqrt(sur_rate t_k) xi
                            (xi: Box-Muller pair of the Philox words 0, 1 of counter
                            (k, m, 2 << 24, epoch)), one Euler adjoint step per uniform step
                            with the Jacobian of the path's own jumps; the gradient records
                            delta phi(Y) (alpha u(Y) + B^T r) are formed on the forward's
                            sub-steps.  An approximation: no states are stored (one value per
                            path and step instead of two) */
  double sur_rate;       /* SURROGATE: variance growth per unit time, >= 0 */
  int particles;         /* interacting particles (Sec. 6.4 eq:interacting_model): 0 for
                            independent paths, else 3..32 particles per ring: path m is
                            particle m % 32 of realization m / 32 (lanes >= particles idle; M
                            must be a multiple of 32), dv_i gains -omega (2 x_i - x_{i-1} -
                            x_{i+1}) with the neighbours' positions at t_k driving the whole
                            step k, and the particles start equidistant on the ellipse
                            (ax cos(2 pi i/N), av sin(2 pi i/N)); J and the gradient average over
                            the M/32 * particles particles.  EXACT adjoint only */
  double omega;          /* ring coupling */
  double ax, av;         /* ellipse half-axes (> 0 for JD_TRACK_ELLIPSE or particles > 0):
                            JD_TRACK_ELLIPSE is -exp(-(x^2/ax^2 + v^2/av^2 - 1)^2 / (2 sigma_J^2))
                            of Sec. 6.4 Eq. phonon_functional_tracking */
} jd_feedback_desc;

/* J(mu).  mu: Nt * L doubles, row-major [k][i][l], in mu_space; J: host pointer.  The
 * problem's device memory gains the weights in kernel precision and M/256 FP64 cost
 * partials (allocated on first use, kept until destroy, within the memory budget).
 * Errors: INVALID_ARG (NULL, a descriptor value out of range, a non-finite weight),
 * UNSUPPORTED (d != 2 or du != 1), OOM, CUDA. */
jd_status jd_fb_cost(jd_problem *p, const jd_feedback_desc *fb, const double *mu,
                     jd_memspace mu_space, double *J);

/* J(mu) and grad = dJ/dmu (Nt * L doubles, [k][i][l]), both mu and grad in `space`; J
 * is a host pointer (nullable).  Runs the forward sweep storing X_k (2 Nt M values in
 * kernel precision) and the jump flags, then the adjoint sweep; steps with jumps are
 * regenerated from X_k.  The gradient partials take M/32 * Nt * L' values in kernel
 * precision (one per warp of 32 paths), L' the padded weight count (16, 100 or 256).
 * Deterministic: the same call gives the same bits.
 * Errors as jd_fb_cost. */
jd_status jd_fb_gradient(jd_problem *p, const jd_feedback_desc *fb, const double *mu,
                         jd_memspace space, double *J, double *grad);

/* Gradient descent with the Armijo rule on the weights (Algorithm 5.4 with
 * eq:Stochastic_Armijo; mu is unconstrained): per iteration one jd_fb_gradient at mu^n,
 * then trial points mu^n - zeta g, g = (dJ/dmu)/dt, until J(trial) <= J(mu^n) -
 * c zeta |g|^2_{L2} (|g|^2_{L2} = dt sum g^2), zeta halved per rejection; zeta doubles
 * (capped at zeta_max) from the second iteration on.  Stops on |g|_{L2} <= tol_rel_grad
 * times its first value, on a step |mu^{n+1} - mu^n|_{L2} < tol_step, or after max_iter
 * updates.  The update kernels and the norms run on the device in FP64; the host reads
 * J and |g|^2 back for each decision.  mu_inout: Nt * L doubles in `space`, updated in
 * place; J_hist (host, max_iter + 1, nullable).  r->status is JD_ERR_LINESEARCH (also
 * returned) when max_backtracks halvings did not satisfy the test.  With the exact
 * adjoint and a fixed sample the trials keep their states and the accepted trial's sweep
 * is the next gradient's forward half; r->sweeps counts the forward sweeps run.  Paired
 * trials (one_trial_per_sweep) are not built here.  Other errors as jd_fb_cost. */
jd_status jd_fb_optimize(jd_problem *p, const jd_feedback_desc *fb, double *mu_inout, jd_memspace space,
                         const jd_opt_params *o, jd_opt_result *r, double *J_hist);

const char *jd_status_string(jd_status s);
const char *jd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* JD_H */
