// jd_internal.h -- types shared by the host library and the path kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "jd.h"

namespace jd {

constexpr int NMAX = 16;   // jumps per uniform step are capped at this count
constexpr int TPB = 128;   // threads (one path each) per block of the path kernels
constexpr int SPREAD_TPB = 32;     // a small problem's pre-drawn sweeps: one warp per block ...
constexpr int SPREAD_LANES = 4;    // ... with this many paths (lanes) active (measured: 4 beat 1, 8, 32)
constexpr int BATCH = 8;   // steps per transposed warp reduction

// FWD_PAIR (with FWD_STORE or FWD_CKPT): a second control on the same random data in the
// same sweep (PathBufs' second set).
enum FwdMode { FWD_COST = 0, FWD_STORE = 1, FWD_CKPT = 2, FWD_PAIR = 4 };
enum AdjVariant { ADJ_STORED_V = 1, ADJ_RECOMPUTE_V = 2 };

// Kernel parameters: coefficients padded to the compiled dimensions D, DU and passed
// by value, so the hot loop reads them as constant-bank operands.
template <typename R, int D, int DU>
struct KParams {
  R A[D * D], C[D * D], dA[D * D], B[D * DU];
  R sigma[D];      // sigma_c
  R sig_sqdt[D];   // sigma_c * sqrt(dt)
  R qdt[D];        // q_c * dt            (cost gradient)
  R hqdt[D];       // q_c * dt / 2        (cost)
  R x0[D];
  R jgain[D];      // jump map y_c <- jgain_c y_c + jscl_c xih_c: gamma on reset velocities,
  R jscl[D];       // else 1; jscl_c = jump_scale on the components a jump moves, else 0
  R dt, sqdt, jump_scale;
  unsigned long long thr[NMAX];  // Poisson thresholds floor(2^32 F(n; lambda dt))
  uint32_t key0, key1, epoch;
  int d, npair, Nt, cubic, jump_law, jumps_on, has_dA, S, nblk;
  int kvel;                       // first component a jump moves (d/2 for Keilson-Storer, else 0)
  int64_t m_begin;                // global index of path 0 of this launch
  int64_t npart;                  // stride of the per-warp gradient partials (all launches)
  // Philox round keys (key0 + r W0, key1 + r W1 mod 2^32, r = 0..9), read by the forward
  // sweeps as constant operands of the rounds' XORs instead of bumping the key in every
  // block; last in the struct, so kernels that do not read them see the same layout
  uint32_t rk0[10], rk1[10];
};

// Device buffers of one launch (unused ones are null).
struct PathBufs {
  void *traj = nullptr;        // stored states
  uint32_t *flags = nullptr;   // jump flags, 1 bit per path-step
  void *ckpt = nullptr;        // checkpoints (recompute variant)
  void *pcost = nullptr;       // per-path cost (optional)
  void *log_kt = nullptr;      // jump log: (step, time fraction) per record
  void *log_y = nullptr;       // jump log: post-jump states
  int *jcnt = nullptr;         // jump log: records per path
  int log_cap = 0;             // jump log: records per path capacity
  double *partC = nullptr, *partG = nullptr, *partT = nullptr;
  void *lam_out = nullptr;     // adjoint states (optional)
  int *status = nullptr;       // device status word (bounded waits record timeouts here)
  // second control of a paired sweep (FWD_PAIR) and its outputs
  const void *uk2 = nullptr;
  void *traj2 = nullptr, *ckpt2 = nullptr, *log_kt2 = nullptr, *log_y2 = nullptr;
  double *partC2 = nullptr;
  // main-stream draws of every (step, path) taken by a parallel pre-pass (small problems,
  // whose sweeps are latency-bound): pre_w [Nt][mloc] Poisson words, pre_z [Nt][D][mloc]
  // normals followed by [Nt][1 + 2D][mloc] slot-0 draws, in kernel precision, then the
  // sweeps' per-path cost pairs [2][mloc]; null = the sweep draws them itself
  uint32_t *pre_w = nullptr;
  void *pre_z = nullptr;
  // key of the draws the pre-pass buffers hold (0: none): the draws depend on the generator's
  // key, epoch and path range and on the jump thresholds only, not on the control, so a sweep
  // with the same key reuses them (the draws kernel returns at once)
  unsigned long long *pre_key = nullptr;
  // partial-stride override: a launch that covers one block of the paths (chunked
  // stored plan) writes its partials at their global positions (partG, partC offset
  // by the caller) with the stride of all M paths; 0 = this launch's own count
  int64_t npart = 0;
};

// Batched sweeps (serving): the problems of one launch, each with its control in kernel
// precision and its plan's buffers.
constexpr int kBatchMax = 16;   // problems per batched launch
struct BatchSweep {
  const struct ::jd_problem *p;
  const void *uk;
  PathBufs b;
};

// Per-instantiation launch table (one entry per precision x compiled dimension).
struct PathOps {
  int D, DU, S, elem;
  int traj_layout;   // unused: every instantiation stores states as traj_shape(D, elem) says
  // per-thread stack bytes the kernels of this instantiation may need (the jump path
  // keeps its sub-step states in local memory behind a non-inlined call)
  size_t (*stack_bytes)();
  // forward sweep in mode FWD_COST / FWD_STORE / FWD_CKPT
  cudaError_t (*fwd)(const struct ::jd_problem *p, int mode, int64_t m_begin, int64_t mloc,
                     const void *uk, const PathBufs &b, cudaStream_t s);
  // adjoint sweep: per-step gradient partials [Nt][DU][nblk * TPB/32] (one per warp);
  // theta partials [D+2][nblk]
  cudaError_t (*adj)(const struct ::jd_problem *p, int variant, bool theta, int64_t m_begin,
                     int64_t mloc, const void *uk, const PathBufs &b, cudaStream_t s);
  // shared memory per block of the recompute adjoint for segments of S steps (null: no
  // recompute plan)
  size_t (*rc_smem)(bool theta, int S);
  // batched stored-plan sweeps over all paths of up to kBatchMax problems of this
  // instantiation (forward in mode FWD_STORE or FWD_STORE | FWD_PAIR; adjoint without
  // parameter gradients); null where not built (built for D <= 2, DU = 1)
  cudaError_t (*fwd_batch)(const BatchSweep *items, int n, int mode, cudaStream_t s);
  cudaError_t (*adj_batch)(const BatchSweep *items, int n, cudaStream_t s);
};

const PathOps *path_ops_dims(int prec, int D, int DU);

// Feedback control kernels (jd_fb_*): d = 2, du = 1, padded NX x NV weights.
constexpr int FB_TPB = 256;   // threads (one path each) per block
constexpr int FB_NB = 16;     // largest centre count per axis
constexpr int FB_GROUP_WARPS = 128;   // warps per group of the first gradient reduction stage
inline int64_t fb_groups(int64_t nwarp) { return (nwarp + FB_GROUP_WARPS - 1) / FB_GROUP_WARPS; }

// Rings of interacting particles (Sec. 6.4): the exchange kind of a ring of N particles
// (0: independent paths, 1: one warp, 2: lanes of one block, 3: a thread-block cluster)
// and its lane count S (particle i of ring r is lane S r + i).
inline int ring_kind(int N) { return N <= 0 ? 0 : N <= 32 ? 1 : N <= 256 ? 2 : 3; }
inline int ring_lanes(int N) {
  if (N <= 32) return 32;
  if (N <= 256) {
    int s = 64;
    while (s < N) s *= 2;
    return s;
  }
  return 256 * ((N + 255) / 256);
}
constexpr int RING_MAX = 2048;   // 8 blocks of 256 lanes: the largest portable cluster

// Draw pre-pass: a problem with d <= 2 whose paths fill at most 2 blocks per SM of a
// GB300 (its sweeps are latency-bound: each thread's steps are a chain of dependent
// operations, and the Philox and Box-Muller of every step sit on that chain) takes its
// main-stream draws in one parallel kernel first, when their buffers stay small.
constexpr int64_t PRE_MAX_PATHS = 152 * 2 * 128;
constexpr size_t PRE_MAX_BYTES = (size_t)128 << 20;
// pre_z holds the normals, the slot-0 draws and then the paths' cost pairs of the sweeps
// (2 controls x M pairs of 2 values)
inline size_t pre_z_values(int Nt, int D, int64_t M) {
  return (size_t)Nt * (1 + 3 * D) * (size_t)M + 4 * (size_t)M;
}
inline size_t pre_bytes(int Nt, int D, int64_t M, size_t es) {
  // words; normals, slot-0 draws and cost pairs; the key of the draws held
  return (size_t)Nt * (size_t)M * 4 + pre_z_values(Nt, D, M) * es + sizeof(unsigned long long);
}
inline bool pre_pass(int d, int Nt, int64_t M, size_t es) {
  const int D = d <= 1 ? 1 : 2;
  return d <= 2 && M <= PRE_MAX_PATHS && pre_bytes(Nt, D, M, es) <= PRE_MAX_BYTES;
}

struct FbBufs {
  const void *mu = nullptr;     // [Nt][NX/2][NV][2] padded, interleaved weights, kernel precision
  void *traj = nullptr;         // [Nt+1][2][M] states (gradient only)
  uint32_t *flags = nullptr;    // [ceil(Nt/32)][M] jump flags (gradient only)
  double *partC = nullptr;      // [nblk] cost partials
  void *partW = nullptr;        // [nwarp][Nt][NX*NV] warp partials, kernel precision
  double *partG = nullptr;      // [ngroup][Nt][NX*NV] FP64 group partials
};

struct FbOps {
  int NX, NV, elem;
  size_t (*stack_bytes)();   // per-thread stack the kernels may need (jump steps)
  // forward sweep (store: keep X_k and the flags); adjoint sweep over the stored states
  cudaError_t (*fwd)(const struct ::jd_problem *p, const jd_feedback_desc &fb, bool store,
                     const FbBufs &b, cudaStream_t s);
  cudaError_t (*adj)(const struct ::jd_problem *p, const jd_feedback_desc &fb, const FbBufs &b,
                     cudaStream_t s);
  // surrogate gradient (Sec. 6.5): surrogate adjoint into b.traj (bhat, [Nt][M]), then the
  // forward sweep with the gradient records into partC / partW
  cudaError_t (*sur)(const struct ::jd_problem *p, const jd_feedback_desc &fb, const FbBufs &b,
                     cudaStream_t s);
  cudaError_t (*reduce)(const struct ::jd_problem *p, const FbBufs &b, cudaStream_t s);   // partW -> partG
  cudaError_t (*prep_mu)(const double *mu64, void *muR, int Nt, int nx, int nv, cudaStream_t s);
};
const FbOps *fb_ops(int prec, int nx, int nv);   // the smallest compiled NX x NV that fits
cudaError_t fb_finalize(const double *partC, const double *partG, int64_t nblk, int64_t ngroup, int Nt, int nx,
                        int nv, int NX, int NV, int64_t M, double *J, double *grad, cudaStream_t s);
// Armijo descent on the weights: |g|^2_{L2} into *out; trial point mu - zeta grad / dt.
cudaError_t fb_norm(const double *grad, int64_t n, double dt, double *out, cudaStream_t s);
cudaError_t fb_trial(const double *mu, const double *grad, int64_t n, double zeta, double dt, double *mt,
                     cudaStream_t s);
int compiled_dim(int d);         // smallest compiled D >= d, or 0

void count_launch(int n = 1);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Stored trajectories are 16-byte vectors of VW = 16 / elem values.  A group of SV
// consecutive steps of one path fills VD vectors, and the value of (step g SV + j,
// component c) sits at position j D + c of its group:  traj[g][v][mloc][VW].  So the
// components of one step are adjacent (the paired FP32 arithmetic takes them as one
// 64-bit operand) and a warp's vector loads cover 512 contiguous bytes.
//   FP32: D = 1 -> 4 steps per vector, D = 2 -> 2, D = 4 -> 1, D = 8 -> 2 vectors per
//   step, D = 32 -> 8 (the tensor-core tiles).  FP64: D = 1 -> 2 steps, D >= 2 -> D/2.
struct TrajShape {
  int VW, SV, VD;
};
constexpr TrajShape traj_shape(int D, int elem) {
  return TrajShape{16 / elem, D >= 16 / elem ? 1 : (16 / elem) / D, D >= 16 / elem ? D / (16 / elem) : 1};
}
// Values (of elem bytes) of the stored states X_0..X_Nt of M paths.
inline size_t traj_values(int Nt, int D, int elem, int64_t M) {
  const TrajShape t = traj_shape(D, elem);
  return (size_t)((Nt + t.SV) / t.SV) * t.VD * (size_t)M * t.VW;
}
// Index of the value (step k, component c) of local path i among `count` paths.
inline size_t traj_index(int k, int c, int64_t i, int64_t count, int D, int elem) {
  const TrajShape t = traj_shape(D, elem);
  const int pos = (k % t.SV) * D + c;
  return (((size_t)(k / t.SV) * t.VD + pos / t.VW) * (size_t)count + (size_t)i) * t.VW + pos % t.VW;
}

// Gradient partials per launch of mloc paths: one per warp of every block.
inline int64_t grad_parts(int64_t mloc) { return ceil_div(mloc, TPB) * (TPB / 32); }

}  // namespace jd

// Host-side problem object (opaque to the ABI user).
struct jd_problem {
  jd_problem_desc desc;              // scalars; array pointers are cleared
  std::vector<double> A, C, B, dA, sigma, x0, q, xd;
  int D = 0, DU = 0;
  const jd::PathOps *ops = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  size_t budget = 0;
  jd_adjoint_mode plan = JD_ADJ_AUTO;
  int S = 16;                // recompute plan: steps per checkpoint segment (16, 32 or 64)
  uint32_t *pre_w = nullptr; // draw pre-pass buffers of a small problem (PathBufs::pre_w, pre_z,
  void *pre_z = nullptr;     // pre_key)
  unsigned long long *pre_key = nullptr;
  bool fwd_valid = false;   // stored states / checkpoints belong to u_in (jd_forward)
  // device buffers
  void *uk = nullptr;        // kernel-precision padded control, Nt*DU
  void *xdk = nullptr;       // kernel-precision padded target, (Nt+1)*D
  double *u_in = nullptr;    // FP64 control copy, Nt*du
  double *grad_d = nullptr;  // FP64 gradient, Nt*du
  double *scal_d = nullptr;  // FP64 scalars: J, theta grads, optimizer values
  double *partC = nullptr, *partG = nullptr, *partT = nullptr;
  double *units = nullptr;   // unit sums [ceil(M / JD_UNIT_PATHS)][1 + Nt du] of the path reduction
  void *traj = nullptr;
  uint32_t *flags = nullptr;
  void *ckpt = nullptr;
  void *log_kt = nullptr, *log_y = nullptr;
  int *jcnt = nullptr;
  int log_cap = 0;
  // second set of the plan's buffers for the paired Armijo trials of jd_optimize
  // (allocated on first use when the memory budget holds it; pair_state 1 ready,
  // -1 unavailable, 0 not tried)
  void *uk2 = nullptr, *traj2 = nullptr, *ckpt2 = nullptr, *log_kt2 = nullptr, *log_y2 = nullptr;
  double *partC2 = nullptr, *opt_ut2 = nullptr;
  int pair_state = 0;
  int64_t chunk = 0;         // stored plan in path blocks of this size (0: all paths at once)
  double *opt_u = nullptr, *opt_ut = nullptr, *opt_g = nullptr;
  int *status_d = nullptr;   // kernel status word (JD_OK or JD_ERR_TIMEOUT)
  void *kp_dev = nullptr;    // coefficient struct of the d = 32 kernels (device copy)
  float *bu_dev = nullptr;   // d = 32: B u_k per step, [Nt][32] (the same for every path)
  double *host_pinned = nullptr;  // small pinned staging buffer
  bool own_pinned = true;
  bool async_alloc = false;  // stream-ordered allocations (server): no device-wide sync on free
  size_t bytes = 0;
  int64_t nblk = 0;
  // feedback control (jd_fb_*): buffers of the last padded size, allocated on use
  void *fb_mu = nullptr, *fb_traj = nullptr;
  uint32_t *fb_flags = nullptr;
  double *fb_mu64 = nullptr, *fb_grad = nullptr, *fb_partC = nullptr, *fb_partG = nullptr;
  void *fb_partW = nullptr;
  void *fb_z0 = nullptr;     // interacting particles: the ring's initial states [2][S], kernel precision
  double *fb_mut = nullptr;  // optimizer: trial weights (FP64)
  int fb_LP = 0;             // padded weights per step of fb_mu / fb_partW / fb_partG
  size_t fb_stack = 0;       // stack limit already ensured for the feedback kernels
};

namespace jd {

// How a problem object gets its resources (jd_problem_create: all owned; the server:
// a slot's stream and pinned buffer, stream-ordered allocations).
struct ProblemOpts {
  cudaStream_t stream = nullptr;     // null: own stream (or desc.cuda_stream)
  double *pinned = nullptr;          // null: own pinned scalar buffer (kScalars doubles)
  bool async_alloc = false;
  bool no_pre = false;               // no draw pre-pass buffers (the problem runs batched sweeps)
};
constexpr int kScalars = 8 + 34 + 4;   // FP64 scalar slots per problem (device and pinned)

jd_status create_problem(const jd_problem_desc &q, const ProblemOpts &o, jd_problem **out);

// Device bytes a problem allocates: the buffers of jd_problem_create plus those of the
// adjoint plan (STORED or RECOMPUTE).  Host arithmetic only.
size_t problem_bytes(const jd_problem_desc &q, jd_adjoint_mode plan);
// The least a problem can run in: RECOMPUTE for d <= 8; for d = 32 the stored plan in
// blocks of 128 paths.
size_t problem_bytes_min(const jd_problem_desc &q);
// Device bytes of the second set of a plan's buffers that jd_optimize's paired Armijo
// trials use (0 where pairs are not used: d > 4).  Host arithmetic only.
size_t pair_bytes(const jd_problem_desc &q, jd_adjoint_mode plan);

// Projected-gradient Armijo iteration (Algorithm 5.4) of one problem as a non-blocking
// state machine: every phase (gradient; one line-search trial; the final copy of u)
// is enqueued on the problem's stream and ends with a copy of the FP64 scalars to
// pinned memory and a record of `ev`; opt_advance, called once `ev` has completed,
// takes the host decision and enqueues the next phase.  jd_optimize drives one
// machine to the end; the server interleaves many.
struct OptMachine {
  enum Phase { IDLE, GRAD, TRIAL, OUTPUT, DONE };
  ::jd_problem *p = nullptr;
  jd_opt_params o{};
  jd_opt_result r{};
  double *J_hist = nullptr;
  double *u_dst = nullptr;
  jd_memspace u_space = JD_MEM_HOST;
  cudaEvent_t ev = nullptr;
  Phase phase = IDLE;
  int it = 0, backtracks = 0, grads = 0;
  double zeta = 1.0, zeta_max = 1e3, pg0 = -1.0;
  bool forward_done = false;
  uint32_t epoch0 = 0;   // the problem's epoch; resampling uses epoch0 + it
  // paired trials: allowed (pairs), whether the running trial is a pair, and the
  // number of consecutive iterations that accepted their first trial point
  bool pairs = false, pair = false;
  int first_accepts = 0;
  // CUDA graphs: each phase's launch sequence is captured on first use and replayed
  // (gradient with and without the forward sweep, single or paired trial), once per
  // assignment of the problem's two buffer sets (bank: swapped when a pair's second
  // point is taken); kernels per graph counted
  bool use_graphs = false;
  int bank = 0;
  cudaGraphExec_t g_grad[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  cudaGraphExec_t g_trial[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  int n_grad[2][2] = {{0, 0}, {0, 0}}, n_trial[2][2] = {{0, 0}, {0, 0}};
  // deferred launches (batched serving): the machine decides its next phase and leaves
  // the phase's work to opt_launch_batch; want = the phase to launch (GRAD or TRIAL, IDLE
  // when none), want_fwd = a gradient with its forward sweep, want_pair = a paired trial
  bool defer = false;
  Phase want = IDLE;
  bool want_fwd = false, want_pair = false;
};
// p->u_in holds u^0.  u_dst (space us) receives the final iterate.
jd_status opt_begin(OptMachine &m, ::jd_problem *p, const jd_opt_params &o, double *u_dst,
                    jd_memspace us, double *J_hist);
jd_status opt_advance(OptMachine &m);
void opt_release(OptMachine &m);   // frees the machine's graphs
// Batched phases: whether a problem's phases can share launches (d <= 2, du = 1, the
// stored plan over all paths at once; the plan's buffers are allocated here); the key of a deferred launch (machines with the
// same key may share one; -1: nothing deferred); and the deferred phases of n <=
// kBatchMax machines with one key, launched together on stream s.  Each machine's event
// is recorded on s after its scalars were copied to its pinned buffer.
bool opt_batchable(::jd_problem *p);
int opt_batch_key(const OptMachine &m);
jd_status opt_launch_batch(OptMachine *const *ms, int n, cudaStream_t s);

}  // namespace jd
