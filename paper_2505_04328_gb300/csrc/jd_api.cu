// jd_api.cu -- host side of the C ABI declared in include/jd.h: validation, memory
// plan, launch sequencing, FP64 finalize kernels and the device-side Armijo test.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "jd_internal.h"

namespace jd {

extern const PathOps ops_f32_d1_u1, ops_f32_d2_u1, ops_f32_d2_u4, ops_f32_d4_u4, ops_f32_d8_u4, ops_f32_d32_u4;
extern const PathOps ops_f64_d1_u1, ops_f64_d2_u1, ops_f64_d2_u4, ops_f64_d4_u4, ops_f64_d8_u4;

static std::atomic<uint64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

// Optional per-kernel-class timing: a CUDA event pair around every launch, on the
// launching stream, summed on read.
enum KernelClass { KC_FWD_COST, KC_FWD_STORE, KC_FWD_CKPT, KC_ADJ_STORED, KC_ADJ_RECOMPUTE,
                   KC_FINALIZE, KC_PREP, KC_OPT, KC_FB_FWD, KC_FB_ADJ, KC_FB_SUR, KC_FB_RED, KC_FB_FIN,
                   KC_FWD_PAIR, KC_COUNT };
static const char *kKernelClassName[KC_COUNT] = {"fwd_cost", "fwd_store", "fwd_ckpt", "adj_stored",
                                                 "adj_recompute", "finalize", "prep_u", "opt_step",
                                                 "fb_fwd", "fb_adj", "fb_sur", "fb_reduce", "fb_finalize",
                                                 "fwd_pair"};
struct ProfRec {
  int kind;
  cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof_recs;
static std::vector<cudaEvent_t> g_prof_pool;

static cudaEvent_t prof_event() {
  cudaEvent_t e = nullptr;
  if (!g_prof_pool.empty()) {
    e = g_prof_pool.back();
    g_prof_pool.pop_back();
  } else {
    cudaEventCreate(&e);
  }
  return e;
}

// Returns a record index or -1 when profiling is off.
static int prof_begin(int kind, cudaStream_t s) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  if (!g_prof_on) return -1;
  ProfRec r{kind, prof_event(), prof_event()};
  cudaEventRecord(r.a, s);
  g_prof_recs.push_back(r);
  return (int)g_prof_recs.size() - 1;
}

static void prof_end(int idx, cudaStream_t s) {
  if (idx < 0) return;
  std::lock_guard<std::mutex> g(g_prof_mu);
  if (idx < (int)g_prof_recs.size()) cudaEventRecord(g_prof_recs[idx].b, s);
}

int compiled_dim(int d) {
  if (d == 1) return 1;
  if (d == 2) return 2;
  if (d <= 4) return 4;
  if (d <= 8) return 8;
  if (d <= 32) return 32;
  return 0;
}

// (D, DU) actually compiled for a (d, du) pair: du == 1 with d <= 2 runs the
// single-control kernels, everything else pads the control to 4 (and d = 1 with
// several controls to D = 2).
static void pick_dims(int d, int du, int *D, int *DU) {
  int Dd = compiled_dim(d);
  if (du == 1 && Dd <= 2) {
    *D = Dd;
    *DU = 1;
    return;
  }
  if (Dd == 1) Dd = 2;
  *D = Dd;
  *DU = 4;
}

extern const FbOps fb_ops_f32[3], fb_ops_f64[3];

const FbOps *fb_ops(int prec, int nx, int nv) {
  const FbOps *t = prec == JD_FP64 ? fb_ops_f64 : fb_ops_f32;
  for (int i = 0; i < 3; ++i)
    if (nx <= t[i].NX && nv <= t[i].NV) return &t[i];
  return nullptr;
}

const PathOps *path_ops_dims(int prec, int D, int DU) {
  const bool f = prec == JD_FP32;
  if (D == 1 && DU == 1) return f ? &ops_f32_d1_u1 : &ops_f64_d1_u1;
  if (D == 2 && DU == 1) return f ? &ops_f32_d2_u1 : &ops_f64_d2_u1;
  if (D == 2 && DU == 4) return f ? &ops_f32_d2_u4 : &ops_f64_d2_u4;
  if (D == 4 && DU == 4) return f ? &ops_f32_d4_u4 : &ops_f64_d4_u4;
  if (D == 8 && DU == 4) return f ? &ops_f32_d8_u4 : &ops_f64_d8_u4;
  if (D == 32 && DU == 4) return f ? &ops_f32_d32_u4 : nullptr;
  return nullptr;
}

// ---------------------------------------------------------------------------
// FP64 finalize kernels (fixed summation order: deterministic)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Scalar slots in p->scal_d
enum { S_J = 0, S_JT = 1, S_DOT = 2, S_PG = 3, S_ACC = 4, S_STEP = 5, S_STATUS = 6, S_BAD = 7, S_THETA = 8,
       S_ZETA = 42, S_JT2 = 44, S_DOT2 = 45 };
constexpr int NSCAL = kScalars;

// Block-wide FP64 sum (blockDim.x == 256) in a fixed tree; result in every thread.
__device__ double block_sum_d(double v, double *sm) {
  v = warp_sum_d(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
    s = warp_sum_d(s);
    if (threadIdx.x == 0) sm[0] = s;
  }
  __syncthreads();
  s = sm[0];
  __syncthreads();
  return s;
}

// ---------------------------------------------------------------------------
// The reduction over paths, defined on units of JD_UNIT_PATHS consecutive paths (128
// blocks, 512 warps): within a unit a fixed tree over its partials, across units a plain
// sum in unit order.  A shard of the paths that starts at a unit boundary yields exactly
// the whole problem's unit sums, so splitting a problem over devices changes no bit.
// ---------------------------------------------------------------------------
constexpr int64_t UNIT_PATHS = JD_UNIT_PATHS;
constexpr int64_t UNIT_BLOCKS = UNIT_PATHS / TPB;
constexpr int64_t UNIT_WARPS = UNIT_PATHS / 32;
static_assert(UNIT_PATHS % TPB == 0, "units hold whole blocks");

inline int64_t n_units(int64_t M) { return ceil_div(M, UNIT_PATHS); }

// units[i][e], e < ne: e = 0 the sum of unit i's cost partials (its blocks), e = 1 + k du + l
// the sum of its gradient partials of entry (k, l) (its warps).  One warp per (unit,
// entry): lane j adds partials j, j + 32, ... in order, then the warp's fixed tree.
// bid: the block's index within this reduction (a batched launch runs several).
__device__ __forceinline__ void unit_sums_body(int64_t bid, const double *__restrict__ partC, int64_t nblk,
                                               const double *__restrict__ partG, int64_t npart, int du, int DU,
                                               int64_t nunits, int ne, double *__restrict__ units) {
  const int64_t gw = (bid * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= nunits * ne) return;   // whole warps (blockDim is a multiple of 32)
  const int64_t i = gw / ne;
  const int e = (int)(gw % ne);
  double s = 0.0;
  if (e == 0) {
    const int64_t b1 = min((i + 1) * UNIT_BLOCKS, nblk);
    for (int64_t b = i * UNIT_BLOCKS + lane; b < b1; b += 32) s += partC[b];
  } else {
    const int k = (e - 1) / du, l = (e - 1) % du;
    const double *row = partG + ((int64_t)k * DU + l) * npart;
    const int64_t w1 = min((i + 1) * UNIT_WARPS, npart);
    for (int64_t w = i * UNIT_WARPS + lane; w < w1; w += 32) s += row[w];
  }
  s = warp_sum_d(s);
  if (lane == 0) units[gw] = s;
}

__global__ void unit_sums_kernel(const double *__restrict__ partC, int64_t nblk, const double *__restrict__ partG,
                                 int64_t npart, int du, int DU, int64_t nunits, int ne, double *__restrict__ units) {
  unit_sums_body(blockIdx.x, partC, nblk, partG, npart, du, DU, nunits, ne, units);
}

// J = (1/M) sum_i units[i][0] + (nu dt / 2) sum_k |u_k|^2          (eq:discrete_functional)
// grad[e-1] = nu dt u[e-1] + (1/M) sum_i units[i][e], e >= 1       (eq:definition_Gradient)
// Sums over units in unit order; sum_k |u_k|^2 as consecutive chunks of 32 squares, each
// added by the xor butterfly of one warp (offsets 16, 8, 4, 2, 1; the two lanes of a pair
// add the same two values, so every lane holds the same sum), the chunk sums added in
// order.  jd_combine_units (host) performs the same operations one for one, so the device
// and the host combine give the same bits.
__device__ __forceinline__ void combine_units_body(int bid, const double *__restrict__ units, int64_t nunits, int ne,
                                                   const double *__restrict__ u, int n, double nu_dt,
                                                   double half_nu_dt, double invM, double *__restrict__ J,
                                                   double *__restrict__ grad, double *__restrict__ bad) {
  const int e = bid * blockDim.x + threadIdx.x;
  if (bid == 0 && threadIdx.x < 32) {   // warp 0 of block 0: J
    const int lane = threadIdx.x;
    double b = 0.0;
    for (int c0 = 0; c0 < n; c0 += 32) {
      const double x = c0 + lane < n ? u[c0 + lane] : 0.0;
      double v = __dmul_rn(x, x);
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
      b = __dadd_rn(b, v);
    }
    if (lane == 0) {
      double s = 0.0;
      for (int64_t i = 0; i < nunits; ++i) s = __dadd_rn(s, units[i * ne]);
      const double v = __fma_rn(half_nu_dt, b, __dmul_rn(s, invM));
      *J = v;
      if (!isfinite(v)) *bad = 1.0;
    }
  }
  if (e >= 1 && e < ne) {
    double s = 0.0;
    for (int64_t i = 0; i < nunits; ++i) s = __dadd_rn(s, units[i * ne + e]);
    const double v = __fma_rn(nu_dt, u[e - 1], __dmul_rn(s, invM));
    grad[e - 1] = v;
    if (!isfinite(v)) *bad = 1.0;
  }
}

__global__ void combine_units_kernel(const double *__restrict__ units, int64_t nunits, int ne,
                                     const double *__restrict__ u, int n, double nu_dt, double half_nu_dt,
                                     double invM, double *__restrict__ J, double *__restrict__ grad,
                                     double *__restrict__ bad) {
  combine_units_body(blockIdx.x, units, nunits, ne, u, n, nu_dt, half_nu_dt, invM, J, grad, bad);
}

// theta[t] = (1/M) sum_b partT[map(t) * nblk + b], map: [0, 1..d, d+1] -> [0, 1..d, D+1]
__global__ void finalize_theta_kernel(const double *__restrict__ partT, int64_t nblk, int d, int D,
                                      double invM, double *__restrict__ out) {
  const int lane = threadIdx.x & 31, t = blockIdx.x;   // one warp-sized block per entry
  const int src = t <= d ? t : D + 1;
  double s = 0.0;
  for (int64_t b = lane; b < nblk; b += 32) s += partT[(int64_t)src * nblk + b];
  s = warp_sum_d(s);
  if (lane == 0) out[t] = s * invM;
}

// Control in kernel precision, padded from du to DU columns.
template <typename R>
__global__ void prep_u_kernel(const double *__restrict__ u, int Nt, int du, int DU, R *__restrict__ uk) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)Nt * DU) return;
  const int k = (int)(i / DU), l = (int)(i % DU);
  uk[i] = l < du ? (R)u[(int64_t)k * du + l] : R(0);
}

// The optimizer's one-block kernels below are bodies (blockDim.x == 256, sm: 32 doubles
// of shared memory) run by their own launch or, one block per problem, by a batched one.

// Control in kernel precision, one block: the elements of prep_u_kernel in a loop.
template <typename R>
__device__ __forceinline__ void prep_u_block(const double *__restrict__ u, int Nt, int du, int DU,
                                             R *__restrict__ uk) {
  for (int64_t i = threadIdx.x; i < (int64_t)Nt * DU; i += blockDim.x) {
    const int k = (int)(i / DU), l = (int)(i % DU);
    uk[i] = l < du ? (R)u[(int64_t)k * du + l] : R(0);
  }
}

// |P(u - g) - u|_{L2} with g = grad / dt; out = value.
__device__ __forceinline__ void opt_pgnorm_body(int n, const double *__restrict__ u, const double *__restrict__ grad,
                                                double dt, double lo, double hi, double *__restrict__ out,
                                                double *sm) {
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double g = grad[i] / dt;
    const double e = fmin(fmax(u[i] - g, lo), hi) - u[i];
    a += dt * e * e;
  }
  a = block_sum_d(a, sm);
  if (threadIdx.x == 0) *out = sqrt(a);
}

__global__ void opt_pgnorm_kernel(int n, const double *__restrict__ u, const double *__restrict__ grad,
                                  double dt, double lo, double hi, double *__restrict__ out) {
  __shared__ double sm[32];
  opt_pgnorm_body(n, u, grad, dt, lo, hi, out, sm);
}

// Trial point ut = clip(u - zeta g) and <g, ut - u>_{L2} = sum grad (ut - u); with ut2
// also the point at zeta / 2 (the second trial of a pair) and its product in dot2.
__device__ __forceinline__ void opt_trial_body(int n, const double *__restrict__ u, const double *__restrict__ grad,
                                               double zeta, double dt, double lo, double hi,
                                               double *__restrict__ ut, double *__restrict__ dot,
                                               double *__restrict__ ut2, double *__restrict__ dot2, double *sm) {
  for (int h = 0; h < (ut2 ? 2 : 1); ++h) {
    const double z = h ? 0.5 * zeta : zeta;
    double *w = h ? ut2 : ut;
    double a = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double g = grad[i] / dt;
      const double v = fmin(fmax(u[i] - z * g, lo), hi);
      w[i] = v;
      a += dt * g * (v - u[i]);
    }
    a = block_sum_d(a, sm);
    if (threadIdx.x == 0) *(h ? dot2 : dot) = a;
  }
}

__global__ void opt_trial_kernel(int n, const double *__restrict__ u, const double *__restrict__ grad,
                                 const double *__restrict__ zeta_p, double dt, double lo, double hi,
                                 double *__restrict__ ut, double *__restrict__ dot, double *__restrict__ ut2,
                                 double *__restrict__ dot2) {
  __shared__ double sm[32];
  opt_trial_body(n, u, grad, *zeta_p, dt, lo, hi, ut, dot, ut2, dot2, sm);
}

// Armijo test J(ut) <= J(u) + c <g, ut - u>; on acceptance u <- ut and J <- J(ut).
// s: [0] J(u), [1] J(ut), [2] dot, [4] accepted (out), [5] |ut - u|^2_{L2} (out).
// With ut2 (a pair of trials, ut2 at half the step, J(ut2) and its product in
// s[S_JT2], s[S_DOT2]) the points are tested in the order of backtracking and the first
// that passes is taken: s[4] = 1 (ut), 2 (ut2) or 0, s[5] the squared step of the taken
// point (of ut2 when neither passes).
__device__ __forceinline__ void opt_accept_body(int n, double *__restrict__ u, const double *__restrict__ ut,
                                                const double *__restrict__ ut2, double c, double dt,
                                                double *__restrict__ s, double *sm) {
  const bool acc1 = s[1] <= s[0] + c * s[2];
  const bool acc2 = ut2 && !acc1 && s[S_JT2] <= s[0] + c * s[S_DOT2];
  const double *w = (ut2 && !acc1) ? ut2 : ut;
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double e = w[i] - u[i];
    a += dt * e * e;
  }
  a = block_sum_d(a, sm);
  if (acc1 || acc2)
    for (int i = threadIdx.x; i < n; i += blockDim.x) u[i] = w[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    s[4] = acc1 ? 1.0 : (acc2 ? 2.0 : 0.0);
    s[5] = a;
    if (acc1) s[0] = s[1];
    if (acc2) s[0] = s[1] = s[S_JT2];
  }
}

__global__ void opt_accept_kernel(int n, double *__restrict__ u, const double *__restrict__ ut,
                                  const double *__restrict__ ut2, double c, double dt, double *__restrict__ s) {
  __shared__ double sm[32];
  opt_accept_body(n, u, ut, ut2, c, dt, s, sm);
}

// ---------------------------------------------------------------------------
// Batched optimizer phases: several problems' phase work in shared launches, one block
// (small kernels) or one range of blocks (reductions, sweeps) per problem.  Each block
// runs the body of the single-problem kernel with its index within its problem, so every
// problem gets the bits of its own launches.
// ---------------------------------------------------------------------------
struct OptBatchItem {
  int n, Nt, du, DU;
  int trial;                      // a trial phase (else a gradient phase)
  int fwd;                        // gradient phase with its forward sweep: the control into uk
  double dt, lo, hi, c, zeta;
  double *u, *grad, *ut, *ut2;    // ut2: the second point of a paired trial (else null)
  double *scal;
  void *uk, *uk2;
};
struct OptBatch {
  int n;
  OptBatchItem it[kBatchMax];
};

// Before the sweeps, one block per problem.  Gradient phase: clear the status word and
// the non-finite flag (the bytes of clear_bad's memset); with the forward sweep, the
// control in kernel precision.  Trial phase: the trial point(s) and their products
// (opt_trial at the machine's zeta), then the point(s) in kernel precision.
template <typename R>
__global__ void opt_pre_batch_kernel(const __grid_constant__ OptBatch t) {
  __shared__ double sm[32];
  const OptBatchItem &b = t.it[blockIdx.x];
  if (!b.trial) {
    if (threadIdx.x < 2) b.scal[S_STATUS + threadIdx.x] = 0.0;
    if (b.fwd) prep_u_block<R>(b.u, b.Nt, b.du, b.DU, static_cast<R *>(b.uk));
    return;
  }
  if (threadIdx.x == 0) b.scal[S_ZETA] = b.zeta;
  opt_trial_body(b.n, b.u, b.grad, b.zeta, b.dt, b.lo, b.hi, b.ut, b.scal + S_DOT, b.ut2, b.scal + S_DOT2, sm);
  __syncthreads();
  prep_u_block<R>(b.ut, b.Nt, b.du, b.DU, static_cast<R *>(b.uk));
  if (b.ut2) prep_u_block<R>(b.ut2, b.Nt, b.du, b.DU, static_cast<R *>(b.uk2));
}

// After the reductions, one block per problem: the projected-gradient norm (gradient
// phase) or the Armijo test (trial phase).
__global__ void opt_post_batch_kernel(const __grid_constant__ OptBatch t) {
  __shared__ double sm[32];
  const OptBatchItem &b = t.it[blockIdx.x];
  if (b.trial)
    opt_accept_body(b.n, b.u, b.ut, b.ut2, b.c, b.dt, b.scal, sm);
  else
    opt_pgnorm_body(b.n, b.u, b.grad, b.dt, b.lo, b.hi, b.scal + S_PG, sm);
}

// The job of a block of a batched reduction: first[i] <= blockIdx.x < first[i + 1].
__device__ __forceinline__ int batch_job(const int *first, int n) {
  int i = 0;
  while (i + 1 < n && (int)blockIdx.x >= first[i + 1]) ++i;
  return i;
}

struct UnitJob {
  const double *partC, *partG;
  int64_t nblk, npart, nunits;
  int du, DU, ne;
  double *units;
};
struct UnitBatch {
  int n;
  int first[2 * kBatchMax + 1];
  UnitJob j[2 * kBatchMax];
};
__global__ void unit_sums_batch_kernel(const __grid_constant__ UnitBatch t) {
  const int i = batch_job(t.first, t.n);
  const UnitJob &j = t.j[i];
  unit_sums_body(blockIdx.x - t.first[i], j.partC, j.nblk, j.partG, j.npart, j.du, j.DU, j.nunits, j.ne, j.units);
}

struct CombineJob {
  const double *units, *u;
  int64_t nunits;
  int ne, n;
  double nu_dt, half_nu_dt, invM;
  double *J, *grad, *bad;
};
struct CombineBatch {
  int n;
  int first[2 * kBatchMax + 1];
  CombineJob j[2 * kBatchMax];
};
__global__ void combine_units_batch_kernel(const __grid_constant__ CombineBatch t) {
  const int i = batch_job(t.first, t.n);
  const CombineJob &j = t.j[i];
  combine_units_body(blockIdx.x - t.first[i], j.units, j.nunits, j.ne, j.u, j.n, j.nu_dt, j.half_nu_dt, j.invM,
                     j.J, j.grad, j.bad);
}

}  // namespace jd

using namespace jd;

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

static jd_status fail(jd_status s, const std::string &msg) {
  g_last_error = msg;
  return s;
}

static jd_status cuda_fail(cudaError_t e, const char *what) {
  return fail(JD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define JD_CUDA(call)                                      \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
  } while (0)


static bool finite_all(const double *a, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

static size_t elem_size(const jd_problem *p) { return p->desc.prec == JD_FP64 ? 8 : 4; }

template <typename T>
static void free_dev(const jd_problem *p, T *&ptr) {
  if (ptr) {
    if (p->async_alloc)
      cudaFreeAsync((void *)ptr, p->stream);
    else
      cudaFree((void *)ptr);
  }
  ptr = nullptr;
}

static jd_status dev_alloc(jd_problem *p, void **ptr, size_t bytes, const char *what) {
  if (p->bytes + bytes > p->budget)
    return fail(JD_ERR_OOM, std::string("memory budget exceeded allocating ") + what);
  cudaError_t e = p->async_alloc ? cudaMallocAsync(ptr, bytes, p->stream) : cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(JD_ERR_OOM, std::string("cudaMalloc failed for ") + what + ": " + cudaGetErrorString(e));
  }
  p->bytes += bytes;
  return JD_OK;
}

// Jump-log capacity per path: mean jump count lambda T plus a wide Poisson margin
// (steps that do not fit are regenerated by the adjoint, so this only trades memory
// for speed).
static int log_capacity(const jd_problem_desc &q) {
  if (q.jump_law == JD_JUMP_NONE || q.lambda <= 0.0) return 0;
  const double mean = q.lambda * q.T;
  double c = std::ceil(mean + 6.0 * std::sqrt(mean) + 8.0);
  if (c > 1024.0) c = 1024.0;
  return (int)c;
}

// Bytes of the stored plan for M paths: states, jump flags, jump log (at least one
// record per path is allocated) and the per-path log counts and closing steps.
static size_t stored_plan_bytes(const jd_problem_desc &q, int D, size_t es, int64_t M) {
  const int cap = log_capacity(q);
  const size_t capa = (size_t)(cap > 0 ? cap : 1);
  return traj_values(q.Nt, D, (int)es, M) * es + (size_t)ceil_div(q.Nt, 32) * M * 4 + capa * M * 2 * es +
         capa * M * D * es + (size_t)M * 8;
}

static size_t stored_bytes(const jd_problem *p) {
  return stored_plan_bytes(p->desc, p->D, elem_size(p), p->desc.M);
}

static PathBufs plan_bufs(const jd_problem *p) {
  PathBufs b;
  b.traj = p->traj;
  b.flags = p->flags;
  b.ckpt = p->ckpt;
  b.log_kt = p->log_kt;
  b.log_y = p->log_y;
  b.jcnt = p->jcnt;
  b.log_cap = p->log_cap;
  b.partC = p->partC;
  b.partG = p->partG;
  b.partT = p->partT;
  b.status = reinterpret_cast<int *>(p->scal_d + S_STATUS);
  b.pre_w = p->pre_w;
  b.pre_z = p->pre_z;
  b.pre_key = p->pre_key;
  return b;
}

// Checkpoint bytes of the recompute plan with segments of S steps.
static size_t ckpt_bytes(const jd_problem_desc &q, int D, size_t es, int S) {
  return (size_t)(ceil_div(q.Nt, S) + 1) * D * (size_t)q.M * es;
}

static size_t recompute_bytes(const jd_problem *p) { return ckpt_bytes(p->desc, p->D, elem_size(p), p->S); }

// Checkpoint spacing of the recompute plan: 16 steps, or (when the budget does not hold
// those checkpoints) the smallest of 32 and 64 whose checkpoints fit and whose segment
// buffer fits a block's shared memory with the parameter gradients (S ~ sqrt(N_t) for
// N_t near 4096).  0 when none fits.
static int choose_spacing(const jd_problem *p, size_t avail) {
  int smax = 0;
  if (cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device) != cudaSuccess)
    smax = 232448;
  for (int S = 16; S <= 64; S *= 2) {
    if (p->ops->rc_smem && p->ops->rc_smem(true, S) > (size_t)smax && S > 16) break;
    if (ckpt_bytes(p->desc, p->D, elem_size(p), S) <= avail) return S;
  }
  return 0;
}

// Buffers jd_problem_create allocates (the ALLOC list there).
static size_t base_bytes(const jd_problem_desc &q, int D, int DU, size_t es) {
  const size_t nu = (size_t)q.Nt * q.du, nblk = (size_t)ceil_div(q.M, TPB);
  return (size_t)q.Nt * DU * es + (size_t)(q.Nt + 1) * D * es + 4 * nu * 8 + NSCAL * 8 + nblk * 8 +
         (size_t)q.Nt * DU * grad_parts(q.M) * 8 + (size_t)(D + 2) * nblk * 8 +
         (size_t)ceil_div(q.M, JD_UNIT_PATHS) * (1 + nu) * 8 +
         (pre_pass(q.d, q.Nt, q.M, es) ? pre_bytes(q.Nt, D, q.M, es) : 0) +
         (D == 32 ? 16384 + (size_t)q.Nt * 32 * sizeof(float) : 0);
}

// Allocate the trajectory or checkpoint buffers on first use.
static jd_status ensure_plan(jd_problem *p) {
  if (p->plan != JD_ADJ_AUTO) return JD_OK;
  jd_adjoint_mode want = p->desc.mode;
  if (p->D == 32) {   // the d = 32 kernels have the stored variant only
    if (want == JD_ADJ_RECOMPUTE)
      return fail(JD_ERR_UNSUPPORTED, "the recompute adjoint is not built for 8 < d <= 32");
    want = JD_ADJ_STORED;
  }
  if (want == JD_ADJ_AUTO)
    want = (p->bytes + stored_bytes(p) <= p->budget) ? JD_ADJ_STORED : JD_ADJ_RECOMPUTE;
  if (want == JD_ADJ_STORED) {
    int64_t M = p->desc.M;
    if (p->D == 32 && p->bytes + stored_bytes(p) > p->budget) {
      // no recompute adjoint at d = 32: store the paths block by block, the largest
      // multiple of 128 paths whose states fit what is left of the budget
      const size_t avail = p->budget > p->bytes ? p->budget - p->bytes : 0;
      const size_t per128 = stored_plan_bytes(p->desc, p->D, elem_size(p), TPB);
      int64_t c = (int64_t)(avail / per128) * TPB;
      while (c >= TPB && stored_plan_bytes(p->desc, p->D, elem_size(p), c) > avail) c -= TPB;
      if (c < TPB) return fail(JD_ERR_OOM, "the memory budget does not hold the states of 128 paths");
      p->chunk = c;
      M = c;
    }
    jd_status s = dev_alloc(p, &p->traj, traj_values(p->desc.Nt, p->D, (int)elem_size(p), M) * elem_size(p),
                            "trajectory");
    if (s) return s;
    s = dev_alloc(p, (void **)&p->flags, (size_t)ceil_div(p->desc.Nt, 32) * M * 4, "jump flags");
    if (s) return s;
    p->log_cap = log_capacity(p->desc);
    const size_t cap = (size_t)(p->log_cap > 0 ? p->log_cap : 1);
    s = dev_alloc(p, &p->log_kt, cap * M * 2 * elem_size(p), "jump log");
    if (s) return s;
    s = dev_alloc(p, &p->log_y, cap * M * p->D * elem_size(p), "jump log states");
    if (s) return s;
    s = dev_alloc(p, (void **)&p->jcnt, (size_t)M * 8, "jump log counts");
    if (s) return s;
  } else {
    const size_t avail = p->budget > p->bytes ? p->budget - p->bytes : 0;
    const int S = choose_spacing(p, avail);
    if (!S) return fail(JD_ERR_OOM, "the memory budget does not hold the checkpoints of the recompute plan");
    p->S = S;
    jd_status s = dev_alloc(p, &p->ckpt, recompute_bytes(p), "checkpoints");
    if (s) return s;
  }
  p->plan = want;
  return JD_OK;
}

// u (Nt*du, host or device) -> p->u_in (FP64 device) -> p->uk (kernel precision, padded)
static jd_status load_u(jd_problem *p, const double *u, jd_memspace us) {
  const size_t n = (size_t)p->desc.Nt * p->desc.du;
  if (!u) return fail(JD_ERR_INVALID_ARG, "u is NULL");
  if (us == JD_MEM_HOST) {
    if (!finite_all(u, n)) return fail(JD_ERR_INVALID_ARG, "u has a non-finite entry");
    JD_CUDA(cudaMemcpyAsync(p->u_in, u, n * sizeof(double), cudaMemcpyHostToDevice, p->stream));
  } else if (us == JD_MEM_DEVICE) {
    if (u != p->u_in)
      JD_CUDA(cudaMemcpyAsync(p->u_in, u, n * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
  } else {
    return fail(JD_ERR_INVALID_ARG, "bad memory space for u");
  }
  return JD_OK;
}

static jd_status prep_u(jd_problem *p, const double *ud, void *dst = nullptr) {
  const int64_t n = (int64_t)p->desc.Nt * p->DU;
  const unsigned grid = (unsigned)ceil_div(n, 256);
  if (!dst) dst = p->uk;
  const int pr = prof_begin(KC_PREP, p->stream);
  if (p->desc.prec == JD_FP64)
    prep_u_kernel<double><<<grid, 256, 0, p->stream>>>(ud, p->desc.Nt, p->desc.du, p->DU, (double *)dst);
  else
    prep_u_kernel<float><<<grid, 256, 0, p->stream>>>(ud, p->desc.Nt, p->desc.du, p->DU, (float *)dst);
  prof_end(pr, p->stream);
  count_launch();
  JD_CUDA(cudaGetLastError());
  return JD_OK;
}

// Unit sums of the launch's partials (ne = 1: cost only; 1 + Nt du: cost and gradient)
// into p->units.
static jd_status unit_sums(jd_problem *p, int ne, const double *partC = nullptr) {
  const jd_problem_desc &q = p->desc;
  const int64_t nun = n_units(q.M), warps = nun * ne;
  unit_sums_kernel<<<(unsigned)ceil_div(warps * 32, 256), 256, 0, p->stream>>>(
      partC ? partC : p->partC, p->nblk, p->partG, grad_parts(q.M), q.du, p->DU, nun, ne, p->units);
  count_launch();
  JD_CUDA(cudaGetLastError());
  return JD_OK;
}

// J (scalar slot) and, for ne > 1, the gradient (grad_d) from p->units.
static jd_status combine_units(jd_problem *p, const double *ud, int ne, int slot) {
  const jd_problem_desc &q = p->desc;
  const double dt = q.T / q.Nt;
  combine_units_kernel<<<(unsigned)ceil_div(ne, 128), 128, 0, p->stream>>>(
      p->units, n_units(q.M), ne, ud, q.Nt * q.du, q.nu * dt, 0.5 * q.nu * dt, 1.0 / (double)q.M,
      p->scal_d + slot, p->grad_d, p->scal_d + S_BAD);
  count_launch();
  JD_CUDA(cudaGetLastError());
  return JD_OK;
}

static jd_status finalize_cost(jd_problem *p, const double *ud, int slot, const double *partC = nullptr) {
  const int pr = prof_begin(KC_FINALIZE, p->stream);
  jd_status s = unit_sums(p, 1, partC);
  if (!s) s = combine_units(p, ud, 1, slot);
  prof_end(pr, p->stream);
  return s;
}

// finalize = false: stop at the unit sums (p->units), for jd_cost_units.
static jd_status run_cost(jd_problem *p, const double *ud, int slot, bool finalize = true) {
  jd_status s = prep_u(p, ud);
  if (s) return s;
  const int pr = prof_begin(KC_FWD_COST, p->stream);
  const cudaError_t e = p->ops->fwd(p, FWD_COST, 0, p->desc.M, p->uk, plan_bufs(p), p->stream);
  prof_end(pr, p->stream);
  JD_CUDA(e);
  if (!finalize) return unit_sums(p, 1);
  return finalize_cost(p, ud, slot);
}

// Forward sweep in the plan's mode (stored states or checkpoints) and J.  Used for the
// line-search trials of jd_optimize, so that the accepted trial's sweep is the forward
// half of the next gradient.
static jd_status run_plan_forward(jd_problem *p, const double *ud, int slot) {
  jd_status s = ensure_plan(p);
  if (s) return s;
  if (p->chunk) return run_cost(p, ud, slot);   // block-wise stored plan: nothing to keep
  s = prep_u(p, ud);
  if (s) return s;
  const PathBufs b = plan_bufs(p);
  const bool stored = p->plan == JD_ADJ_STORED;
  const int pr = prof_begin(stored ? KC_FWD_STORE : KC_FWD_CKPT, p->stream);
  const cudaError_t e = p->ops->fwd(p, stored ? FWD_STORE : FWD_CKPT, 0, p->desc.M, p->uk, b, p->stream);
  prof_end(pr, p->stream);
  JD_CUDA(e);
  return finalize_cost(p, ud, slot);
}

// Paired sweeps pay where the second control adds little to the draws' cost: d <= 4
// (measured: a pair costs 1.2-1.36 single sweeps there; at d = 8 the second state and its
// drift double the register footprint, 2.5 single sweeps in FP32).
static bool pairs_built(int D) { return D <= 4; }

// Second set of the plan's buffers for paired trials: allocated once, when the memory
// budget holds it beside everything else; not for the block-wise stored plan nor d > 4.
static bool ensure_pair(jd_problem *p) {
  if (p->pair_state) return p->pair_state > 0;
  p->pair_state = -1;
  if (!pairs_built(p->D) || ensure_plan(p) || p->chunk) return false;
  const jd_problem_desc &q = p->desc;
  const size_t es = elem_size(p), n = (size_t)q.Nt * q.du, M = (size_t)q.M;
  const bool stored = p->plan == JD_ADJ_STORED;
  const size_t cap = (size_t)(p->log_cap > 0 ? p->log_cap : 1);
  const size_t b_traj = traj_values(q.Nt, p->D, (int)es, (int64_t)M) * es;
  if (p->bytes + jd::pair_bytes(q, p->plan) > p->budget) return false;
  const std::string saved_error = g_last_error;   // a failed allocation here is not the caller's error
  jd_status s = dev_alloc(p, &p->uk2, (size_t)q.Nt * p->DU * es, "paired control");
  if (!s) s = dev_alloc(p, (void **)&p->partC2, (size_t)p->nblk * 8, "paired cost partials");
  if (!s) s = dev_alloc(p, (void **)&p->opt_ut2, n * 8, "paired trial");
  if (!s && stored) s = dev_alloc(p, &p->traj2, b_traj, "paired trajectory");
  if (!s && stored) s = dev_alloc(p, &p->log_kt2, cap * M * 2 * es, "paired jump log");
  if (!s && stored) s = dev_alloc(p, &p->log_y2, cap * M * p->D * es, "paired jump log states");
  if (!s && !stored) s = dev_alloc(p, &p->ckpt2, recompute_bytes(p), "paired checkpoints");
  if (s) {   // single trials; what was allocated is freed with the problem
    g_last_error = saved_error;
    return false;
  }
  p->pair_state = 1;
  return true;
}

// The second set becomes the plan's (after the second trial of a pair was taken).
static void swap_pair(jd_problem *p) {
  std::swap(p->uk, p->uk2);
  std::swap(p->partC, p->partC2);
  std::swap(p->traj, p->traj2);
  std::swap(p->log_kt, p->log_kt2);
  std::swap(p->log_y, p->log_y2);
  std::swap(p->ckpt, p->ckpt2);
}

// Paired forward sweep (FWD_PAIR) of ud and ud2 on the same random data, in the plan's
// mode: ud's outputs in the plan's buffers, ud2's in the second set; J(ud) to slot,
// J(ud2) to slot2.
static jd_status run_pair_forward(jd_problem *p, const double *ud, int slot, const double *ud2, int slot2) {
  jd_status s = prep_u(p, ud);
  if (!s) s = prep_u(p, ud2, p->uk2);
  if (s) return s;
  PathBufs b = plan_bufs(p);
  b.uk2 = p->uk2;
  b.traj2 = p->traj2;
  b.ckpt2 = p->ckpt2;
  b.log_kt2 = p->log_kt2;
  b.log_y2 = p->log_y2;
  b.partC2 = p->partC2;
  const bool stored = p->plan == JD_ADJ_STORED;
  const int pr = prof_begin(KC_FWD_PAIR, p->stream);
  const cudaError_t e =
      p->ops->fwd(p, (stored ? FWD_STORE : FWD_CKPT) | FWD_PAIR, 0, p->desc.M, p->uk, b, p->stream);
  prof_end(pr, p->stream);
  JD_CUDA(e);
  s = finalize_cost(p, ud, slot);
  if (!s) s = finalize_cost(p, ud2, slot2, p->partC2);
  return s;
}

// Gradient at ud.  With forward_done the stored states / checkpoints, the control in
// kernel precision and the cost partials already belong to ud (the accepted trial of
// the previous line search), and only the adjoint half runs.
// finalize = false: stop at the unit sums (p->units), for jd_gradient_units.
static jd_status run_gradient(jd_problem *p, const double *ud, bool theta, bool forward_done = false,
                              bool finalize = true) {
  jd_status s = ensure_plan(p);
  if (s) return s;
  const jd_problem_desc &q = p->desc;
  const int64_t M = q.M;
  cudaError_t e1 = cudaSuccess, e2;
  const PathBufs b = plan_bufs(p);
  if (!forward_done) {
    s = prep_u(p, ud);
    if (s) return s;
  }
  if (p->plan == JD_ADJ_STORED && p->chunk) {
    // block-wise stored plan: forward and adjoint per block of paths; the blocks write
    // their cost and gradient partials at their global positions, so the reductions
    // see the same partials as one launch over all paths
    for (int64_t c0 = 0; c0 < M && e1 == cudaSuccess; c0 += p->chunk) {
      const int64_t cn = std::min(p->chunk, M - c0);
      PathBufs bc = b;
      bc.partC = b.partC + c0 / TPB;
      bc.partG = b.partG + c0 / 32;
      bc.npart = grad_parts(M);
      int pr = prof_begin(KC_FWD_STORE, p->stream);
      e1 = p->ops->fwd(p, FWD_STORE, c0, cn, p->uk, bc, p->stream);
      prof_end(pr, p->stream);
      if (e1 != cudaSuccess) break;
      pr = prof_begin(KC_ADJ_STORED, p->stream);
      e1 = p->ops->adj(p, ADJ_STORED_V, theta, c0, cn, p->uk, bc, p->stream);
      prof_end(pr, p->stream);
    }
    e2 = cudaSuccess;
  } else if (p->plan == JD_ADJ_STORED) {
    if (!forward_done) {
      const int pr = prof_begin(KC_FWD_STORE, p->stream);
      e1 = p->ops->fwd(p, FWD_STORE, 0, M, p->uk, b, p->stream);
      prof_end(pr, p->stream);
    }
    const int pr = prof_begin(KC_ADJ_STORED, p->stream);
    e2 = p->ops->adj(p, ADJ_STORED_V, theta, 0, M, p->uk, b, p->stream);
    prof_end(pr, p->stream);
  } else {
    if (!forward_done) {
      const int pr = prof_begin(KC_FWD_CKPT, p->stream);
      e1 = p->ops->fwd(p, FWD_CKPT, 0, M, p->uk, b, p->stream);
      prof_end(pr, p->stream);
    }
    const int pr = prof_begin(KC_ADJ_RECOMPUTE, p->stream);
    e2 = p->ops->adj(p, ADJ_RECOMPUTE_V, theta, 0, M, p->uk, b, p->stream);
    prof_end(pr, p->stream);
  }
  JD_CUDA(e1);
  JD_CUDA(e2);
  const int ne = 1 + q.Nt * q.du;
  const int pr = prof_begin(KC_FINALIZE, p->stream);
  s = unit_sums(p, ne);
  if (!s && finalize) s = combine_units(p, ud, ne, S_J);
  prof_end(pr, p->stream);
  if (s) return s;
  if (theta) {
    finalize_theta_kernel<<<q.d + 2, 32, 0, p->stream>>>(p->partT, p->nblk, q.d, p->D,
                                                               1.0 / (double)M, p->scal_d + S_THETA);
    count_launch();
    JD_CUDA(cudaGetLastError());
  }
  return JD_OK;
}

// Copy n scalars from scal_d to the pinned staging buffer and wait.
static jd_status read_scalars(jd_problem *p, int first, int n) {
  JD_CUDA(cudaMemcpyAsync(p->host_pinned + first, p->scal_d + first, n * sizeof(double),
                          cudaMemcpyDeviceToHost, p->stream));
  JD_CUDA(cudaStreamSynchronize(p->stream));
  return JD_OK;
}

// Status after host scalars were read: a bounded device wait that gave up, then
// non-finite results.
static jd_status status_of_scalars(jd_problem *p) {
  if (*reinterpret_cast<const int *>(p->host_pinned + S_STATUS) == (int)JD_ERR_TIMEOUT)
    return fail(JD_ERR_TIMEOUT, "a bounded tensor-core wait timed out");
  if (p->host_pinned[S_BAD] != 0.0) return fail(JD_ERR_NONFINITE, "cost or gradient is not finite");
  return JD_OK;
}

static jd_status check_bad(jd_problem *p) {
  jd_status s = read_scalars(p, S_STATUS, 2);
  if (s) return s;
  return status_of_scalars(p);
}

static jd_status clear_bad(jd_problem *p) {
  JD_CUDA(cudaMemsetAsync(p->scal_d + S_STATUS, 0, 2 * sizeof(double), p->stream));
  return JD_OK;
}

static jd_status set_device(const jd_problem *p) {
  int cur = -1;
  JD_CUDA(cudaGetDevice(&cur));
  if (cur != p->device) JD_CUDA(cudaSetDevice(p->device));
  return JD_OK;
}

// Padded target in kernel precision, p->xd -> p->xdk, in stream order; returns after
// the copy has completed (the staging vector is local).
static cudaError_t upload_target(jd_problem *p) {
  const jd_problem_desc &q = p->desc;
  std::vector<double> xdp((size_t)(q.Nt + 1) * p->D, 0.0);
  for (int k = 0; k <= q.Nt; ++k)
    for (int c = 0; c < q.d; ++c) xdp[(size_t)k * p->D + c] = p->xd[(size_t)k * q.d + c];
  std::vector<float> xf;
  const void *src = xdp.data();
  size_t bytes = xdp.size() * 8;
  if (q.prec == JD_FP32) {
    xf.assign(xdp.begin(), xdp.end());
    src = xf.data();
    bytes = xf.size() * 4;
  }
  cudaError_t e = cudaMemcpyAsync(p->xdk, src, bytes, cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  return e;
}

// Checks of jd_problem_create, shared with jd_problem_update.
static jd_status validate_desc(const jd_problem_desc &q) {
  if (q.d < 1 || q.du < 1) return fail(JD_ERR_INVALID_ARG, "d and du must be >= 1");
  if (q.d > 32) return fail(JD_ERR_UNSUPPORTED, "d > 32 is not compiled");
  if (q.d > 8 && (q.prec != JD_FP32 || q.drift != JD_DRIFT_LINEAR))
    return fail(JD_ERR_UNSUPPORTED, "8 < d <= 32 is built for FP32 paths with a linear drift only");
  if (q.du > 4) return fail(JD_ERR_UNSUPPORTED, "du > 4 is not compiled");
  if (q.Nt < 1 || q.Nt > (1 << 24)) return fail(JD_ERR_INVALID_ARG, "Nt must be in [1, 2^24]");
  if (q.M < 1 || q.M > 0xFFFFFFFFll) return fail(JD_ERR_INVALID_ARG, "M must be in [1, 2^32 - 1]");
  if (q.m_offset < 0 || q.m_offset + q.M > 0x100000000ll)
    return fail(JD_ERR_INVALID_ARG, "m_offset must be >= 0 with m_offset + M <= 2^32");
  if (!(q.T > 0.0) || !std::isfinite(q.T)) return fail(JD_ERR_INVALID_ARG, "T must be finite and > 0");
  if (q.drift != JD_DRIFT_LINEAR && q.drift != JD_DRIFT_CUBIC) return fail(JD_ERR_INVALID_ARG, "bad drift");
  if (q.jump_law < JD_JUMP_NONE || q.jump_law > JD_JUMP_KS) return fail(JD_ERR_INVALID_ARG, "bad jump law");
  if (q.jump_law == JD_JUMP_KS && q.d > 8)
    return fail(JD_ERR_UNSUPPORTED, "the Keilson-Storer law is built for d <= 8");
  if (q.jump_law == JD_JUMP_KS && !std::isfinite(q.jump_gain))
    return fail(JD_ERR_INVALID_ARG, "jump_gain must be finite");
  if (q.prec != JD_FP32 && q.prec != JD_FP64) return fail(JD_ERR_INVALID_ARG, "bad precision");
  if (q.mode < JD_ADJ_AUTO || q.mode > JD_ADJ_RECOMPUTE) return fail(JD_ERR_INVALID_ARG, "bad adjoint mode");
  if (!q.A || !q.B || !q.sigma || !q.x0 || !q.q || !q.xd)
    return fail(JD_ERR_INVALID_ARG, "A, B, sigma, x0, q, xd must be non-NULL");
  if (q.drift == JD_DRIFT_CUBIC && !q.C) return fail(JD_ERR_INVALID_ARG, "C must be non-NULL for CUBIC");
  if (!(q.lambda >= 0.0) || !std::isfinite(q.lambda)) return fail(JD_ERR_INVALID_ARG, "lambda must be finite and >= 0");
  if (!(q.jump_scale >= 0.0) || !std::isfinite(q.jump_scale))
    return fail(JD_ERR_INVALID_ARG, "jump_scale must be finite and >= 0");
  if (!std::isfinite(q.nu) || q.nu < 0.0) return fail(JD_ERR_INVALID_ARG, "nu must be finite and >= 0");
  if (!(q.u_min <= q.u_max)) return fail(JD_ERR_INVALID_ARG, "u_min must be <= u_max");
  if (q.use_tensor_cores < 0 || q.use_tensor_cores > 3)
    return fail(JD_ERR_INVALID_ARG,
                "use_tensor_cores must be 0, 1 (BF16), 2 (BF16 x3) or 3 (BF16 x3 in the adjoint only)");
  if (q.use_tensor_cores && q.d <= 8)
    return fail(JD_ERR_UNSUPPORTED, "tensor cores are used for 8 < d <= 32 (linear drift, FP32)");
  const size_t dd = (size_t)q.d * q.d, dn = (size_t)(q.Nt + 1) * q.d;
  if (!finite_all(q.A, dd) || !finite_all(q.B, (size_t)q.d * q.du) || !finite_all(q.sigma, q.d) ||
      !finite_all(q.x0, q.d) || !finite_all(q.q, q.d) || !finite_all(q.xd, dn) ||
      (q.drift == JD_DRIFT_CUBIC && !finite_all(q.C, dd)) || (q.dA && !finite_all(q.dA, dd)))
    return fail(JD_ERR_INVALID_ARG, "a coefficient array has a non-finite entry");

  return JD_OK;
}


// ---------------------------------------------------------------------------
// Optimizer state machine (Algorithm 5.4, eq:Stochastic_Armijo)
// ---------------------------------------------------------------------------

// Work of a gradient phase: gradient at u^n (the accepted trial's forward sweep is reused
// when forward_done), projected-gradient norm, first scalars to pinned memory.
static jd_status enqueue_grad(jd_problem *p, bool forward_done) {
  const jd_problem_desc &q = p->desc;
  jd_status s = clear_bad(p);
  if (!s) s = run_gradient(p, p->opt_u, false, forward_done);
  if (s) return s;
  const int pr = prof_begin(KC_OPT, p->stream);
  opt_pgnorm_kernel<<<1, 256, 0, p->stream>>>(q.Nt * q.du, p->opt_u, p->grad_d, q.T / q.Nt, q.u_min, q.u_max,
                                              p->scal_d + S_PG);
  prof_end(pr, p->stream);
  count_launch();
  JD_CUDA(cudaGetLastError());
  JD_CUDA(cudaMemcpyAsync(p->host_pinned, p->scal_d, 8 * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  return JD_OK;
}

// Work of a trial phase: zeta from pinned memory, trial point, forward sweep in the
// plan's mode, device-side acceptance test, first scalars to pinned memory.  pair: the
// trial points at zeta and zeta / 2 in one paired sweep, tested in that order.
static jd_status enqueue_trial(jd_problem *p, double armijo_c, bool pair) {
  const jd_problem_desc &q = p->desc;
  const int n = q.Nt * q.du;
  const double dt = q.T / q.Nt;
  JD_CUDA(cudaMemcpyAsync(p->scal_d + S_ZETA, p->host_pinned + S_ZETA, sizeof(double), cudaMemcpyHostToDevice,
                          p->stream));
  int pr = prof_begin(KC_OPT, p->stream);
  opt_trial_kernel<<<1, 256, 0, p->stream>>>(n, p->opt_u, p->grad_d, p->scal_d + S_ZETA, dt, q.u_min, q.u_max,
                                             p->opt_ut, p->scal_d + S_DOT, pair ? p->opt_ut2 : nullptr,
                                             p->scal_d + S_DOT2);
  prof_end(pr, p->stream);
  count_launch();
  JD_CUDA(cudaGetLastError());
  jd_status s = pair ? run_pair_forward(p, p->opt_ut, S_JT, p->opt_ut2, S_JT2) : run_plan_forward(p, p->opt_ut, S_JT);
  if (s) return s;
  pr = prof_begin(KC_OPT, p->stream);
  opt_accept_kernel<<<1, 256, 0, p->stream>>>(n, p->opt_u, p->opt_ut, pair ? p->opt_ut2 : nullptr, armijo_c, dt,
                                              p->scal_d);
  prof_end(pr, p->stream);
  count_launch();
  JD_CUDA(cudaGetLastError());
  JD_CUDA(cudaMemcpyAsync(p->host_pinned, p->scal_d, 8 * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  return JD_OK;
}

// Run one phase's work: captured into a graph on first use and replayed afterwards
// (use_graphs), or enqueued directly.  The phase ends with a record of m.ev.
template <typename F>
static jd_status run_phase(jd::OptMachine &m, cudaGraphExec_t *exec, int *nlaunch, F &&enqueue) {
  jd_problem *p = m.p;
  if (!m.use_graphs) {
    jd_status s = enqueue();
    if (s) return s;
  } else {
    if (!*exec) {
      const uint64_t before = g_launches.load();
      JD_CUDA(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
      const jd_status s = enqueue();
      cudaGraph_t graph = nullptr;
      const cudaError_t e = cudaStreamEndCapture(p->stream, &graph);
      if (s) {
        if (graph) cudaGraphDestroy(graph);
        return s;
      }
      JD_CUDA(e);
      const cudaError_t ei = cudaGraphInstantiate(exec, graph, 0);
      cudaGraphDestroy(graph);
      JD_CUDA(ei);
      *nlaunch = (int)(g_launches.load() - before);   // captured, not launched: count on replay
      g_launches.fetch_sub((uint64_t)*nlaunch);
    }
    JD_CUDA(cudaGraphLaunch(*exec, p->stream));
    count_launch(*nlaunch);
  }
  JD_CUDA(cudaEventRecord(m.ev, p->stream));
  return JD_OK;
}

static jd_status launch_grad(jd::OptMachine &m) {
  const int v = m.forward_done ? 1 : 0;
  jd_problem *p = m.p;
  if (m.o.resample) p->desc.epoch = m.epoch0 + (uint32_t)m.it;   // fresh sample per iteration
  if (m.defer) {   // opt_launch_batch runs the work
    m.want = jd::OptMachine::GRAD;
    m.want_fwd = v == 0;
  } else {
    const jd_status s =
        run_phase(m, &m.g_grad[m.bank][v], &m.n_grad[m.bank][v], [&]() { return enqueue_grad(p, v == 1); });
    if (s) return s;
  }
  m.forward_done = false;
  m.r.evals++;
  if (v == 0) m.r.sweeps++;
  m.grads++;
  m.phase = jd::OptMachine::GRAD;
  return JD_OK;
}

// One Armijo trial at the current zeta, or the pair (zeta, zeta / 2) in one sweep.  A
// pair costs about a third more than one trial and saves a whole sweep when the first
// point is rejected: it is taken for an iteration's first trial (zeta was doubled, so
// a backtrack is the common case) unless the last two iterations accepted their first
// point (a run of growing steps); later trials of the iteration are single (after two
// rejections the next point is the likely one).  Never beyond the backtrack budget.
static jd_status launch_trial(jd::OptMachine &m) {
  jd_problem *p = m.p;
  p->host_pinned[S_ZETA] = m.zeta;   // read by the trial's copy when it executes
  const double c = m.o.armijo_c;
  const bool want = m.backtracks == 0 && m.first_accepts < 2;
  m.pair = m.pairs && want && m.backtracks + 1 <= m.o.max_backtracks && ensure_pair(p);
  const bool pair = m.pair;
  const int v = pair ? 1 : 0;
  if (m.defer) {   // opt_launch_batch runs the work
    m.want = jd::OptMachine::TRIAL;
    m.want_pair = pair;
  } else {
    const jd_status s =
        run_phase(m, &m.g_trial[m.bank][v], &m.n_trial[m.bank][v], [&]() { return enqueue_trial(p, c, pair); });
    if (s) return s;
  }
  m.r.evals++;
  m.r.sweeps++;
  m.phase = jd::OptMachine::TRIAL;
  return JD_OK;
}

void jd::opt_release(OptMachine &m) {
  for (auto &gb : m.g_grad)
    for (auto &g : gb)
      if (g) cudaGraphExecDestroy(g), g = nullptr;
  for (auto &gb : m.g_trial)
    for (auto &g : gb)
      if (g) cudaGraphExecDestroy(g), g = nullptr;
}

// Final iterate to the caller's buffer.
static jd_status launch_output(jd::OptMachine &m, jd_status status) {
  jd_problem *p = m.p;
  p->desc.epoch = m.epoch0;
  m.r.iters = m.it;
  m.r.zeta = m.zeta;
  m.r.status = status;
  const size_t n = (size_t)p->desc.Nt * p->desc.du;
  JD_CUDA(cudaMemcpyAsync(m.u_dst, p->opt_u, n * 8,
                          m.u_space == JD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                          p->stream));
  JD_CUDA(cudaEventRecord(m.ev, p->stream));
  m.phase = jd::OptMachine::OUTPUT;
  return JD_OK;
}

jd_status jd::opt_begin(OptMachine &m, jd_problem *p, const jd_opt_params &o, double *u_dst, jd_memspace us,
                        double *J_hist) {
  if (o.max_iter < 0 || o.max_backtracks < 0 || !(o.armijo_c >= 0.0))
    return fail(JD_ERR_INVALID_ARG, "bad optimizer parameters");
  if (us != JD_MEM_HOST && us != JD_MEM_DEVICE) return fail(JD_ERR_INVALID_ARG, "bad memory space for u");
  m.p = p;
  m.o = o;
  std::memset(&m.r, 0, sizeof(m.r));
  m.J_hist = J_hist;
  m.u_dst = u_dst;
  m.u_space = us;
  m.it = m.backtracks = m.grads = 0;
  m.pairs = o.one_trial_per_sweep == 0;
  m.first_accepts = 0;
  m.pair = false;
  m.bank = 0;
  m.zeta = o.zeta0 > 0.0 ? o.zeta0 : 1.0;
  m.zeta_max = o.zeta_max > 0.0 ? o.zeta_max : 1e3;
  m.pg0 = -1.0;
  m.forward_done = false;
  m.epoch0 = p->desc.epoch;
  if (o.resample) m.use_graphs = false;   // every iteration's launches carry a new epoch
  const size_t n = (size_t)p->desc.Nt * p->desc.du;
  if (m.use_graphs) {
    // graphs hold fixed launches: not for the d = 32 kernels (their coefficient upload
    // is a pageable copy per launch) nor while kernel timing is recorded; the plan's
    // buffers are allocated before the first capture
    bool prof;
    {
      std::lock_guard<std::mutex> g(g_prof_mu);
      prof = g_prof_on;
    }
    if (p->D == 32 || prof) m.use_graphs = false;
    jd_status s = ensure_plan(p);
    if (s) return s;
  }
  JD_CUDA(cudaMemcpyAsync(p->opt_u, p->u_in, n * 8, cudaMemcpyDeviceToDevice, p->stream));
  if (o.max_iter == 0) return launch_output(m, JD_OK);
  return launch_grad(m);
}

jd_status jd::opt_advance(OptMachine &m) {
  jd_problem *p = m.p;
  const double *h = p->host_pinned;
  switch (m.phase) {
    case OptMachine::GRAD: {
      const jd_status st = status_of_scalars(p);
      if (st != JD_OK) return launch_output(m, st);
      const double J = h[S_J], pg = h[S_PG];
      if (m.J_hist) m.J_hist[m.it] = J;
      m.r.J = J;
      if (m.pg0 < 0.0) m.pg0 = pg;
      m.r.rel_grad_norm = m.pg0 > 0.0 ? pg / m.pg0 : 0.0;
      if (m.r.rel_grad_norm <= m.o.tol_rel_grad) return launch_output(m, JD_OK);
      if (m.it > 0) m.zeta = std::fmin(2.0 * m.zeta, m.zeta_max);
      m.backtracks = 0;
      return launch_trial(m);
    }
    case OptMachine::TRIAL: {
      if (m.backtracks == 0) m.first_accepts = h[S_ACC] == 1.0 ? m.first_accepts + 1 : 0;
      if (m.pair && h[S_ACC] != 1.0) {
        // the pair's second trial counts as the evaluation sequential backtracking makes next
        m.r.evals++;
        m.zeta *= 0.5;
        ++m.backtracks;
        if (h[S_ACC] == 2.0) {   // its states become the plan's
          swap_pair(p);
          m.bank ^= 1;   // graphs captured with the other assignment of the two sets
        }
      }
      if (h[S_ACC] != 0.0) {
        m.forward_done = !m.o.resample;   // the trial's sweep is the next gradient's forward
        const double step2 = h[S_STEP];
        m.r.J = h[S_J];
        if (m.J_hist) m.J_hist[m.it + 1] = m.r.J;
        m.it++;
        if (std::sqrt(step2) < m.o.tol_step || m.it >= m.o.max_iter) return launch_output(m, JD_OK);
        return launch_grad(m);
      }
      m.zeta *= 0.5;
      if (++m.backtracks > m.o.max_backtracks)
        return launch_output(m, fail(JD_ERR_LINESEARCH, "Armijo backtracking exhausted"));
      return launch_trial(m);
    }
    case OptMachine::OUTPUT:
      m.phase = OptMachine::DONE;
      return JD_OK;
    default:
      return fail(JD_ERR_INVALID_ARG, "optimizer machine is not running");
  }
}

bool jd::opt_batchable(jd_problem *p) {
  if (ensure_plan(p)) return false;
  return p->ops->fwd_batch && p->ops->adj_batch && p->desc.du == 1 && p->D <= 2 && p->plan == JD_ADJ_STORED &&
         !p->chunk;
}

// Machines with the same key (precision and compiled dimension) share launches whatever
// their phases.
int jd::opt_batch_key(const OptMachine &m) {
  if (m.want == OptMachine::IDLE) return -1;
  return m.p->D + 4 * (m.p->desc.prec == JD_FP64 ? 1 : 0);
}

// The deferred phases of machines with one batch key: the work of enqueue_grad or
// enqueue_trial for each, in shared launches -- one optimizer block per problem before
// and after, one forward sweep over the blocks of the problems whose phase has a single
// forward (a trial, or a gradient without a kept forward), one over those with a paired
// trial, one adjoint sweep over the gradient phases' problems (after their forward, in
// stream order), one launch for all unit sums and one for all combines -- then each
// machine's scalars to its pinned buffer and its event.
jd_status jd::opt_launch_batch(OptMachine *const *ms, int n, cudaStream_t st) {
  if (n < 1 || n > kBatchMax) return fail(JD_ERR_INVALID_ARG, "batch size");
  const int key = opt_batch_key(*ms[0]);
  const PathOps *ops = ms[0]->p->ops;
  for (int i = 0; i < n; ++i) {
    OptMachine &m = *ms[i];
    jd_problem *p = m.p;
    if (opt_batch_key(m) != key || p->ops != ops) return fail(JD_ERR_INVALID_ARG, "mixed batch");
    jd_status s = ensure_plan(p);
    if (s) return s;
    if (!opt_batchable(p)) return fail(JD_ERR_UNSUPPORTED, "problem cannot run batched");
    // the batch follows everything queued on the problem's own stream (allocations,
    // copies of the control)
    JD_CUDA(cudaEventRecord(m.ev, p->stream));
    JD_CUDA(cudaStreamWaitEvent(st, m.ev, 0));
  }
  const bool f64 = ops->elem == 8;
  OptBatch ob;
  ob.n = n;
  BatchSweep fs[kBatchMax], fp[kBatchMax], ad[kBatchMax];   // single forward, paired forward, adjoint
  int nfs = 0, nfp = 0, nad = 0;
  UnitBatch ub;
  CombineBatch cb;
  ub.n = cb.n = 0;
  int ubl = 0, cbl = 0;
  auto add_unit = [&](jd_problem *p, const double *partC, int ne, double *units) {
    const jd_problem_desc &q = p->desc;
    const int64_t nun = n_units(q.M);
    ub.first[ub.n] = ubl;
    ub.j[ub.n++] = UnitJob{partC, p->partG, p->nblk, grad_parts(q.M), nun, q.du, p->DU, ne, units};
    ubl += (int)ceil_div(nun * ne * 32, 256);
  };
  auto add_combine = [&](jd_problem *p, const double *units, int ne, const double *u, int slot) {
    const jd_problem_desc &q = p->desc;
    const double dt = q.T / q.Nt;
    cb.first[cb.n] = cbl;
    cb.j[cb.n++] = CombineJob{units, u, n_units(q.M), ne, q.Nt * q.du, q.nu * dt, 0.5 * q.nu * dt,
                              1.0 / (double)q.M, p->scal_d + slot, p->grad_d, p->scal_d + S_BAD};
    cbl += (int)ceil_div(ne, 128);
  };
  for (int i = 0; i < n; ++i) {
    OptMachine &m = *ms[i];
    jd_problem *p = m.p;
    const jd_problem_desc &q = p->desc;
    const OptMachine::Phase kind = m.want;
    const bool fwd = m.want_fwd, pair = m.want_pair;
    OptBatchItem &b = ob.it[i];
    b.trial = kind == OptMachine::TRIAL;
    b.n = q.Nt * q.du;
    b.Nt = q.Nt;
    b.du = q.du;
    b.DU = p->DU;
    b.fwd = kind == OptMachine::GRAD && fwd;
    b.dt = q.T / q.Nt;
    b.lo = q.u_min;
    b.hi = q.u_max;
    b.c = m.o.armijo_c;
    b.zeta = m.zeta;
    b.u = p->opt_u;
    b.grad = p->grad_d;
    b.ut = p->opt_ut;
    b.ut2 = kind == OptMachine::TRIAL && pair ? p->opt_ut2 : nullptr;
    b.scal = p->scal_d;
    b.uk = p->uk;
    b.uk2 = p->uk2;
    const BatchSweep sw{p, p->uk, plan_bufs(p)};
    if (kind == OptMachine::TRIAL && pair) {
      BatchSweep &x = fp[nfp++];
      x = sw;
      x.b.uk2 = p->uk2;
      x.b.traj2 = p->traj2;
      x.b.log_kt2 = p->log_kt2;
      x.b.log_y2 = p->log_y2;
      x.b.partC2 = p->partC2;
    } else if (kind == OptMachine::TRIAL || fwd) {
      fs[nfs++] = sw;
    }
    if (kind == OptMachine::GRAD) ad[nad++] = sw;
    const int64_t nun = n_units(q.M);
    if (kind == OptMachine::GRAD) {
      const int ne = 1 + q.Nt * q.du;
      add_unit(p, p->partC, ne, p->units);
      add_combine(p, p->units, ne, p->opt_u, S_J);
    } else {   // the second point's cost units after the first's (the cost needs nun of them)
      add_unit(p, p->partC, 1, p->units);
      add_combine(p, p->units, 1, p->opt_ut, S_JT);
      if (pair) {
        add_unit(p, p->partC2, 1, p->units + nun);
        add_combine(p, p->units + nun, 1, p->opt_ut2, S_JT2);
      }
    }
  }
  ub.first[ub.n] = ubl;
  cb.first[cb.n] = cbl;
  if (f64)
    opt_pre_batch_kernel<double><<<n, 256, 0, st>>>(ob);
  else
    opt_pre_batch_kernel<float><<<n, 256, 0, st>>>(ob);
  count_launch();
  JD_CUDA(cudaGetLastError());
  cudaError_t e = cudaSuccess;
  if (nfs) e = ops->fwd_batch(fs, nfs, FWD_STORE, st);
  if (e == cudaSuccess && nfp) e = ops->fwd_batch(fp, nfp, FWD_STORE | FWD_PAIR, st);
  if (e == cudaSuccess && nad) e = ops->adj_batch(ad, nad, st);
  JD_CUDA(e);
  unit_sums_batch_kernel<<<ubl, 256, 0, st>>>(ub);
  combine_units_batch_kernel<<<cbl, 128, 0, st>>>(cb);
  opt_post_batch_kernel<<<n, 256, 0, st>>>(ob);
  count_launch(3);
  JD_CUDA(cudaGetLastError());
  for (int i = 0; i < n; ++i) {
    OptMachine &m = *ms[i];
    JD_CUDA(cudaMemcpyAsync(m.p->host_pinned, m.p->scal_d, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
    JD_CUDA(cudaEventRecord(m.ev, st));
    m.want = OptMachine::IDLE;
  }
  return JD_OK;
}

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *jd_status_string(jd_status s) {
  switch (s) {
    case JD_OK: return "ok";
    case JD_ERR_INVALID_ARG: return "invalid argument";
    case JD_ERR_OOM: return "out of device memory or over the memory budget";
    case JD_ERR_CUDA: return "CUDA runtime error";
    case JD_ERR_NONFINITE: return "non-finite cost or gradient";
    case JD_ERR_LINESEARCH: return "Armijo line search exhausted its backtracks";
    case JD_ERR_TIMEOUT: return "bounded device wait timed out";
    case JD_ERR_UNSUPPORTED: return "unsupported by this build";
    case JD_ERR_BUSY: return "result not ready";
  }
  return "unknown status";
}

const char *jd_last_error(void) { return g_last_error.c_str(); }

uint64_t jd_kernel_launch_count(void) { return g_launches.load(); }

void jd_profile_enable(int on) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  for (auto &r : g_prof_recs) {
    cudaEventSynchronize(r.b);
    g_prof_pool.push_back(r.a);
    g_prof_pool.push_back(r.b);
  }
  g_prof_recs.clear();
  g_prof_on = on != 0;
}

int jd_profile_read(jd_kernel_stat *out, int max_entries) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  double ms[KC_COUNT] = {0};
  uint64_t n[KC_COUNT] = {0};
  for (auto &r : g_prof_recs) {
    float t = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      ms[r.kind] += t;
      n[r.kind] += 1;
    }
  }
  int k = 0;
  for (int c = 0; c < KC_COUNT && k < max_entries; ++c) {
    if (!n[c]) continue;
    out[k].name = kKernelClassName[c];
    out[k].launches = n[c];
    out[k].total_ms = ms[c];
    ++k;
  }
  return k;
}

jd_status jd_problem_destroy(jd_problem *p) {
  if (!p) return JD_OK;
  cudaSetDevice(p->device);
  if (p->stream) cudaStreamSynchronize(p->stream);
  free_dev(p, p->uk);
  free_dev(p, p->xdk);
  free_dev(p, p->u_in);
  free_dev(p, p->grad_d);
  free_dev(p, p->scal_d);
  free_dev(p, p->partC);
  free_dev(p, p->partG);
  free_dev(p, p->units);
  free_dev(p, p->pre_w);
  free_dev(p, p->pre_z);
  free_dev(p, p->pre_key);
  free_dev(p, p->partT);
  free_dev(p, p->traj);
  free_dev(p, p->flags);
  free_dev(p, p->ckpt);
  free_dev(p, p->log_kt);
  free_dev(p, p->log_y);
  free_dev(p, p->jcnt);
  free_dev(p, p->opt_u);
  free_dev(p, p->opt_ut);
  free_dev(p, p->opt_g);
  free_dev(p, p->uk2);
  free_dev(p, p->partC2);
  free_dev(p, p->opt_ut2);
  free_dev(p, p->traj2);
  free_dev(p, p->log_kt2);
  free_dev(p, p->log_y2);
  free_dev(p, p->ckpt2);
  free_dev(p, p->kp_dev);
  free_dev(p, p->bu_dev);
  free_dev(p, p->fb_mu);
  free_dev(p, p->fb_traj);
  free_dev(p, p->fb_z0);
  free_dev(p, p->fb_flags);
  free_dev(p, p->fb_mu64);
  free_dev(p, p->fb_grad);
  free_dev(p, p->fb_partC);
  free_dev(p, p->fb_partG);
  free_dev(p, p->fb_partW);
  free_dev(p, p->fb_mut);
  if (p->host_pinned && p->own_pinned) cudaFreeHost(p->host_pinned);
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
  delete p;
  return JD_OK;
}

jd_status jd_problem_create(const jd_problem_desc *desc, jd_problem **out) {
  if (!desc || !out) return fail(JD_ERR_INVALID_ARG, "desc and out must be non-NULL");
  return jd::create_problem(*desc, jd::ProblemOpts{}, out);
}

jd_status jd_problem_footprint(const jd_problem_desc *desc, jd_adjoint_mode plan, size_t *bytes) {
  if (!desc || !bytes) return fail(JD_ERR_INVALID_ARG, "desc and bytes must be non-NULL");
  jd_status s = validate_desc(*desc);
  if (s) return s;
  if (plan != JD_ADJ_STORED && plan != JD_ADJ_RECOMPUTE)
    return fail(JD_ERR_INVALID_ARG, "plan must be JD_ADJ_STORED or JD_ADJ_RECOMPUTE");
  if (plan == JD_ADJ_RECOMPUTE && desc->d > 8)
    return fail(JD_ERR_UNSUPPORTED, "the recompute adjoint is not built for 8 < d <= 32");
  *bytes = jd::problem_bytes(*desc, plan);
  return JD_OK;
}

}  // extern "C"

jd_status jd::create_problem(const jd_problem_desc &q, const jd::ProblemOpts &opts, jd_problem **out) {
  *out = nullptr;
  jd_status vs = validate_desc(q);
  if (vs) return vs;
  const size_t dd = (size_t)q.d * q.d, dn = (size_t)(q.Nt + 1) * q.d;

  jd_problem *p = new jd_problem();
  p->desc = q;
  p->A.assign(q.A, q.A + dd);
  if (q.drift == JD_DRIFT_CUBIC) p->C.assign(q.C, q.C + dd);
  p->B.assign(q.B, q.B + (size_t)q.d * q.du);
  if (q.dA) p->dA.assign(q.dA, q.dA + dd);
  p->sigma.assign(q.sigma, q.sigma + q.d);
  p->x0.assign(q.x0, q.x0 + q.d);
  p->q.assign(q.q, q.q + q.d);
  p->xd.assign(q.xd, q.xd + dn);
  p->desc.A = p->desc.C = p->desc.B = p->desc.dA = p->desc.sigma = p->desc.x0 = p->desc.q = p->desc.xd = nullptr;
  pick_dims(q.d, q.du, &p->D, &p->DU);
  p->ops = path_ops_dims(q.prec, p->D, p->DU);
  if (!p->ops) {
    delete p;
    return fail(JD_ERR_UNSUPPORTED, "no kernels compiled for this (d, du)");
  }
  p->nblk = ceil_div(q.M, TPB);

  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "cudaGetDevice");
  }
  {
    // the jump path keeps sub-step states on the per-thread stack: make sure this
    // context's stack limit covers the largest kernel of this instantiation
    const size_t need = p->ops->stack_bytes();
    size_t cur = 0;
    e = cudaDeviceGetLimit(&cur, cudaLimitStackSize);
    if (e == cudaSuccess && cur < need) e = cudaDeviceSetLimit(cudaLimitStackSize, need);
    if (e != cudaSuccess) {
      delete p;
      return cuda_fail(e, "cudaDeviceSetLimit(cudaLimitStackSize)");
    }
  }
  p->async_alloc = opts.async_alloc;
  if (opts.stream) {
    p->stream = opts.stream;
  } else if (q.cuda_stream) {
    p->stream = (cudaStream_t)q.cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete p;
      return cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    p->own_stream = true;
  }
  if (q.mem_budget_bytes) {
    p->budget = q.mem_budget_bytes;
  } else {
    size_t fr = 0, tot = 0;
    e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) {
      jd_problem_destroy(p);
      return cuda_fail(e, "cudaMemGetInfo");
    }
    p->budget = fr / 2;
  }
  const size_t es = elem_size(p), nu = (size_t)q.Nt * q.du;
  jd_status s = JD_OK;
#define ALLOC(ptr, bytes, name)                                  \
  do {                                                           \
    s = dev_alloc(p, (void **)&(ptr), (bytes), name);            \
    if (s) {                                                     \
      jd_problem_destroy(p);                                     \
      return s;                                                  \
    }                                                            \
  } while (0)
  ALLOC(p->uk, (size_t)q.Nt * p->DU * es, "control");
  ALLOC(p->xdk, (size_t)(q.Nt + 1) * p->D * es, "target");
  ALLOC(p->u_in, nu * 8, "control (FP64)");
  ALLOC(p->grad_d, nu * 8, "gradient");
  ALLOC(p->scal_d, NSCAL * 8, "scalars");
  ALLOC(p->partC, (size_t)p->nblk * 8, "cost partials");
  ALLOC(p->partG, (size_t)q.Nt * p->DU * grad_parts(q.M) * 8, "gradient partials");
  ALLOC(p->partT, (size_t)(p->D + 2) * p->nblk * 8, "parameter partials");
  ALLOC(p->units, (size_t)n_units(q.M) * (1 + nu) * 8, "unit sums");
  if (!opts.no_pre && pre_pass(q.d, q.Nt, q.M, es)) {   // a small problem: the draws' pre-pass buffers
    ALLOC(p->pre_w, (size_t)q.Nt * q.M * 4, "pre-drawn Poisson words");
    ALLOC(p->pre_z, pre_z_values(q.Nt, p->D, q.M) * es, "pre-drawn normals and slot draws");
    ALLOC(p->pre_key, sizeof(unsigned long long), "pre-drawn key");
    if (cudaMemsetAsync(p->pre_key, 0, sizeof(unsigned long long), p->stream) != cudaSuccess) {
      jd_problem_destroy(p);
      return cuda_fail(cudaGetLastError(), "clearing the pre-drawn key");
    }
  }
  ALLOC(p->opt_u, nu * 8, "optimizer iterate");
  ALLOC(p->opt_ut, nu * 8, "optimizer trial");
  if (p->D == 32) {
    ALLOC(p->kp_dev, 16384, "d = 32 coefficients");
    ALLOC(p->bu_dev, (size_t)q.Nt * 32 * sizeof(float), "d = 32 control drift");
  }
#undef ALLOC
  if (opts.pinned) {
    p->host_pinned = opts.pinned;
    p->own_pinned = false;
  } else {
    e = cudaMallocHost((void **)&p->host_pinned, NSCAL * 8);
    if (e != cudaSuccess) {
      jd_problem_destroy(p);
      return cuda_fail(e, "cudaMallocHost");
    }
  }
  e = upload_target(p);
  if (e != cudaSuccess) {
    jd_problem_destroy(p);
    return cuda_fail(e, "cudaMemcpy target");
  }
  e = cudaMemsetAsync(p->scal_d, 0, NSCAL * 8, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) {
    jd_problem_destroy(p);
    return cuda_fail(e, "cudaMemset");
  }
  *out = p;
  return JD_OK;
}

size_t jd::problem_bytes_min(const jd_problem_desc &q) {
  int D = 0, DU = 0;
  pick_dims(q.d, q.du, &D, &DU);
  const size_t es = q.prec == JD_FP64 ? 8 : 4;
  if (D != 32) return problem_bytes(q, JD_ADJ_RECOMPUTE);
  return base_bytes(q, D, DU, es) + stored_plan_bytes(q, D, es, TPB);
}

size_t jd::pair_bytes(const jd_problem_desc &q, jd_adjoint_mode plan) {
  int D = 0, DU = 0;
  pick_dims(q.d, q.du, &D, &DU);
  if (!pairs_built(D)) return 0;
  const size_t es = q.prec == JD_FP64 ? 8 : 4, M = (size_t)q.M;
  const int cap = log_capacity(q);
  const size_t capa = (size_t)(cap > 0 ? cap : 1);
  size_t b = (size_t)q.Nt * DU * es + (size_t)ceil_div(q.M, TPB) * 8 + (size_t)q.Nt * q.du * 8;
  if (plan == JD_ADJ_STORED) {
    b += traj_values(q.Nt, D, (int)es, (int64_t)M) * es + capa * M * 2 * es + capa * M * D * es;
  } else {
    const jd::PathOps *ops = path_ops_dims(q.prec, D, DU);
    b += ckpt_bytes(q, D, es, ops ? ops->S : 16);
  }
  return b;
}

size_t jd::problem_bytes(const jd_problem_desc &q, jd_adjoint_mode plan) {
  int D = 0, DU = 0;
  pick_dims(q.d, q.du, &D, &DU);
  const size_t es = q.prec == JD_FP64 ? 8 : 4;
  size_t b = base_bytes(q, D, DU, es);
  if (plan == JD_ADJ_STORED) {
    b += stored_plan_bytes(q, D, es, q.M);
  } else if (plan == JD_ADJ_RECOMPUTE) {
    const jd::PathOps *ops = path_ops_dims(q.prec, D, DU);
    b += ckpt_bytes(q, D, es, ops ? ops->S : 16);
  }
  return b;
}

extern "C" {

jd_status jd_problem_info(const jd_problem *p, size_t *device_bytes, jd_adjoint_mode *mode) {
  if (!p) return fail(JD_ERR_INVALID_ARG, "p is NULL");
  if (device_bytes) *device_bytes = p->bytes;
  if (mode) *mode = p->plan;
  return JD_OK;
}

jd_status jd_cost(jd_problem *p, const double *u, jd_memspace us, double *J) {
  if (!p || !J) return fail(JD_ERR_INVALID_ARG, "p and J must be non-NULL");
  p->fwd_valid = false;
  jd_status s = set_device(p);
  if (!s) s = load_u(p, u, us);
  if (!s) s = clear_bad(p);
  if (!s) s = run_cost(p, p->u_in, S_J);
  if (!s) s = read_scalars(p, S_J, 1);
  if (s) return s;
  *J = p->host_pinned[S_J];
  return check_bad(p);
}

jd_status jd_gradient(jd_problem *p, const double *u, jd_memspace us, double *J, double *grad,
                      jd_memspace gs, double *grad_theta) {
  if (!p) return fail(JD_ERR_INVALID_ARG, "p is NULL");
  if (grad && gs != JD_MEM_HOST && gs != JD_MEM_DEVICE) return fail(JD_ERR_INVALID_ARG, "bad memory space for grad");
  if (grad_theta && p->D == 32)
    return fail(JD_ERR_UNSUPPORTED, "parameter gradients are not built for 8 < d <= 32");
  p->fwd_valid = false;
  jd_status s = set_device(p);
  if (!s) s = load_u(p, u, us);
  if (!s) s = clear_bad(p);
  if (!s) s = run_gradient(p, p->u_in, grad_theta != nullptr);
  if (s) return s;
  p->fwd_valid = true;   // the plan's states belong to u_in: jd_backward may follow
  const size_t n = (size_t)p->desc.Nt * p->desc.du;
  if (grad) {
    JD_CUDA(cudaMemcpyAsync(grad, p->grad_d, n * 8,
                            gs == JD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, p->stream));
  }
  const bool host_out = J || grad_theta || (grad && gs == JD_MEM_HOST);
  if (!host_out) return JD_OK;
  s = read_scalars(p, 0, NSCAL);
  if (s) return s;
  if (J) *J = p->host_pinned[S_J];
  if (grad_theta)
    for (int t = 0; t < p->desc.d + 2; ++t) grad_theta[t] = p->host_pinned[S_THETA + t];
  return status_of_scalars(p);
}

// The unit sums of a problem (or of one shard of a problem) at u: the sweeps of
// jd_gradient (grad = true) or jd_cost, then the copy of p->units to `units`.
static jd_status units_out(jd_problem *p, const double *u, jd_memspace us, double *units, jd_memspace os,
                           bool grad) {
  if (!p || !units) return fail(JD_ERR_INVALID_ARG, "p and units must be non-NULL");
  if (os != JD_MEM_HOST && os != JD_MEM_DEVICE) return fail(JD_ERR_INVALID_ARG, "bad memory space for units");
  if (p->desc.m_offset % JD_UNIT_PATHS)
    return fail(JD_ERR_INVALID_ARG, "a shard's m_offset must be a multiple of JD_UNIT_PATHS");
  p->fwd_valid = false;
  jd_status s = set_device(p);
  if (!s) s = load_u(p, u, us);
  if (!s) s = clear_bad(p);
  if (!s) s = grad ? run_gradient(p, p->u_in, false, false, /*finalize=*/false) : run_cost(p, p->u_in, S_J, false);
  if (s) return s;
  if (grad) p->fwd_valid = true;
  const int ne = grad ? 1 + p->desc.Nt * p->desc.du : 1;
  const size_t n = (size_t)n_units(p->desc.M) * ne;
  JD_CUDA(cudaMemcpyAsync(units, p->units, n * 8, os == JD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                          p->stream));
  if (os == JD_MEM_DEVICE) return JD_OK;
  JD_CUDA(cudaStreamSynchronize(p->stream));
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(units[i])) return fail(JD_ERR_NONFINITE, "non-finite unit sum");
  return JD_OK;
}

jd_status jd_gradient_units(jd_problem *p, const double *u, jd_memspace us, double *units, jd_memspace os) {
  return units_out(p, u, us, units, os, true);
}

jd_status jd_cost_units(jd_problem *p, const double *u, jd_memspace us, double *units, jd_memspace os) {
  return units_out(p, u, us, units, os, false);
}

// The device combine (combine_units_kernel) operation for operation, on the host.
jd_status jd_combine_units(int64_t M_total, int Nt, int du, double T, double nu, const double *u,
                           const double *units, int64_t nunits, int ne, double *J, double *grad) {
  if (M_total < 1 || Nt < 1 || du < 1 || !(T > 0.0) || !std::isfinite(T) || !std::isfinite(nu) || !u || !units ||
      !J || nunits != ceil_div(M_total, JD_UNIT_PATHS) || (ne != 1 && ne != 1 + Nt * du) || (ne > 1 && !grad))
    return fail(JD_ERR_INVALID_ARG, "jd_combine_units: bad sizes or NULL arrays");
  const double dt = T / Nt, nu_dt = nu * dt, half_nu_dt = 0.5 * nu * dt, invM = 1.0 / (double)M_total;
  bool finite = true;
  for (int e = 0; e < ne; ++e) {
    double s = 0.0;
    for (int64_t i = 0; i < nunits; ++i) s = s + units[i * ne + e];
    double v;
    if (e == 0) {
      // chunks of 32 squares, each by the xor butterfly of combine_units_kernel
      const int n = Nt * du;
      double b = 0.0;
      for (int c0 = 0; c0 < n; c0 += 32) {
        double w[32];
        for (int l = 0; l < 32; ++l) {
          const double x = c0 + l < n ? u[c0 + l] : 0.0;
          w[l] = x * x;
        }
        for (int o = 16; o >= 1; o >>= 1) {
          double t[32];
          for (int l = 0; l < 32; ++l) t[l] = w[l] + w[l ^ o];
          for (int l = 0; l < 32; ++l) w[l] = t[l];
        }
        b = b + w[0];
      }
      const double sm = s * invM;
      v = std::fma(half_nu_dt, b, sm);
      *J = v;
    } else {
      const double sm = s * invM;
      v = std::fma(nu_dt, u[e - 1], sm);
      grad[e - 1] = v;
    }
    finite = finite && std::isfinite(v);
  }
  return finite ? JD_OK : fail(JD_ERR_NONFINITE, "non-finite J or gradient");
}

jd_status jd_forward(jd_problem *p, const double *u, jd_memspace us, double *J, jd_memspace js) {
  if (!p) return fail(JD_ERR_INVALID_ARG, "p is NULL");
  if (J && js != JD_MEM_HOST && js != JD_MEM_DEVICE) return fail(JD_ERR_INVALID_ARG, "bad memory space for J");
  p->fwd_valid = false;
  jd_status s = set_device(p);
  if (!s) s = load_u(p, u, us);
  if (!s) s = clear_bad(p);
  if (!s) s = run_plan_forward(p, p->u_in, S_J);
  if (s) return s;
  p->fwd_valid = true;
  if (!J) return JD_OK;
  if (js == JD_MEM_DEVICE) {
    JD_CUDA(cudaMemcpyAsync(J, p->scal_d + S_J, sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
    return JD_OK;
  }
  s = read_scalars(p, 0, NSCAL);
  if (s) return s;
  *J = p->host_pinned[S_J];
  return status_of_scalars(p);
}

jd_status jd_backward(jd_problem *p, double *grad, jd_memspace gs, double *grad_theta) {
  if (!p) return fail(JD_ERR_INVALID_ARG, "p is NULL");
  if (gs != JD_MEM_HOST && gs != JD_MEM_DEVICE) return fail(JD_ERR_INVALID_ARG, "bad memory space for grad");
  if (!p->fwd_valid)
    return fail(JD_ERR_INVALID_ARG, "jd_backward needs a jd_forward (or jd_gradient) on this problem first");
  if (grad_theta && p->D == 32)
    return fail(JD_ERR_UNSUPPORTED, "parameter gradients are not built for 8 < d <= 32");
  jd_status s = set_device(p);
  if (!s) s = run_gradient(p, p->u_in, grad_theta != nullptr, /*forward_done=*/true);
  if (s) return s;
  const size_t n = (size_t)p->desc.Nt * p->desc.du;
  const cudaMemcpyKind kind = gs == JD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (grad) JD_CUDA(cudaMemcpyAsync(grad, p->grad_d, n * 8, kind, p->stream));
  if (gs == JD_MEM_DEVICE) {
    if (grad_theta)
      JD_CUDA(cudaMemcpyAsync(grad_theta, p->scal_d + S_THETA, (size_t)(p->desc.d + 2) * 8,
                              cudaMemcpyDeviceToDevice, p->stream));
    return JD_OK;
  }
  s = read_scalars(p, 0, NSCAL);
  if (s) return s;
  if (grad_theta)
    for (int t = 0; t < p->desc.d + 2; ++t) grad_theta[t] = p->host_pinned[S_THETA + t];
  return status_of_scalars(p);
}

jd_status jd_problem_update(jd_problem *p, const jd_problem_desc *desc) {
  if (!p || !desc) return fail(JD_ERR_INVALID_ARG, "p and desc must be non-NULL");
  const jd_problem_desc &q = *desc, &o = p->desc;
  jd_status s = validate_desc(q);
  if (s) return s;
  if (q.d != o.d || q.du != o.du || q.T != o.T || q.Nt != o.Nt || q.M != o.M || q.drift != o.drift ||
      q.prec != o.prec || q.mode != o.mode || q.use_tensor_cores != o.use_tensor_cores)
    return fail(JD_ERR_INVALID_ARG,
                "jd_problem_update may change coefficients only (d, du, T, Nt, M, drift, prec, mode, "
                "use_tensor_cores must match)");
  s = set_device(p);
  if (s) return s;
  p->fwd_valid = false;
  const size_t dd = (size_t)q.d * q.d, dn = (size_t)(q.Nt + 1) * q.d;
  p->A.assign(q.A, q.A + dd);
  if (q.drift == JD_DRIFT_CUBIC) p->C.assign(q.C, q.C + dd);
  p->B.assign(q.B, q.B + (size_t)q.d * q.du);
  if (q.dA)
    p->dA.assign(q.dA, q.dA + dd);
  else
    p->dA.clear();
  p->sigma.assign(q.sigma, q.sigma + q.d);
  p->x0.assign(q.x0, q.x0 + q.d);
  p->q.assign(q.q, q.q + q.d);
  const bool new_target = !std::equal(q.xd, q.xd + dn, p->xd.begin());
  if (new_target) p->xd.assign(q.xd, q.xd + dn);
  p->desc.lambda = q.lambda;
  p->desc.jump_law = q.jump_law;
  p->desc.jump_scale = q.jump_scale;
  p->desc.jump_gain = q.jump_gain;
  p->desc.nu = q.nu;
  p->desc.u_min = q.u_min;
  p->desc.u_max = q.u_max;
  p->desc.seed = q.seed;
  p->desc.epoch = q.epoch;
  if (new_target) {
    const cudaError_t e = upload_target(p);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy target");
  }
  return JD_OK;
}

jd_status jd_sample_paths(jd_problem *p, const double *u, jd_memspace us, int64_t m0, int64_t count,
                          double *X, double *lam, double *cost) {
  if (!p) return fail(JD_ERR_INVALID_ARG, "p is NULL");
  if (m0 < 0 || count < 1 || m0 + count > p->desc.M)
    return fail(JD_ERR_INVALID_ARG, "path range outside [0, M)");
  p->fwd_valid = false;
  jd_status s = set_device(p);
  if (!s) s = load_u(p, u, us);
  if (!s) s = prep_u(p, p->u_in);
  if (s) return s;
  const jd_problem_desc &q = p->desc;
  const int D = p->D, Nt = q.Nt, d = q.d;
  const size_t es = elem_size(p);
  const int64_t nb = ceil_div(count, TPB);
  const size_t traj_b = traj_values(Nt, D, (int)es, count) * es, flag_b = (size_t)ceil_div(Nt, 32) * count * 4;
  const size_t lam_b = (size_t)(Nt + 1) * D * count * es;
  const int cap = log_capacity(q);
  const size_t capa = (size_t)(cap > 0 ? cap : 1);
  void *traj = nullptr, *flags = nullptr, *lamd = nullptr, *pc = nullptr, *pC = nullptr, *pG = nullptr;
  void *lkt = nullptr, *ly = nullptr, *jc = nullptr;
  cudaError_t e = cudaMalloc(&traj, traj_b);
  if (e == cudaSuccess) e = cudaMalloc(&flags, flag_b);
  if (e == cudaSuccess) e = cudaMalloc(&lamd, lam_b);
  if (e == cudaSuccess) e = cudaMalloc(&pc, count * es);
  if (e == cudaSuccess) e = cudaMalloc(&pC, nb * 8);
  if (e == cudaSuccess) e = cudaMalloc(&pG, (size_t)Nt * p->DU * grad_parts(count) * 8);
  if (e == cudaSuccess) e = cudaMalloc(&lkt, capa * count * 2 * es);
  if (e == cudaSuccess) e = cudaMalloc(&ly, capa * count * D * es);
  if (e == cudaSuccess) e = cudaMalloc(&jc, (size_t)count * 8);
  PathBufs b;
  b.traj = traj;
  b.flags = (uint32_t *)flags;
  b.pcost = pc;
  b.log_kt = lkt;
  b.log_y = ly;
  b.jcnt = (int *)jc;
  b.log_cap = cap;
  b.partC = (double *)pC;
  b.partG = (double *)pG;
  b.lam_out = lamd;
  b.status = reinterpret_cast<int *>(p->scal_d + S_STATUS);
  if (e == cudaSuccess) e = p->ops->fwd(p, FWD_STORE, m0, count, p->uk, b, p->stream);
  if (e == cudaSuccess && lam) e = p->ops->adj(p, ADJ_STORED_V, false, m0, count, p->uk, b, p->stream);
  std::vector<unsigned char> ht, hl, hc;
  if (e == cudaSuccess) {
    ht.resize(traj_b);
    hc.resize(count * es);
    e = cudaMemcpyAsync(ht.data(), traj, traj_b, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), pc, count * es, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess && lam) {
      hl.resize(lam_b);
      e = cudaMemcpyAsync(hl.data(), lamd, lam_b, cudaMemcpyDeviceToHost, p->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  }
  cudaFree(traj);
  cudaFree(flags);
  cudaFree(lamd);
  cudaFree(pc);
  cudaFree(pC);
  cudaFree(pG);
  cudaFree(lkt);
  cudaFree(ly);
  cudaFree(jc);
  if (e != cudaSuccess) return cuda_fail(e, "jd_sample_paths");
  auto rd = [&](const std::vector<unsigned char> &v, size_t idx) -> double {
    if (es == 8) return reinterpret_cast<const double *>(v.data())[idx];
    return (double)reinterpret_cast<const float *>(v.data())[idx];
  };
  for (int64_t i = 0; i < count; ++i) {
    if (cost) cost[i] = rd(hc, i);
    for (int k = 0; k <= Nt; ++k)
      for (int c = 0; c < d; ++c) {
        const size_t base = (size_t)(i * (Nt + 1) + k) * d + c;
        if (X) {
          X[base] = rd(ht, traj_index(k, c, i, count, D, (int)es));
        }
        if (lam) lam[base] = rd(hl, ((size_t)k * D + c) * count + i);
      }
  }
  return JD_OK;
}

// ---------------------------------------------------------------------------
// Feedback control (jd_fb_cost, jd_fb_gradient)
// ---------------------------------------------------------------------------
static jd_status fb_validate(const jd_problem *p, const jd_feedback_desc *fb) {
  if (!p || !fb) return fail(JD_ERR_INVALID_ARG, "p and fb must be non-NULL");
  if (p->desc.d != 2 || p->desc.du != 1)
    return fail(JD_ERR_UNSUPPORTED, "feedback control is built for d = 2 (x, v) and du = 1");
  if (fb->nx < 1 || fb->nx > FB_NB || fb->nv < 1 || fb->nv > FB_NB)
    return fail(JD_ERR_INVALID_ARG, "nx and nv must be in [1, 16]");
  if (!(fb->x_max > 0.0) || !std::isfinite(fb->x_max) || !(fb->v_max > 0.0) || !std::isfinite(fb->v_max) ||
      !(fb->eps > 0.0) || !std::isfinite(fb->eps))
    return fail(JD_ERR_INVALID_ARG, "x_max, v_max and eps must be finite and > 0");
  if (fb->track != JD_TRACK_QUADRATIC && fb->track != JD_TRACK_GAUSS && fb->track != JD_TRACK_ELLIPSE)
    return fail(JD_ERR_INVALID_ARG, "bad tracking term");
  if (fb->track != JD_TRACK_QUADRATIC && (!(fb->sigma_J > 0.0) || !std::isfinite(fb->sigma_J)))
    return fail(JD_ERR_INVALID_ARG, "sigma_J must be finite and > 0");
  if ((fb->track == JD_TRACK_ELLIPSE || fb->particles) &&
      (!(fb->ax > 0.0) || !std::isfinite(fb->ax) || !(fb->av > 0.0) || !std::isfinite(fb->av)))
    return fail(JD_ERR_INVALID_ARG, "ax and av must be finite and > 0");
  if (fb->particles != 0 && (fb->particles < 3 || fb->particles > RING_MAX))
    return fail(JD_ERR_INVALID_ARG, "particles must be 0 or in [3, 2048]");
  if (fb->particles) {
    // rings are whole: M a multiple of the ring's lanes S, and of the block for rings
    // beyond one warp (their exchange has block or cluster barriers)
    const int64_t S = ring_lanes(fb->particles), unit = fb->particles <= 32 ? S : std::max<int64_t>(S, FB_TPB);
    if (p->desc.M % unit != 0 || !std::isfinite(fb->omega))
      return fail(JD_ERR_INVALID_ARG,
                  "interacting particles need a finite omega and M a multiple of the ring's lanes (32 for up to 32 "
                  "particles, else the next power of two and at least 256 up to 256 particles, then the next "
                  "multiple of 256)");
  }
  if (fb->particles && fb->adjoint != JD_FB_EXACT)
    return fail(JD_ERR_UNSUPPORTED, "interacting particles take the exact adjoint only");
  if (fb->adjoint != JD_FB_EXACT && fb->adjoint != JD_FB_SURROGATE)
    return fail(JD_ERR_INVALID_ARG, "bad feedback adjoint");
  if (fb->adjoint == JD_FB_SURROGATE && (!(fb->sur_rate >= 0.0) || !std::isfinite(fb->sur_rate)))
    return fail(JD_ERR_INVALID_ARG, "sur_rate must be finite and >= 0");
  return JD_OK;
}

// Initial states of a ring's particles, equidistant on the ellipse (Sec. 6.4): particle
// i at (ax cos(2 pi i / N), av sin(2 pi i / N)), in kernel precision, [2][S] (idle lanes 0).
static jd_status fb_upload_ring(jd_problem *p, const jd_feedback_desc &fb) {
  const int N = fb.particles, S = ring_lanes(N);
  std::vector<double> z(2 * (size_t)S, 0.0);
  for (int i = 0; i < N; ++i) {
    const double th = 2.0 * 3.14159265358979323846 * i / N;
    z[i] = fb.ax * std::cos(th);
    z[S + i] = fb.av * std::sin(th);
  }
  if (elem_size(p) == 8) {
    JD_CUDA(cudaMemcpy(p->fb_z0, z.data(), z.size() * 8, cudaMemcpyHostToDevice));
  } else {
    std::vector<float> zf(z.size());
    for (size_t i = 0; i < z.size(); ++i) zf[i] = (float)z[i];
    JD_CUDA(cudaMemcpy(p->fb_z0, zf.data(), zf.size() * 4, cudaMemcpyHostToDevice));
  }
  return JD_OK;
}

// Buffers of the feedback sweeps for padded size LP (the gradient also needs the states,
// the flags and the gradient partials); raises the stack limit for the jump routines.
static jd_status fb_ensure(jd_problem *p, const FbOps *ops, bool grad) {
  const int LP = ops->NX * ops->NV, Nt = p->desc.Nt;
  const int64_t M = p->desc.M, nblk = ceil_div(M, FB_TPB);
  const size_t es = elem_size(p);
  const int64_t nwarp = nblk * (FB_TPB / 32);
  if (p->fb_LP != LP) {
    free_dev(p, p->fb_mu);
    free_dev(p, p->fb_partW);
    free_dev(p, p->fb_partG);
    p->fb_LP = LP;
  }
  jd_status s = JD_OK;
  if (!p->fb_mu) s = dev_alloc(p, &p->fb_mu, (size_t)Nt * LP * es, "feedback weights");
  if (!s && !p->fb_mu64)
    s = dev_alloc(p, (void **)&p->fb_mu64, (size_t)Nt * FB_NB * FB_NB * 8, "feedback weights (FP64)");
  if (!s && !p->fb_partC) s = dev_alloc(p, (void **)&p->fb_partC, (size_t)nblk * 8, "feedback cost partials");
  if (!s && grad && !p->fb_grad)
    s = dev_alloc(p, (void **)&p->fb_grad, (size_t)Nt * FB_NB * FB_NB * 8, "feedback gradient");
  if (!s && grad && !p->fb_traj)
    s = dev_alloc(p, &p->fb_traj, (size_t)(Nt + 1) * 2 * M * es, "feedback states");
  if (!s && grad && !p->fb_flags)
    s = dev_alloc(p, (void **)&p->fb_flags, (size_t)ceil_div(Nt, 32) * M * 4, "feedback jump flags");
  if (!s && grad && !p->fb_partW)
    s = dev_alloc(p, &p->fb_partW, (size_t)nwarp * Nt * LP * es, "feedback warp partials");
  if (!s && grad && !p->fb_partG)
    s = dev_alloc(p, (void **)&p->fb_partG, (size_t)fb_groups(nwarp) * Nt * LP * 8, "feedback group partials");
  if (!s && !p->fb_z0) s = dev_alloc(p, &p->fb_z0, (size_t)2 * RING_MAX * es, "ring initial states");
  if (s) return s;
  // once per padded size: raising the limit reallocates local memory (a device-wide sync)
  const size_t need = ops->stack_bytes();
  if (need > p->fb_stack) {
    size_t cur = 0;
    JD_CUDA(cudaDeviceGetLimit(&cur, cudaLimitStackSize));
    if (cur < need) JD_CUDA(cudaDeviceSetLimit(cudaLimitStackSize, need));
    p->fb_stack = need;
  }
  return JD_OK;
}

// Forward (and with grad the adjoint) sweep under feedback, then the FP64 finalize into
// scal_d[S_J] and grad_out (device, Nt*L; null for the cost only).
// store: a cost evaluation that also keeps the states (the exact adjoint's forward half;
// used for line-search trials).  forward_done: the states, the weights in kernel
// precision and the cost partials already belong to mu (the accepted trial): only the
// adjoint half runs.
static jd_status fb_run(jd_problem *p, const jd_feedback_desc *fb, const double *mu, jd_memspace ms,
                        double *grad_out, bool store = false, bool forward_done = false) {
  jd_status s = fb_validate(p, fb);
  if (s) return s;
  if (!mu) return fail(JD_ERR_INVALID_ARG, "mu is NULL");
  if (ms != JD_MEM_HOST && ms != JD_MEM_DEVICE) return fail(JD_ERR_INVALID_ARG, "bad memory space for mu");
  const FbOps *ops = fb_ops(p->desc.prec, fb->nx, fb->nv);
  if (!ops) return fail(JD_ERR_UNSUPPORTED, "no compiled feedback size fits nx x nv");
  const int Nt = p->desc.Nt;
  const size_t L = (size_t)fb->nx * fb->nv;
  s = set_device(p);
  if (!s) s = fb_ensure(p, ops, grad_out != nullptr || store);
  if (s) return s;
  const double *mud = mu;
  if (ms == JD_MEM_HOST) {
    if (!finite_all(mu, (size_t)Nt * L)) return fail(JD_ERR_INVALID_ARG, "mu has a non-finite entry");
    JD_CUDA(cudaMemcpyAsync(p->fb_mu64, mu, (size_t)Nt * L * 8, cudaMemcpyHostToDevice, p->stream));
    mud = p->fb_mu64;
  }
  if (!forward_done) JD_CUDA(ops->prep_mu(mud, p->fb_mu, Nt, fb->nx, fb->nv, p->stream));
  if (fb->particles && !forward_done) {
    s = fb_upload_ring(p, *fb);
    if (s) return s;
  }
  FbBufs b;
  b.mu = p->fb_mu;
  b.traj = p->fb_traj;
  b.flags = p->fb_flags;
  b.partC = p->fb_partC;
  b.partW = p->fb_partW;
  b.partG = p->fb_partG;
  int pr = -1;
  if (grad_out && fb->adjoint == JD_FB_SURROGATE) {
    // Sec. 6.5: the surrogate adjoint (bhat into the state buffer), then the forward sweep
    // with the gradient records
    pr = prof_begin(KC_FB_SUR, p->stream);
    JD_CUDA(ops->sur(p, *fb, b, p->stream));
    prof_end(pr, p->stream);
  } else if (!forward_done) {
    pr = prof_begin(KC_FB_FWD, p->stream);
    JD_CUDA(ops->fwd(p, *fb, grad_out != nullptr || store, b, p->stream));
    prof_end(pr, p->stream);
  }
  if (grad_out) {
    if (fb->adjoint != JD_FB_SURROGATE) {
      pr = prof_begin(KC_FB_ADJ, p->stream);
      JD_CUDA(ops->adj(p, *fb, b, p->stream));
      prof_end(pr, p->stream);
    }
    pr = prof_begin(KC_FB_RED, p->stream);
    JD_CUDA(ops->reduce(p, b, p->stream));
    prof_end(pr, p->stream);
  }
  pr = prof_begin(KC_FB_FIN, p->stream);
  const int64_t nblk = ceil_div(p->desc.M, FB_TPB);
  // the average runs over the particles that exist: M paths, or M/S rings of N particles
  const int64_t count = fb->particles ? p->desc.M / ring_lanes(fb->particles) * fb->particles : p->desc.M;
  JD_CUDA(fb_finalize(p->fb_partC, p->fb_partG, nblk, fb_groups(nblk * (FB_TPB / 32)), Nt, fb->nx, fb->nv,
                      ops->NX, ops->NV, count, p->scal_d + S_J, grad_out, p->stream));
  prof_end(pr, p->stream);
  return JD_OK;
}

jd_status jd_fb_cost(jd_problem *p, const jd_feedback_desc *fb, const double *mu, jd_memspace mu_space,
                     double *J) {
  if (!J) return fail(JD_ERR_INVALID_ARG, "J is NULL");
  jd_status s = fb_run(p, fb, mu, mu_space, nullptr);
  if (!s) s = read_scalars(p, S_J, 1);
  if (s) return s;
  *J = p->host_pinned[S_J];
  return std::isfinite(*J) ? JD_OK : fail(JD_ERR_NONFINITE, "J is not finite");
}

jd_status jd_fb_gradient(jd_problem *p, const jd_feedback_desc *fb, const double *mu, jd_memspace space,
                         double *J, double *grad) {
  if (!grad) return fail(JD_ERR_INVALID_ARG, "grad is NULL");
  if (space != JD_MEM_HOST && space != JD_MEM_DEVICE) return fail(JD_ERR_INVALID_ARG, "bad memory space");
  jd_status s = fb_validate(p, fb);
  if (!s && !p->fb_grad)   // the gradient buffer exists before fb_run picks its target
    s = dev_alloc(p, (void **)&p->fb_grad, (size_t)p->desc.Nt * FB_NB * FB_NB * 8, "feedback gradient");
  if (s) return s;
  s = fb_run(p, fb, mu, space, space == JD_MEM_DEVICE ? grad : p->fb_grad);
  if (s) return s;
  if (space == JD_MEM_HOST)
    JD_CUDA(cudaMemcpyAsync(grad, p->fb_grad, (size_t)p->desc.Nt * fb->nx * fb->nv * 8, cudaMemcpyDeviceToHost,
                            p->stream));
  s = read_scalars(p, S_J, 1);
  if (s) return s;
  if (J) *J = p->host_pinned[S_J];
  return std::isfinite(p->host_pinned[S_J]) ? JD_OK : fail(JD_ERR_NONFINITE, "J is not finite");
}

jd_status jd_fb_optimize(jd_problem *p, const jd_feedback_desc *fb, double *mu_inout, jd_memspace space,
                         const jd_opt_params *o, jd_opt_result *r, double *J_hist) {
  if (!mu_inout || !o || !r) return fail(JD_ERR_INVALID_ARG, "mu_inout, o and r must be non-NULL");
  if (space != JD_MEM_HOST && space != JD_MEM_DEVICE) return fail(JD_ERR_INVALID_ARG, "bad memory space");
  std::memset(r, 0, sizeof(*r));
  jd_status s = fb_validate(p, fb);
  if (s) return s;
  const int64_t n = (int64_t)p->desc.Nt * fb->nx * fb->nv;
  const double dt = p->desc.T / p->desc.Nt;
  s = set_device(p);
  if (!s && !p->fb_mu64)
    s = dev_alloc(p, (void **)&p->fb_mu64, (size_t)p->desc.Nt * FB_NB * FB_NB * 8, "feedback weights (FP64)");
  if (!s && !p->fb_mut)
    s = dev_alloc(p, (void **)&p->fb_mut, (size_t)p->desc.Nt * FB_NB * FB_NB * 8, "feedback trial weights");
  if (!s && !p->fb_grad)
    s = dev_alloc(p, (void **)&p->fb_grad, (size_t)p->desc.Nt * FB_NB * FB_NB * 8, "feedback gradient");
  if (s) return s;
  if (space == JD_MEM_HOST && !finite_all(mu_inout, (size_t)n)) return fail(JD_ERR_INVALID_ARG, "mu has a non-finite entry");
  JD_CUDA(cudaMemcpyAsync(p->fb_mu64, mu_inout, n * 8,
                          space == JD_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, p->stream));
  // Algorithm 5.4 on mu: gradient at mu^n, Armijo backtracking along -g (g = grad / dt),
  // update; the host takes each decision from the FP64 scalars read back
  double J = 0.0, pg0 = -1.0, zeta = o->zeta0 > 0 ? o->zeta0 : 1.0;
  const double zeta_max = o->zeta_max > 0 ? o->zeta_max : 1e3;
  int status = 0, it = 0;
  const uint32_t epoch0 = p->desc.epoch;
  struct EpochBack {   // the problem's sample is restored on every way out
    jd_problem *p;
    uint32_t e;
    ~EpochBack() { p->desc.epoch = e; }
  } epoch_back{p, epoch0};
  // the accepted trial's forward sweep (states kept) is the next gradient's forward half
  // (exact adjoint, one fixed sample)
  const bool reuse = fb->adjoint == JD_FB_EXACT && !o->resample;
  bool forward_done = false;
  for (it = 0; it < o->max_iter; ++it) {
    if (o->resample) p->desc.epoch = epoch0 + (uint32_t)it;   // fresh sample per iteration
    s = fb_run(p, fb, p->fb_mu64, JD_MEM_DEVICE, p->fb_grad, false, forward_done);
    if (!forward_done) r->sweeps++;
    forward_done = false;
    if (!s) JD_CUDA(fb_norm(p->fb_grad, n, dt, p->scal_d + S_PG, p->stream));
    if (!s) s = read_scalars(p, S_J, S_PG + 1);
    if (s) return s;
    r->evals++;
    J = p->host_pinned[S_J];
    const double g2 = p->host_pinned[S_PG];
    if (!std::isfinite(J) || !std::isfinite(g2)) return fail(JD_ERR_NONFINITE, "J or the gradient is not finite");
    if (J_hist) J_hist[it] = J;
    const double pg = std::sqrt(g2);
    if (pg0 < 0.0) pg0 = pg;
    r->rel_grad_norm = pg0 > 0.0 ? pg / pg0 : 0.0;
    if (r->rel_grad_norm <= o->tol_rel_grad) break;
    if (it > 0) zeta = std::fmin(2.0 * zeta, zeta_max);
    bool accepted = false;
    double Jt = 0.0;
    for (int b = 0; b <= o->max_backtracks; ++b) {
      JD_CUDA(fb_trial(p->fb_mu64, p->fb_grad, n, zeta, dt, p->fb_mut, p->stream));
      s = fb_run(p, fb, p->fb_mut, JD_MEM_DEVICE, nullptr, reuse);
      if (!s) s = read_scalars(p, S_J, 1);
      if (s) return s;
      r->evals++;
      r->sweeps++;
      Jt = p->host_pinned[S_J];
      if (Jt <= J - o->armijo_c * zeta * g2) {
        accepted = true;
        break;
      }
      zeta *= 0.5;
    }
    if (!accepted) {
      status = JD_ERR_LINESEARCH;
      break;
    }
    std::swap(p->fb_mu64, p->fb_mut);   // mu^{n+1}
    forward_done = reuse;
    J = Jt;
    if (J_hist) J_hist[it + 1] = J;
    if (zeta * pg < o->tol_step) {   // |mu^{n+1} - mu^n|_{L2} = zeta |g|_{L2}
      it++;
      break;
    }
  }
  r->iters = it;
  r->J = J;
  r->zeta = zeta;
  r->status = (jd_status)status;
  JD_CUDA(cudaMemcpyAsync(mu_inout, p->fb_mu64, n * 8,
                          space == JD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, p->stream));
  JD_CUDA(cudaStreamSynchronize(p->stream));
  return status == 0 ? JD_OK : fail((jd_status)status, "line search failed");
}

jd_status jd_optimize(jd_problem *p, double *u_inout, jd_memspace us, const jd_opt_params *o,
                      jd_opt_result *r, double *J_hist) {
  if (!p || !u_inout || !o || !r) return fail(JD_ERR_INVALID_ARG, "p, u_inout, o, r must be non-NULL");
  std::memset(r, 0, sizeof(*r));
  p->fwd_valid = false;
  jd_status s = set_device(p);
  if (!s) s = load_u(p, u_inout, us);
  if (s) return s;
  jd::OptMachine m;
  JD_CUDA(cudaEventCreateWithFlags(&m.ev, cudaEventDisableTiming));
  s = jd::opt_begin(m, p, *o, u_inout, us, J_hist);
  while (!s && m.phase != jd::OptMachine::DONE) {
    const cudaError_t e = cudaEventSynchronize(m.ev);
    s = e == cudaSuccess ? jd::opt_advance(m) : cuda_fail(e, "cudaEventSynchronize");
  }
  cudaEventDestroy(m.ev);
  if (s) return s;
  *r = m.r;
  return m.r.status;
}

}  // extern "C"
