// jd_kernels.cuh -- path kernels: one thread per Monte Carlo path, state in registers.
//
//  fwd_kernel       forward Euler-Maruyama sweep on the jump-adapted grid
//                   (Algorithms 5.1/5.2) with the running cost of
//                   eq:discrete_functional; optionally stores every state (stored
//                   variant) or a checkpoint every S steps (recompute variant).
//  adj_stored       backward adjoint sweep (eq:AdjointModel, eq:adjoint_eq_approximation)
//                   over the stored states; per-step contributions delta B^T lambda
//                   reduced across the block into FP64 partials (eq:definition_Gradient).
//  adj_recompute    the same sweep without stored states: each S-step segment is
//                   regenerated from its checkpoint and the counter-based streams into
//                   shared memory, then swept backwards.  Same arithmetic, same bits.
//
// Layouts (mloc = paths of the launch, lm = local path index):
//   traj  [ceil((Nt+1)/SV)][VD][mloc][VW] states X_k in 16-byte vectors (traj_shape: the
//                                        components of a step adjacent, SV steps a group)
//   flags [ceil(Nt/32)][mloc]           bit k%32 set when step k had a jump
//   jcnt  [2][mloc]                      jump-log records per path; first step not logged
//   ckpt  [nseg+1][D][mloc]              X_{sS} for s < nseg, X_Nt at s = nseg
//   partC [nblk]                          FP64 block sums of the per-path cost
//   partG [Nt][DU][nblk * TPB/32]         FP64 warp sums of the control sensitivities
//   partT [D+2][nblk]                     FP64 block sums of the parameter sensitivities
#pragma once

#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "jd_device.cuh"

namespace jd {

// One 16-byte vector of VW = 16 / sizeof(R) values (the unit of the stored trajectory).
template <typename R>
struct Vec16;
template <>
struct Vec16<float> {
  static __device__ __forceinline__ void store(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
  static __device__ __forceinline__ void load(const float *p, float (&o)[4]) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
};
template <>
struct Vec16<double> {
  static __device__ __forceinline__ void store(double *p, const double (&v)[2]) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
  }
  static __device__ __forceinline__ void load(const double *p, double (&o)[2]) {
    const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    o[0] = v.x; o[1] = v.y;
  }
};

template <typename R, int D>
struct TS {
  static constexpr TrajShape s = traj_shape(D, (int)sizeof(R));
  static constexpr int VW = s.VW, SV = s.SV, VD = s.VD;
};

// Asynchronous 16-byte copies global -> shared (cp.async, L2 only): each thread stages
// the vectors it will read itself, so a thread waits for its own copies only
// (cp.async.wait_group) and no barrier is needed.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename R>
struct Vec4;
template <>
struct Vec4<float> {
  static __device__ __forceinline__ void store(float *p, float a, float b, float c, float d) {
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
  }
  static __device__ __forceinline__ void load(const float *p, float (&o)[4]) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
};
template <>
struct Vec4<double> {
  static __device__ __forceinline__ void store(double *p, double a, double b, double c, double d) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(a, b);
    reinterpret_cast<double2 *>(p)[1] = make_double2(c, d);
  }
  static __device__ __forceinline__ void load(const double *p, double (&o)[4]) {
    const double2 v0 = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 v1 = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    o[0] = v0.x; o[1] = v0.y; o[2] = v1.x; o[3] = v1.y;
  }
};

// ---------------------------------------------------------------------------
// Jump log: for every step with jumps, the post-jump sub-states of the jump-adapted
// grid in time order (one record per jump: step index k with the jump's position i
// within its step, time fraction theta, state Y right after the jump).  A step is logged
// only when all its records fit, and the first step that does not fit closes the log, so
// the logged steps are exactly the jump steps before that one; any other jump step is
// regenerated from the counter-based streams.
//   kt[r * stride + idx] = (16 k + i, theta),   y[(r * D + c) * stride + idx] = Y_c
// (i < NMAX = 16; in FP32 the code is stored as the bits of an int, exact for every N_t)
// ---------------------------------------------------------------------------
template <typename R>
struct V2;
template <>
struct V2<float> {
  using T = float2;
  static __device__ __forceinline__ T make(float a, float b) { return make_float2(a, b); }
  // a log record (code 16 k + i, theta); the code travels as the bits of an int
  static __device__ __forceinline__ T rec(int code, float theta) { return make_float2(__int_as_float(code), theta); }
  static __device__ __forceinline__ int code(T t) { return __float_as_int(t.x); }
};
template <>
struct V2<double> {
  using T = double2;
  static __device__ __forceinline__ T make(double a, double b) { return make_double2(a, b); }
  static __device__ __forceinline__ T rec(int code, double theta) { return make_double2((double)code, theta); }
  static __device__ __forceinline__ int code(T t) { return (int)t.x; }
};

template <typename R, int D>
struct JLog {
  typename V2<R>::T *kt;
  R *y;
  int64_t stride;   // mloc (global log) or TPB (shared log)
  int cap;          // records per path
};

template <typename R, int D>
struct LogWriter {
  JLog<R, D> L;
  int64_t idx;
  int r = 0;
  int kovf = 0x7fffffff;   // first step whose records did not fit
  __device__ __forceinline__ bool fits(int n) const { return r + n <= L.cap; }
  // Whether the n records of step k fit.  A step that does not fit closes the log, so
  // the logged steps are exactly the jump steps before kovf: a backward sweep that has
  // not reached kovf regenerates nothing.  In FP32 a step with three or more jumps
  // (probability about (lambda dt)^3 / 6) closes it too, so a logged step holds one or two
  // records and the FP32 readers take them without a loop or a call.
  __device__ __forceinline__ bool take(int n, int k) {
    if ((sizeof(R) == 8 || n <= 2) && r + n <= L.cap) return true;
    kovf = min(kovf, k);
    L.cap = r;
    return false;
  }
  // record of the i-th jump (time order) of step k
  __device__ __forceinline__ void put(int k, int i, R theta, const R (&y)[D]) {
    L.kt[(int64_t)r * L.stride + idx] = V2<R>::rec(16 * k + i, theta);
#pragma unroll
    for (int c = 0; c < D; ++c) L.y[((int64_t)r * D + c) * L.stride + idx] = y[c];
    ++r;
  }
};

template <typename R, int D>
struct LogReader {
  JLog<R, D> L;
  int64_t idx;
  int rec;   // latest unconsumed record, -1 when empty
  R rk;      // its step index (or -1)
  __device__ __forceinline__ R step_of(int r) const {
    return r >= 0 ? (R)(V2<R>::code(L.kt[(int64_t)r * L.stride + idx]) >> 4) : R(-1);
  }
  __device__ __forceinline__ void init(int count) {
    rec = count - 1;
    rk = step_of(rec);
  }
  __device__ __forceinline__ bool has(int k) const { return rk == (R)k; }
  __device__ __forceinline__ void pop(R &theta, R (&y)[D]) {
    theta = L.kt[(int64_t)rec * L.stride + idx].y;
#pragma unroll
    for (int c = 0; c < D; ++c) y[c] = L.y[((int64_t)rec * D + c) * L.stride + idx];
    --rec;
    rk = step_of(rec);
  }
};

// Reads the log backwards for sweeps that know from the jump flags which steps had jumps
// (every jump step before the log's closing step is logged).  The current record (its
// time fraction, post-jump state and position within its step) waits in registers; a
// pop hands it over and loads the next one, which is needed only at the path's next jump
// step.  The popped record's position tells whether another record of the same step
// follows, so no pop waits for a load except within a step of two or more jumps.
template <typename R, int D>
struct LogReader2 {
  const typename V2<R>::T *kt;   // row of the current record in this path's column
  const R *y;
  int64_t stride;
  int rec;                        // index of the current record (-1: none left)
  int ci;                         // current record: position within its step,
  R cth, cy[D];                   // time fraction, post-jump state
  __device__ __forceinline__ void load() {
    const typename V2<R>::T t = kt[0];
    ci = V2<R>::code(t) & 15;
    cth = t.y;
#pragma unroll
    for (int c = 0; c < D; ++c) cy[c] = y[(int64_t)c * stride];
  }
  __device__ __forceinline__ void init(const JLog<R, D> &L, int64_t idx, int count) {
    stride = L.stride;
    rec = count - 1;
    const int64_t r0 = max(rec, 0);
    kt = L.kt + r0 * stride + idx;
    y = L.y + r0 * D * stride + idx;
    if (count > 0) load();
  }
  // take: hand over the current record (position i within its step, time fraction theta,
  // state yo) and load the next one; otherwise theta = 1, yo = x, i = 0 and the reader
  // keeps its record (it loads the same row again).  No branch.
  __device__ __forceinline__ int pop_if(bool take, const R (&x)[D], R &theta, R (&yo)[D]) {
    theta = take ? cth : R(1);
#pragma unroll
    for (int c = 0; c < D; ++c) yo[c] = take ? cy[c] : x[c];
    const int i = take ? ci : 0;
    const int64_t back = (take && rec > 0) ? stride : 0;
    kt -= back;
    y -= back * D;
    rec -= take ? 1 : 0;
    load();
    return i;
  }
  // hands over the current record; returns its position within its step (another record
  // of the same step follows when it is > 0)
  __device__ __forceinline__ int pop(R &theta, R (&yo)[D]) {
    theta = cth;
#pragma unroll
    for (int c = 0; c < D; ++c) yo[c] = cy[c];
    const int i = ci;
    const int64_t back = rec > 0 ? stride : 0;   // the last record is reloaded, not passed
    kt -= back;
    y -= back * D;
    --rec;
    load();
    return i;
  }
};

struct NoLog {};

// Recompute variant: the preferred steps per checkpoint segment (the plan widens it to
// 32 or 64 when the memory budget does not hold the checkpoints; KParams::S).
template <int D>
__host__ __device__ constexpr int seg_len() {
  return D <= 8 ? 16 : 8;
}

// Steps with one jump take a short path (the common case); two or more go through
// build_jump_step.  The one-jump paths (inline and out of line) apply the additive map;
// a step of a Keilson-Storer problem with jumps always takes build_jump_step, whose jump
// map covers every law.
// The one-jump step out of line: sub-step to the jump, jump, sub-step to t_{k+1}.  x is
// updated in place; y1 receives the post-jump state; returns the jump's time fraction.
template <typename R, int D, int DU>
__device__ __noinline__ R one_jump_substeps(const KParams<R, D, DU> &kp, int k, uint32_t m, const R *z,
                                            const R *uk, R *x, R *y1) {
  using M = Ar<R>;
  R xih[D], z1[D], zz[D], ul[DU], xl[D];
#pragma unroll
  for (int c = 0; c < D; ++c) {
    zz[c] = z[c];
    xl[c] = x[c];
  }
#pragma unroll
  for (int l = 0; l < DU; ++l) ul[l] = uk[l];
  const R th = slot0_draws(kp, k, m, xih, z1);
  euler_substep(kp, M::mul(kp.dt, th), zz, ul, xl);
#pragma unroll
  for (int c = 0; c < D; ++c) {
    xl[c] = M::add(xl[c], M::mul(kp.jump_scale, xih[c]));
    y1[c] = xl[c];
  }
  euler_substep(kp, M::mul(kp.dt, M::sub(R(1), th)), z1, ul, xl);
#pragma unroll
  for (int c = 0; c < D; ++c) x[c] = xl[c];
  return th;
}

// The step has exactly one jump and the additive jump map (the one-jump paths).
template <typename R, int D, int DU>
__device__ __forceinline__ bool one_jump(const KParams<R, D, DU> &kp, uint32_t w0) {
  return kp.jump_law != JD_JUMP_KS && kp.npair == MainWords<D>::PD && (unsigned long long)w0 < kp.thr[1];
}

// The one-jump step inline, its slot draws (time fraction th, jump size xih, second
// sub-step normals z1) given: sub-step to the jump, jump, sub-step to t_{k+1}.
template <typename R, int D, int DU, typename LW>
__device__ __forceinline__ void one_jump_inline(const KParams<R, D, DU> &kp, int k, R th, const R (&xih)[D],
                                                const R (&z)[D], const R (&z1)[D], const R (&uk)[DU], R (&x)[D],
                                                LW &lw) {
  using M = Ar<R>;
  euler_substep(kp, M::mul(kp.dt, th), z, uk, x);
#pragma unroll
  for (int c = 0; c < D; ++c) x[c] = M::add(x[c], M::mul(kp.jump_scale, xih[c]));
  if constexpr (!std::is_same<LW, NoLog>::value) {
    if (lw.take(1, k)) lw.put(k, 0, th, x);
  }
  euler_substep(kp, M::mul(kp.dt, M::sub(R(1), th)), z1, uk, x);
}

// x <- x + dt f + sigma sqrt(dt) z: the step without jumps.
template <typename KP, typename R, int D>
__device__ __forceinline__ void plain_update(const KP &kp, const R (&f)[D], const R (&z)[D], R (&x)[D]) {
  using M = Ar<R>;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    if constexpr (Pr<R>::on && D % 2 == 0) {   // components c, c+1 in one paired FMA each
      if (c % 2 == 0) {
        Pr<R>::fma(kp.dt, kp.dt, f[c], f[c + 1], x[c], x[c + 1]);
        Pr<R>::fma(kp.sig_sqdt[c], kp.sig_sqdt[c + 1], z[c], z[c + 1], x[c], x[c + 1]);
      }
    } else {
      x[c] = M::fma(kp.sig_sqdt[c], z[c], M::fma(kp.dt, f[c], x[c]));
    }
  }
}

// Step k from x (in place) once the main-stream draws z and the Poisson word w0 are
// taken; returns the number of jumps.
// INLINE_JUMP: the one-jump case inline, or out of line (the replay of the parameter-
// gradient recompute adjoint, whose loop must stay small for the instruction cache, and
// the paired sweep of two controls).
// kh: the source of the drift, noise and step coefficients of the step without jumps
// (kp itself or a HotFwd); the jump paths read kp.  RK: the inline slot draws take the
// round keys of kp (a __grid_constant__ parameter).
template <typename R, int D, int DU, typename LW, bool INLINE_JUMP = true, typename KH = KParams<R, D, DU>,
          bool RK = false>
__device__ __forceinline__ int step_from_draws(const KParams<R, D, DU> &kp, const KH &kh, int k, uint32_t m,
                                               uint32_t w0, const R (&z)[D], const R (&uk)[DU], R (&x)[D],
                                               LW &lw) {
  using M = Ar<R>;
  constexpr bool LOG = !std::is_same<LW, NoLog>::value;
  if (!has_jump(kp, w0)) {
    R f[D];
    drift(kh, x, uk, f);
    plain_update(kh, f, z, x);
    return 0;
  }
  if (!INLINE_JUMP && one_jump(kp, w0)) {
    // copies: an address taken of x or uk themselves would move them to local memory
    R zc[D], xc[D], uc[DU], y1[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      zc[c] = z[c];
      xc[c] = x[c];
    }
#pragma unroll
    for (int l = 0; l < DU; ++l) uc[l] = uk[l];
    const R th = one_jump_substeps(kp, k, m, zc, uc, xc, y1);
#pragma unroll
    for (int c = 0; c < D; ++c) x[c] = xc[c];
    if constexpr (LOG) {
      if (lw.take(1, k)) lw.put(k, 0, th, y1);
    }
    return 1;
  }
  if (INLINE_JUMP && one_jump(kp, w0)) {
    R xih[D], z1[D];
    const R th = slot0_draws<RK>(kp, k, m, xih, z1);
    one_jump_inline(kp, k, th, xih, z, z1, uk, x, lw);
    return 1;
  }
  // two or more jumps: the general routine takes pointers, so pass copies and keep
  // z, uk and x themselves in registers on the common paths
  JumpStep<R, D> S;
  R xl[D], zl[D], ul[DU];
#pragma unroll
  for (int c = 0; c < D; ++c) {
    xl[c] = x[c];
    zl[c] = z[c];
  }
#pragma unroll
  for (int l = 0; l < DU; ++l) ul[l] = uk[l];
  build_jump_step(kp, k, m, w0, zl, ul, xl, &S);
#pragma unroll
  for (int c = 0; c < D; ++c) x[c] = S.Y[S.n + 1][c];
  if constexpr (LOG) {
    if (lw.take(S.n, k)) {
      for (int i = 0; i < S.n; ++i) {
        R y[D];
#pragma unroll
        for (int c = 0; c < D; ++c) y[c] = S.Y[i + 1][c];
        lw.put(k, i, S.th[i], y);
      }
    }
  }
  return S.n;
}

// One uniform step k from x (in place); returns the number of jumps.  With a LogWriter
// the post-jump states of the step are recorded.  zo (optional, stride zs) receives the
// step's main-stream normals Z_{k,0}.
template <typename R, int D, int DU, typename LW, bool ZOUT = false, bool INLINE_JUMP = true,
          typename KH = KParams<R, D, DU>, bool RK = false>
__device__ __forceinline__ int forward_step_h(const KParams<R, D, DU> &kp, const KH &kh, int k, uint32_t m,
                                              const R *__restrict__ u, R (&x)[D], LW &lw,
                                              R *zo = nullptr, int zs = 0) {
  R z[D];
  const uint32_t w0 = main_draws<RK>(kp, k, m, z);
  if constexpr (ZOUT) {
#pragma unroll
    for (int c = 0; c < D; ++c) zo[c * zs] = z[c];
  }
  R uk[DU];
#pragma unroll
  for (int l = 0; l < DU; ++l) uk[l] = __ldg(u + (size_t)k * DU + l);
  return step_from_draws<R, D, DU, LW, INLINE_JUMP, KH, RK>(kp, kh, k, m, w0, z, uk, x, lw);
}

template <typename R, int D, int DU, typename LW, bool ZOUT = false, bool INLINE_JUMP = true>
__device__ __forceinline__ int forward_step(const KParams<R, D, DU> &kp, int k, uint32_t m,
                                            const R *__restrict__ u, R (&x)[D], LW &lw,
                                            R *zo = nullptr, int zs = 0) {
  return forward_step_h<R, D, DU, LW, ZOUT, INLINE_JUMP>(kp, kp, k, m, u, x, lw, zo, zs);
}

// Step k of two controls u, u2 on the same random data (the pair of Armijo trials of one
// sweep): one draw of the main stream, and on a jump step the same jump times and sizes
// for both states.  Each state's arithmetic is forward_step's, so each result is bitwise
// the one of a sweep of its control alone.  Returns the number of jumps.
template <typename R, int D, int DU, typename LW, typename KH, bool RK = false>
__device__ __forceinline__ int forward_step2(const KParams<R, D, DU> &kp, const KH &kh, int k, uint32_t m,
                                             uint32_t w0, const R (&z)[D], const R *__restrict__ u, R (&x)[D],
                                             LW &lw, const R *__restrict__ u2, R (&x2)[D], LW &lw2) {
  R uk[DU], uk2[DU];
#pragma unroll
  for (int l = 0; l < DU; ++l) {
    uk[l] = __ldg(u + (size_t)k * DU + l);
    uk2[l] = __ldg(u2 + (size_t)k * DU + l);
  }
  if (!has_jump(kp, w0)) {
    R f[D], f2[D];
    drift(kh, x, uk, f);
    drift(kh, x2, uk2, f2);
    plain_update(kh, f, z, x);
    plain_update(kh, f2, z, x2);
    return 0;
  }
  if (one_jump(kp, w0)) {   // one slot draw for both states
    R xih[D], z1[D];
    const R th = slot0_draws<RK>(kp, k, m, xih, z1);
    one_jump_inline(kp, k, th, xih, z, z1, uk, x, lw);
    one_jump_inline(kp, k, th, xih, z, z1, uk2, x2, lw2);
    return 1;
  }
  const int n = step_from_draws<R, D, DU, LW, false>(kp, kp, k, m, w0, z, uk, x, lw);
  step_from_draws<R, D, DU, LW, false>(kp, kp, k, m, w0, z, uk2, x2, lw2);
  return n;
}

// dt l(x, t_k) = sum_c (q_c dt / 2) (x_c - xd_c(t_k))^2
template <typename KP, typename R, int D>
__device__ __forceinline__ R cost_term(const KP &kp, const R (&x)[D], const R *__restrict__ xdk) {
  using M = Ar<R>;
  R t = R(0);
  if constexpr (Pr<R>::on && D % 2 == 0) {
    // differences and weights in pairs, the sum in the same order as below
#pragma unroll
    for (int c = 0; c < D; c += 2) {
      R e0, e1, h0, h1;
      Pr<R>::sub(x[c], x[c + 1], __ldg(xdk + c), __ldg(xdk + c + 1), e0, e1);
      Pr<R>::mul(kp.hqdt[c], kp.hqdt[c + 1], e0, e1, h0, h1);
      t = M::fma(h0, e0, t);
      t = M::fma(h1, e1, t);
    }
    return t;
  }
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const R e = M::sub(x[c], __ldg(xdk + c));
    t = M::fma(M::mul(kp.hqdt[c], e), e, t);
  }
  return t;
}

// Backward through a step that had jumps: regenerate its draws and sub-states from
// X_k, then sweep the sub-steps in reverse.  mu enters as the derivative w.r.t.
// X_{k+1} and leaves as the derivative w.r.t. X_k (before the cost term at t_k).
template <typename R, int D, int DU, bool THETA>
__device__ __noinline__ void jump_backward(const KParams<R, D, DU> &kp, int k, uint32_t m,
                                           const R *xk, const R *uk, R *mu_io, R *g_io,
                                           R *th_io) {
  using M = Ar<R>;
  R z0[D];
  const uint32_t w0 = main_draws(kp, k, m, z0);
  JumpStep<R, D> S;
  build_jump_step(kp, k, m, w0, z0, uk, xk, &S);
  R mu[D], g[DU];
#pragma unroll
  for (int c = 0; c < D; ++c) mu[c] = mu_io[c];
#pragma unroll
  for (int l = 0; l < DU; ++l) g[l] = g_io[l];
  // parameter sensitivities need the sub-step normals Z_i and the unit jump sizes;
  // they are regenerated per slot, walking the slots backwards (slot order[i] gives
  // the jump after sub-step i and the normals of sub-step i+1)
  R xih_cur[D], z_cur[D];
  if (THETA && S.n > 0) slot_draws(kp, k, m, S.order[S.n - 1], xih_cur, z_cur);
#pragma unroll 1
  for (int i = S.n; i >= 0; --i) {
    R y[D];
#pragma unroll
    for (int c = 0; c < D; ++c) y[c] = S.Y[i][c];
    const R de = S.delta[i];
    if (i < S.n) {
      if (THETA) {
        // jump of slot order[i] after sub-step i: xih_cur holds its unit size; the
        // derivative in s sums over the components the jump moves
        R s = R(0);
#pragma unroll
        for (int c = 0; c < D; ++c)
          if (c >= kp.kvel) s = M::fma(mu[c], xih_cur[c], s);
        th_io[D + 1] = M::add(th_io[D + 1], s);
      }
      if (kp.jump_law == JD_JUMP_KS) jump_adjoint(kp, mu);   // now w.r.t. the pre-jump state
    }
    if (THETA) {
      R zi[D];
      if (i == 0) {
#pragma unroll
        for (int c = 0; c < D; ++c) zi[c] = z0[c];
      } else {
        // normals of sub-step i come from slot order[i-1]
        if (i < S.n) slot_draws(kp, k, m, S.order[i - 1], xih_cur, z_cur);
#pragma unroll
        for (int c = 0; c < D; ++c) zi[c] = z_cur[c];
      }
      const R sq = M::sqrt(de);
#pragma unroll
      for (int c = 0; c < D; ++c) th_io[1 + c] = M::fma(M::mul(mu[c], sq), zi[c], th_io[1 + c]);
      if (kp.has_dA) {
        R s = R(0);
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
          for (int c = 0; c < D; ++c) s = M::fma(M::mul(mu[r], kp.dA[r * D + c]), y[c], s);
        th_io[0] = M::fma(de, s, th_io[0]);
      }
    }
    control_sensitivity(kp, mu, de, g);
    adjoint_update(kp, y, de, mu);
  }
#pragma unroll
  for (int c = 0; c < D; ++c) mu_io[c] = mu[c];
#pragma unroll
  for (int l = 0; l < DU; ++l) g_io[l] = g[l];
}

// Coefficients of the forward step without jumps (drift, noise scale, step, cost
// weights), held in registers for the forward kernel's step loop like HotCoef below.
template <typename R, int D, int DU>
struct HotFwd {
  R A[D * D], C[D * D], B[D * DU], sig_sqdt[D], hqdt[D];
  R dt;
  int cubic;
};

// Coefficients of the adjoint step (A, C, B, dt, q dt) held in registers for a kernel's
// step loop.  Each value passes through an empty asm statement, so the compiler cannot
// rematerialise it from the parameter bank at every use inside the loop.  CUB = 0 or 1
// makes the drift family a compile-time constant (no branch on it in the loop); -1 reads
// it at run time.
template <int CUB>
struct CubicFlag {
  static constexpr int cubic = CUB;
};
template <>
struct CubicFlag<-1> {
  int cubic;
};
template <typename R, int D, int DU, int CUB = -1>
struct HotCoef : CubicFlag<CUB> {
  R A[D * D], C[D * D], B[D * DU], qdt[D], jgain[D];
  R dt;
  int jump_law;
};

__device__ __forceinline__ float reg_pin(float v) {
  asm volatile("" : "+f"(v));
  return v;
}
__device__ __forceinline__ double reg_pin(double v) {
  asm volatile("" : "+d"(v));
  return v;
}

// withB = false zeroes B: the control sensitivities of that thread are then exactly 0
// (an inactive thread of the last block, which replays path 0, adds nothing without a
// select per step).
template <int CUB = -1, typename R, int D, int DU>
__device__ __forceinline__ HotCoef<R, D, DU, CUB> hot_coef(const KParams<R, D, DU> &kp, bool withB = true) {
  HotCoef<R, D, DU, CUB> h;
#pragma unroll
  for (int i = 0; i < D * D; ++i) {
    h.A[i] = reg_pin(kp.A[i]);
    h.C[i] = (CUB == 1 || (CUB == -1 && kp.cubic)) ? reg_pin(kp.C[i]) : R(0);
  }
#pragma unroll
  for (int i = 0; i < D * DU; ++i) h.B[i] = reg_pin(withB ? kp.B[i] : R(0));
#pragma unroll
  for (int c = 0; c < D; ++c) {
    h.qdt[c] = reg_pin(kp.qdt[c]);
    h.jgain[c] = reg_pin(kp.jgain[c]);
  }
  h.dt = reg_pin(kp.dt);
  h.jump_law = kp.jump_law;
  if constexpr (CUB == -1) h.cubic = kp.cubic;
  return h;
}

template <typename R, int D, int DU>
__device__ __forceinline__ HotFwd<R, D, DU> hot_fwd(const KParams<R, D, DU> &kp) {
  HotFwd<R, D, DU> h;
#pragma unroll
  for (int i = 0; i < D * D; ++i) {
    h.A[i] = reg_pin(kp.A[i]);
    h.C[i] = kp.cubic ? reg_pin(kp.C[i]) : R(0);
  }
#pragma unroll
  for (int i = 0; i < D * DU; ++i) h.B[i] = reg_pin(kp.B[i]);
#pragma unroll
  for (int c = 0; c < D; ++c) {
    h.sig_sqdt[c] = reg_pin(kp.sig_sqdt[c]);
    h.hqdt[c] = reg_pin(kp.hqdt[c]);
  }
  h.dt = reg_pin(kp.dt);
  h.cubic = kp.cubic;
  return h;
}

// Pinned copies pay for d <= 2 (a handful of registers); for larger d the A and C blocks
// alone would take 2 d^2 registers, and the kernels read kp.
template <int D>
constexpr bool pin_coef() {
  return D <= 2;
}
template <bool PIN, typename H, typename R, int D, int DU>
__device__ __forceinline__ const typename std::conditional<PIN, H, KParams<R, D, DU>>::type &coef_src(
    const KParams<R, D, DU> &kp, const H &h) {
  if constexpr (PIN)
    return h;
  else
    return kp;
}

// Backward through step k from the state X_k; g receives the step's contribution.
// Jump steps use the log when it holds the step (u-gradient only), else regenerate.
// zi (optional, stride zs): the step's main-stream normals kept by the forward replay;
// without it the parameter gradients regenerate them.
// kh: the source of A, C, B, dt and q dt for the arithmetic (kp itself or a HotCoef).
template <typename R, int D, int DU, bool THETA, typename LR, bool ZIN = false, typename KH = KParams<R, D, DU>>
__device__ __forceinline__ void backward_step(const KParams<R, D, DU> &kp, const KH &kh, int k, uint32_t m,
                                              bool jumped, const R (&xk)[D],
                                              const R *__restrict__ u, const R *__restrict__ xd,
                                              R (&mu)[D], R (&g)[DU], R (&th)[D + 2], LR &lr,
                                              const R *zi = nullptr, int zs = 0) {
  using M = Ar<R>;
#pragma unroll
  for (int l = 0; l < DU; ++l) g[l] = R(0);
  if (jumped && !THETA && lr.has(k)) {
    // sub-steps n..1 from the logged post-jump states, then sub-step 0 from X_k
    R thn = R(1);
    while (lr.has(k)) {
      R the, y[D];
      lr.pop(the, y);
      const R de = M::mul(kh.dt, M::sub(thn, the));
      control_sensitivity(kh, mu, de, g);
      adjoint_update(kh, y, de, mu);
      jump_adjoint(kp, mu);   // across the jump that produced y
      thn = the;
    }
    const R de0 = M::mul(kh.dt, thn);
    control_sensitivity(kh, mu, de0, g);
    adjoint_update(kh, xk, de0, mu);
  } else if (jumped) {
    while (lr.has(k)) {   // THETA: the log is not used, but stay in step with it
      R the, y[D];
      lr.pop(the, y);
    }
    R xl[D], ml[D], gl[DU], tl[D + 2], ul[DU];
#pragma unroll
    for (int c = 0; c < D; ++c) { xl[c] = xk[c]; ml[c] = mu[c]; }
#pragma unroll
    for (int l = 0; l < DU; ++l) { gl[l] = R(0); ul[l] = __ldg(u + (size_t)k * DU + l); }
#pragma unroll
    for (int t = 0; t < D + 2; ++t) tl[t] = th[t];
    jump_backward<R, D, DU, THETA>(kp, k, m, xl, ul, ml, gl, tl);
#pragma unroll
    for (int c = 0; c < D; ++c) mu[c] = ml[c];
#pragma unroll
    for (int l = 0; l < DU; ++l) g[l] = gl[l];
#pragma unroll
    for (int t = 0; t < D + 2; ++t) th[t] = tl[t];
  } else {
    if (THETA) {
      R z[D];
      if constexpr (ZIN) {
#pragma unroll
        for (int c = 0; c < D; ++c) z[c] = zi[c * zs];
      } else {
        (void)main_draws(kp, k, m, z);
      }
#pragma unroll
      for (int c = 0; c < D; ++c) th[1 + c] = M::fma(M::mul(mu[c], kp.sqdt), z[c], th[1 + c]);
      if (kp.has_dA) {
        R s = R(0);
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
          for (int c = 0; c < D; ++c) s = M::fma(M::mul(mu[r], kp.dA[r * D + c]), xk[c], s);
        th[0] = M::fma(kp.dt, s, th[0]);
      }
    }
    control_sensitivity(kh, mu, kh.dt, g);
    adjoint_update(kh, xk, kh.dt, mu);
  }
  if (k >= 1) {
    if constexpr (Pr<R>::on && D % 2 == 0) {
#pragma unroll
      for (int c = 0; c < D; c += 2) {
        R e0, e1;
        Pr<R>::sub(xk[c], xk[c + 1], __ldg(xd + (size_t)k * D + c), __ldg(xd + (size_t)k * D + c + 1), e0, e1);
        Pr<R>::fma(kh.qdt[c], kh.qdt[c + 1], e0, e1, mu[c], mu[c + 1]);
      }
    } else {
#pragma unroll
      for (int c = 0; c < D; ++c)
        mu[c] = M::fma(kh.qdt[c], M::sub(xk[c], __ldg(xd + (size_t)k * D + c)), mu[c]);
    }
  }
}

// Target row x_d(t_k): D values, as vector loads where the row's size and alignment allow.
template <typename R, int D>
__device__ __forceinline__ void load_row(const R *__restrict__ p, R (&o)[D]) {
  if constexpr (sizeof(R) == 4 && D % 4 == 0) {
#pragma unroll
    for (int c = 0; c < D; c += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4 *>(p + c));
      o[c] = v.x; o[c + 1] = v.y; o[c + 2] = v.z; o[c + 3] = v.w;
    }
  } else if constexpr (sizeof(R) == 4 && D % 2 == 0) {
#pragma unroll
    for (int c = 0; c < D; c += 2) {
      const float2 v = __ldg(reinterpret_cast<const float2 *>(p + c));
      o[c] = v.x; o[c + 1] = v.y;
    }
  } else if constexpr (sizeof(R) == 8 && D % 2 == 0) {
#pragma unroll
    for (int c = 0; c < D; c += 2) {
      const double2 v = __ldg(reinterpret_cast<const double2 *>(p + c));
      o[c] = v.x; o[c + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int c = 0; c < D; ++c) o[c] = __ldg(p + c);
  }
}

// mu += q dt (X_k - x_d(t_k)): the running cost's gradient at a grid point k >= 1 (the
// operations of backward_step's last part).
template <typename KH, typename R, int D>
__device__ __forceinline__ void cost_gradient(const KH &kh, const R (&xk)[D], const R (&xdk)[D], R (&mu)[D]) {
  using M = Ar<R>;
  if constexpr (Pr<R>::on && D % 2 == 0) {
#pragma unroll
    for (int c = 0; c < D; c += 2) {
      R e0, e1;
      Pr<R>::sub(xk[c], xk[c + 1], xdk[c], xdk[c + 1], e0, e1);
      Pr<R>::fma(kh.qdt[c], kh.qdt[c + 1], e0, e1, mu[c], mu[c + 1]);
    }
  } else {
#pragma unroll
    for (int c = 0; c < D; ++c) mu[c] = M::fma(kh.qdt[c], M::sub(xk[c], xdk[c]), mu[c]);
  }
}

// Backward through step k (no parameter gradients) when the log holds the step's jump
// sub-grid (jumped: the step had jumps), or the step had no jump: the logged sub-steps in
// reverse (sub-step i from its post-jump state Y_i over delta_i = dt (theta_{i+1} -
// theta_i), then back across the jump that produced Y_i), then sub-step 0 from X_k over
// dt theta_1, which is dt for a step without jumps.  The operations of backward_step's log
// branch, and of jump_backward sub-step by sub-step, so the result is the same bits
// whichever form a sweep takes.  maybe = false: no lane of the warp jumped at step k (a
// warp-uniform hint).  The cost term at t_k is the caller's.
// One logged sub-step backwards: the record's sub-step, then back across its jump.
template <typename R, int D, int DU, typename KH>
__device__ __forceinline__ int logged_substep(const KH &kh, R (&mu)[D], R (&g)[DU], R &thn, LogReader2<R, D> &lr) {
  using M = Ar<R>;
  R the, y[D];
  const int i = lr.pop(the, y);
  const R de = M::mul(kh.dt, M::sub(thn, the));
  control_sensitivity(kh, mu, de, g);
  adjoint_update(kh, y, de, mu);
  jump_adjoint(kh, mu);   // the identity for the additive laws (times 1, bit for bit)
  thn = the;
  return i;
}

// The records of a step's second and later jumps, out of line, on copies: the FP64 form
// (with it the scalar FP64 problem's stored adjoint took 0.085 ms per launch, with the FP32
// form and its log closed at three jumps 0.135 ms).
template <typename R, int D, int DU, typename KH>
__device__ __noinline__ void logged_more(const KH kh, R *mu_io, R *g_io, R *thn_io, LogReader2<R, D> *lr) {
  R mu[D], g[DU], thn = *thn_io;
#pragma unroll
  for (int c = 0; c < D; ++c) mu[c] = mu_io[c];
#pragma unroll
  for (int l = 0; l < DU; ++l) g[l] = g_io[l];
  int i;
  do {
    i = logged_substep(kh, mu, g, thn, *lr);
  } while (i > 0);
#pragma unroll
  for (int c = 0; c < D; ++c) mu_io[c] = mu[c];
#pragma unroll
  for (int l = 0; l < DU; ++l) g_io[l] = g[l];
  *thn_io = thn;
}

template <typename R, int D, int DU, typename KH>
__device__ __forceinline__ void backward_logged(const KH &kh, const R (&xk)[D], R (&mu)[D], R (&g)[DU],
                                                LogReader2<R, D> &lr, bool maybe, bool jumped) {
  using M = Ar<R>;
#pragma unroll
  for (int l = 0; l < DU; ++l) g[l] = R(0);
  R thn = R(1), de0 = kh.dt;
  if (maybe) {
    // every lane of the warp runs one sub-step: the lanes that jumped at step k take
    // their step's last logged jump (its sub-step, then back across the jump); the others
    // a sub-step of length 0, which leaves g and mu as they are (g + 0 s, mu + 0 t)
    R the, y[D];
    const int i = lr.pop_if(jumped, xk, the, y);
    const R de = M::mul(kh.dt, M::sub(thn, the));
    control_sensitivity(kh, mu, de, g);
    adjoint_update(kh, y, de, mu);
    if (kh.jump_law == JD_JUMP_KS) {   // the additive laws' jump map has Jacobian I
      R mj[D];
#pragma unroll
      for (int c = 0; c < D; ++c) mj[c] = mu[c];
      jump_adjoint(kh, mj);
#pragma unroll
      for (int c = 0; c < D; ++c) mu[c] = jumped ? mj[c] : mu[c];
    }
    thn = the;
    // a step with two or more jumps (rare): the records of its earlier jumps follow; in
    // FP32 a logged step holds at most two (LogWriter::take), taken inline
    if (i > 0) {
      if constexpr (sizeof(R) == 4) {
        logged_substep(kh, mu, g, thn, lr);
      } else {
        R ml[D], gl[DU], tl = thn;
        LogReader2<R, D> ll = lr;
#pragma unroll
        for (int c = 0; c < D; ++c) ml[c] = mu[c];
#pragma unroll
        for (int l = 0; l < DU; ++l) gl[l] = g[l];
        logged_more<R, D, DU, KH>(kh, ml, gl, &tl, &ll);
#pragma unroll
        for (int c = 0; c < D; ++c) mu[c] = ml[c];
#pragma unroll
        for (int l = 0; l < DU; ++l) g[l] = gl[l];
        thn = tl;
        lr = ll;
      }
    }
    de0 = M::mul(kh.dt, thn);
  }
  control_sensitivity(kh, mu, de0, g);
  adjoint_update(kh, xk, de0, mu);
}

// As backward_logged, and a jump step the log does not hold (logged = false: the step
// lies at or after the log's closing step) is regenerated from X_k and the counter-based
// streams (jump_backward).  The cost term at t_k is the caller's.
template <typename R, int D, int DU, typename KH>
__device__ __forceinline__ void backward_checked(const KParams<R, D, DU> &kp, const KH &kh, int k, uint32_t m,
                                                 bool maybe, bool jumped, bool logged, const R (&xk)[D],
                                                 const R *__restrict__ u, R (&mu)[D], R (&g)[DU],
                                                 LogReader2<R, D> &lr) {
  if (jumped && !logged) {
    R xl[D], ml[D], gl[DU], tl[D + 2], ul[DU];
#pragma unroll
    for (int c = 0; c < D; ++c) { xl[c] = xk[c]; ml[c] = mu[c]; }
#pragma unroll
    for (int l = 0; l < DU; ++l) { gl[l] = R(0); ul[l] = __ldg(u + (size_t)k * DU + l); }
#pragma unroll
    for (int t = 0; t < D + 2; ++t) tl[t] = R(0);
    jump_backward<R, D, DU, false>(kp, k, m, xl, ul, ml, gl, tl);
#pragma unroll
    for (int c = 0; c < D; ++c) mu[c] = ml[c];
#pragma unroll
    for (int l = 0; l < DU; ++l) g[l] = gl[l];
  } else {
    backward_logged(kh, xk, mu, g, lr, maybe, jumped);
  }
}

// ---------------------------------------------------------------------------
// Paired sweeps are compiled for d <= 4 (the host's pairs_built rule).
template <int D>
constexpr bool PAIR_SWEEPS = D <= 4;

// Outputs of the second control of a paired sweep (PAIR): its control, cost partials,
// stored states or checkpoints and jump-log states.  The jump flags and log counts are
// the same for both controls and are written once.
template <typename R, int D>
struct PairOut {
  const R *u;
  double *partC;
  R *traj;
  R *ckpt;
  JLog<R, D> jl;
};

// Store mode: the first SV - 1 states of the current group ride in registers (buf) and
// the group leaves as VD 16-byte vectors (traj_shape).  The last group may be partial
// (k == Nt); its unused positions are written as 0.
template <typename R, int D>
struct StageBuf {
  static constexpr int N = TS<R, D>::SV > 1 ? TS<R, D>::SV - 1 : 1;
  R v[N][D];
};

template <typename R, int D>
__device__ __forceinline__ void stage_state(R *__restrict__ traj, int k, int Nt, int64_t mloc, int64_t lm,
                                            bool active, const R (&x)[D], StageBuf<R, D> &b) {
  constexpr int SV = TS<R, D>::SV, VD = TS<R, D>::VD, VW = TS<R, D>::VW;
  const int j = k % SV;
  if (j == SV - 1 || k == Nt) {
    if (active) {
#pragma unroll
      for (int v = 0; v < VD; ++v) {
        R o[VW];
#pragma unroll
        for (int w = 0; w < VW; ++w) {
          const int pos = v * VW + w, jj = pos / D, c = pos % D;
          if (jj == SV - 1)
            o[w] = j == jj ? x[c] : R(0);
          else
            o[w] = j == jj ? x[c] : (jj < j ? b.v[jj][c] : R(0));
        }
        Vec16<R>::store(traj + (((size_t)(k / SV) * VD + v) * mloc + lm) * VW, o);
      }
    }
  } else if constexpr (SV > 1) {
#pragma unroll
    for (int jj = 0; jj < SV - 1; ++jj)
#pragma unroll
      for (int c = 0; c < D; ++c) b.v[jj][c] = j == jj ? x[c] : b.v[jj][c];
  }
}

// Main-stream draws of every step of every path of a launch, taken in parallel (one thread
// per (step, path)): the Poisson word w[k][lm] and the normals z[k][c][lm] of main_draws,
// and for a step with exactly one jump its slot-0 draws s[k][.][lm] (slot0_draws).
template <typename R, int D, int DU>
__global__ void __launch_bounds__(256)
draws_kernel(const __grid_constant__ KParams<R, D, DU> kp, int64_t mloc, uint32_t *__restrict__ w,
             R *__restrict__ z, R *__restrict__ s, const unsigned long long *__restrict__ held,
             unsigned long long key) {
  if (*held == key) return;   // the buffers hold these draws already
  const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (i >= (int64_t)kp.Nt * mloc) return;
  const int k = (int)(i / mloc);
  const int64_t lm = i - (int64_t)k * mloc;
  const uint32_t m = (uint32_t)(kp.m_begin + lm);
  R zz[D];
  const uint32_t w0 = main_draws(kp, k, m, zz);
  w[i] = w0;
#pragma unroll
  for (int c = 0; c < D; ++c) z[((int64_t)k * D + c) * mloc + lm] = zz[c];
  if (has_jump(kp, w0) && one_jump(kp, w0)) {
    R xih[D], z1[D];
    R *sk = s + (int64_t)k * (1 + 2 * D) * mloc + lm;
    sk[0] = slot0_draws(kp, k, m, xih, z1);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      sk[(1 + c) * mloc] = xih[c];
      sk[(1 + D + c) * mloc] = z1[c];
    }
  }
}

template <typename R, int D>
struct PreDraws {
  const uint32_t *w;   // [Nt][mloc] Poisson words
  const R *z;          // [Nt][D][mloc] sub-step 0 normals
  const R *s;          // [Nt][1 + 2D][mloc] a step with exactly one (additive) jump: its
                       // slot-0 draws (time fraction, unit size, next normals); else unset
  Pair<R> *cw, *cw2;   // [mloc] each path's cost pair (first, second control)
  unsigned long long *held, key;   // the sweep records that the buffers hold the draws of key
};

// A step with one jump, its slot draws pre-drawn: sub-step to the jump, jump, sub-step.
template <typename R, int D, int DU, typename LW>
__device__ __forceinline__ void one_jump_pre(const KParams<R, D, DU> &kp, int k, const R *__restrict__ sk,
                                             int64_t mloc, const R (&z)[D], const R (&uk)[DU], R (&x)[D], LW &lw) {
  R xih[D], z1[D];
  const R th = sk[0];
#pragma unroll
  for (int c = 0; c < D; ++c) {
    xih[c] = sk[(1 + c) * mloc];
    z1[c] = sk[(1 + D + c) * mloc];
  }
  one_jump_inline(kp, k, th, xih, z, z1, uk, x, lw);
}

// PRE: the main-stream draws come from draws_kernel (PreDraws) instead of the step's own
// Philox and Box-Muller; the same values, so the same bits.
// fwd_body: the sweep of block bid of a launch over mloc paths (fwd_kernel: bid =
// blockIdx.x; fwd_batch_kernel: the block's index within its problem).
// With PRE the launch has one warp per block with SPREAD_LANES paths (the other lanes
// leave at once): a small problem's few paths spread over many SMs and warp schedulers,
// each warp carrying few lanes (an FP64 warp instruction of this part occupies its
// scheduler's FP64 pipe for many cycles).  Each path leaves its cost pair in pd.cw, and
// spread_combine_kernel forms every 128-path block's cost partial from them exactly as
// block_sum_to_double does in the one-path-per-thread launch.
// RK: kp is the launch's __grid_constant__ parameter, whose Philox round keys the draws
// take as constant operands (fwd_kernel); the batched sweeps' kp lies in a table.
template <typename R, int D, int DU, int MODE, bool PAIR = false, bool PRE = false, bool RK = false>
__device__ __forceinline__ void fwd_body(const KParams<R, D, DU> &kp, int64_t bid, const R *__restrict__ u,
                                         const R *__restrict__ xd, double *__restrict__ partC, R *__restrict__ traj,
                                         uint32_t *__restrict__ flags, R *__restrict__ ckpt, R *__restrict__ pcost,
                                         const JLog<R, D> &jl, int *__restrict__ jcnt, int64_t mloc,
                                         const PairOut<R, D> &p2, const PreDraws<R, D> &pd, Pair<R> *red) {
  if (PRE && threadIdx.x >= SPREAD_LANES) return;   // no warp-wide operation follows in this mode
  const int64_t lm = PRE ? bid * SPREAD_LANES + threadIdx.x : bid * TPB + threadIdx.x;
  const bool active = lm < mloc;
  const uint32_t m = (uint32_t)(kp.m_begin + lm);
  const int Nt = kp.Nt;
  R x[D], x2[D];
#pragma unroll
  for (int c = 0; c < D; ++c) x[c] = x2[c] = kp.x0[c];
  Kahan<R> cost, cost2;
  uint32_t fw = 0;
  using LW = typename std::conditional<MODE == FWD_STORE, LogWriter<R, D>, NoLog>::type;
  LW lw, lw2;
  if constexpr (MODE == FWD_STORE) {
    lw.L = jl;
    lw.idx = lm;
    if (!active) lw.L.cap = 0;   // inactive threads log nothing
    if constexpr (PAIR) {
      lw2.L = p2.jl;
      lw2.idx = lm;
      if (!active) lw2.L.cap = 0;
    }
  }
  constexpr bool PIN = pin_coef<D>();
  using KH = typename std::conditional<PIN, HotFwd<R, D, DU>, KParams<R, D, DU>>::type;
  HotFwd<R, D, DU> khv;
  if constexpr (PIN) khv = hot_fwd(kp);
  const KH &kh = coef_src<PIN>(kp, khv);
  // the loop of the single store and cost sweeps is not unrolled, which keeps the step's
  // code small (unrolled twice they ran slower); for d <= 2 the pair and checkpoint
  // sweeps' loops are unrolled twice (faster, measured; at d = 4 the unrolled pair sweep
  // took twice as long)
  StageBuf<R, D> sb, sb2;
#pragma unroll
  for (int i = 0; i < StageBuf<R, D>::N; ++i)
#pragma unroll
    for (int c = 0; c < D; ++c) sb.v[i][c] = sb2.v[i][c] = R(0);
  constexpr int UNR = ((PAIR || MODE == FWD_CKPT) && D <= 2) ? 2 : 1;
#pragma unroll UNR
  for (int k = 0; k <= Nt; ++k) {
    if (MODE == FWD_STORE) {
      stage_state<R, D>(traj, k, Nt, mloc, lm, active, x, sb);
      if constexpr (PAIR) stage_state<R, D>(p2.traj, k, Nt, mloc, lm, active, x2, sb2);
    }
    if (k == Nt) break;
    if (MODE == FWD_CKPT && active && (k & (kp.S - 1)) == 0) {   // S is a power of two
#pragma unroll
      for (int c = 0; c < D; ++c) {
        ckpt[((size_t)(k / kp.S) * D + c) * mloc + lm] = x[c];
        if constexpr (PAIR) p2.ckpt[((size_t)(k / kp.S) * D + c) * mloc + lm] = x2[c];
      }
    }
    int nj;
    if constexpr (PRE) {   // inactive threads read path 0's draws
      const int64_t lmc = active ? lm : 0, ik = (int64_t)k * mloc + lmc;
      const uint32_t w0 = pd.w[ik];
      R z[D];
#pragma unroll
      for (int c = 0; c < D; ++c) z[c] = pd.z[((int64_t)k * D + c) * mloc + lmc];
      const R *sk = pd.s + (int64_t)k * (1 + 2 * D) * mloc + lmc;
      R uk[DU];
#pragma unroll
      for (int l = 0; l < DU; ++l) uk[l] = __ldg(u + (size_t)k * DU + l);
      if (has_jump(kp, w0) && one_jump(kp, w0)) {   // the common jump step, pre-drawn
        one_jump_pre(kp, k, sk, mloc, z, uk, x, lw);
        if constexpr (PAIR) {
          R uk2[DU];
#pragma unroll
          for (int l = 0; l < DU; ++l) uk2[l] = __ldg(p2.u + (size_t)k * DU + l);
          one_jump_pre(kp, k, sk, mloc, z, uk2, x2, lw2);
        }
        nj = 1;
      } else if constexpr (PAIR) {
        nj = forward_step2<R, D, DU, LW, KH, RK>(kp, kh, k, m, w0, z, u, x, lw, p2.u, x2, lw2);
      } else {
        nj = step_from_draws<R, D, DU, LW, true, KH, RK>(kp, kh, k, m, w0, z, uk, x, lw);
      }
    } else if constexpr (PAIR) {
      R z[D];
      const uint32_t w0 = main_draws<RK>(kp, k, m, z);
      nj = forward_step2<R, D, DU, LW, KH, RK>(kp, kh, k, m, w0, z, u, x, lw, p2.u, x2, lw2);
    } else {
      nj = forward_step_h<R, D, DU, LW, false, true, KH, RK>(kp, kh, k, m, u, x, lw);
    }
    if (nj) fw |= 1u << (k & 31);
    cost.add(cost_term(kh, x, xd + (size_t)(k + 1) * D));
    if constexpr (PAIR) cost2.add(cost_term(kh, x2, xd + (size_t)(k + 1) * D));
    if (MODE == FWD_STORE && ((k & 31) == 31 || k == Nt - 1)) {
      if (active && (!PRE || flags)) flags[(size_t)(k >> 5) * mloc + lm] = fw;
      fw = 0;
    }
  }
  if constexpr (MODE == FWD_STORE) {
    if (active && (!PRE || jcnt)) {   // the same count and closing step for the second control
      jcnt[lm] = lw.r;
      jcnt[mloc + lm] = min(lw.kovf, Nt);
    }
  }
  if (MODE == FWD_CKPT && active) {
    const int nseg = (Nt + kp.S - 1) / kp.S;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      ckpt[((size_t)nseg * D + c) * mloc + lm] = x[c];
      if constexpr (PAIR) p2.ckpt[((size_t)nseg * D + c) * mloc + lm] = x2[c];
    }
  }
  Pair<R> v = cost.pair();
  if (!active) v = {R(0), R(0)};
  if (pcost && active) pcost[lm] = Ar<R>::add(v.s, v.e);
  if constexpr (PRE) {   // the path's pair; spread_combine_kernel sums them
    if (bid == 0 && threadIdx.x == 0) *pd.held = pd.key;   // the draws kernel has completed
    if (active) pd.cw[lm] = v;
    if constexpr (PAIR) {
      if (active) pd.cw2[lm] = cost2.pair();
    }
  } else {
    const double s = block_sum_to_double(v, red);
    if (threadIdx.x == 0) partC[bid] = s;
    if constexpr (PAIR) {
      Pair<R> v2 = cost2.pair();
      if (!active) v2 = {R(0), R(0)};
      const double s2 = block_sum_to_double(v2, red);
      if (threadIdx.x == 0) p2.partC[bid] = s2;
    }
  }
}

// The cost partials of a spread sweep: block b of TPB threads takes the pairs of paths
// b TPB .. b TPB + TPB - 1 (the zero pair past mloc, as an idle thread of the sweep has) and
// sums them with block_sum_to_double, so partC[b] is the one-path-per-thread sweep's.
template <typename R>
__global__ void __launch_bounds__(TPB) spread_combine_kernel(const Pair<R> *__restrict__ cw,
                                                             const Pair<R> *__restrict__ cw2, int64_t mloc,
                                                             double *__restrict__ partC,
                                                             double *__restrict__ partC2) {
  __shared__ Pair<R> red[TPB / 32];
  const int64_t lm = (int64_t)blockIdx.x * TPB + threadIdx.x;
  for (int h = 0; h < (cw2 ? 2 : 1); ++h) {
    const Pair<R> *w = h ? cw2 : cw;
    const Pair<R> v = lm < mloc ? w[lm] : Pair<R>{R(0), R(0)};
    const double s = block_sum_to_double(v, red);
    if (threadIdx.x == 0) (h ? partC2 : partC)[blockIdx.x] = s;
  }
}

template <typename R, int D, int DU, int MODE, bool PAIR = false, bool PRE = false>
__global__ void __launch_bounds__(TPB)
fwd_kernel(const __grid_constant__ KParams<R, D, DU> kp, const R *__restrict__ u,
           const R *__restrict__ xd, double *__restrict__ partC, R *__restrict__ traj,
           uint32_t *__restrict__ flags, R *__restrict__ ckpt, R *__restrict__ pcost,
           JLog<R, D> jl, int *__restrict__ jcnt, int64_t mloc, PairOut<R, D> p2, PreDraws<R, D> pd = {}) {
  __shared__ Pair<R> red[TPB / 32];
  // the round keys of kp in the draws: the paired, checkpoint and cost sweeps run faster
  // with them; the single store sweep's register allocation did not (288.7 -> 298.4
  // warp-instructions per warp-step, 9.75 -> 9.97 ms per launch at M = 2^20, N_t = 1000)
  constexpr bool RK = !(MODE == FWD_STORE && !PAIR);
  if constexpr (PAIR && PRE) {
    // a pre-drawn pair: each control on its own warps (the first half of the blocks, then
    // the second), each a single sweep -- the pair sweep's per-control arithmetic; the
    // flags and log counts (the same for both) from the first control
    const unsigned nb = gridDim.x / 2;
    const bool second = blockIdx.x >= nb;
    PreDraws<R, D> pd1 = pd;
    if (second) pd1.cw = pd.cw2;
    fwd_body<R, D, DU, MODE, false, true, RK>(kp, second ? blockIdx.x - nb : blockIdx.x, second ? p2.u : u, xd, partC,
                                          second ? p2.traj : traj, second ? nullptr : flags,
                                          second ? p2.ckpt : ckpt, nullptr, second ? p2.jl : jl,
                                          second ? nullptr : jcnt, mloc, PairOut<R, D>{}, pd1, red);
  } else {
    fwd_body<R, D, DU, MODE, PAIR, PRE, RK>(kp, blockIdx.x, u, xd, partC, traj, flags, ckpt, pcost, jl, jcnt, mloc,
                                            p2, pd, red);
  }
}

// X_k of one path from the stored trajectory.
template <typename R, int D>
__device__ __forceinline__ void load_state(const R *__restrict__ traj, int k, int64_t mloc,
                                           int64_t lm, R (&x)[D]) {
  constexpr int SV = TS<R, D>::SV, VD = TS<R, D>::VD, VW = TS<R, D>::VW;
  const int g = k / SV, j = k % SV;
#pragma unroll
  for (int v = 0; v < VD; ++v) {
    R o[VW];
    Vec16<R>::load(traj + (((size_t)g * VD + v) * mloc + lm) * VW, o);
#pragma unroll
    for (int w = 0; w < VW; ++w) {
      const int pos = v * VW + w;
      if (pos / D == j) x[pos % D] = o[w];
    }
  }
}

// Steps per chunk of the stored adjoint (CH), and the 16-byte vectors per thread and
// chunk (NV): a chunk's states are staged in shared memory by cp.async one chunk ahead
// of their use (two stages), so the loads in flight cost no registers.
template <typename R, int D>
struct AdjChunk {
  static constexpr int CH = D <= 2 ? 8 : 4;
  static constexpr int NV = CH / TS<R, D>::SV * TS<R, D>::VD;
};

// Stage bytes per block: the states (NV vectors per thread) and, per warp, the chunk's
// target rows x_d(t_k) (XB bytes, copied by the first XB / 16 lanes), both twice.
template <typename R, int D>
struct AdjStage {
  static constexpr int XB = AdjChunk<R, D>::CH * D * (int)sizeof(R);
  static constexpr size_t STATES = (size_t)2 * AdjChunk<R, D>::NV * TPB * 16;
  static constexpr size_t BYTES = STATES + (size_t)2 * (TPB / 32) * XB;
  static_assert(XB % 16 == 0, "target rows of a chunk in 16-byte copies");
};
template <typename R, int D>
__host__ __device__ constexpr size_t adj_stage_bytes() {   // per block
  return AdjStage<R, D>::BYTES;
}

// Issue the copies of the states of steps c CH .. c CH + CH - 1 into stage st (groups
// past the last one are read as the last group: those steps lie beyond N_t and are never
// used) and, when the rows exist (steps below N_t), the warp's copy of the chunk's target
// rows; then commit them as one group.
template <typename R, int D>
__device__ __forceinline__ void issue_chunk(const R *__restrict__ traj, const R *__restrict__ xd, int c, int ng,
                                            int Nt, int64_t mloc, int64_t lm, unsigned char *stage, int st) {
  constexpr int CH = AdjChunk<R, D>::CH, NV = AdjChunk<R, D>::NV, XB = AdjStage<R, D>::XB;
  constexpr int SV = TS<R, D>::SV, VD = TS<R, D>::VD, VW = TS<R, D>::VW;
  static_assert(CH % SV == 0 && 16 % CH == 0, "chunk geometry");
#pragma unroll
  for (int gi = 0; gi < CH / SV; ++gi) {
    const int g = min(c * (CH / SV) + gi, ng - 1);
#pragma unroll
    for (int v = 0; v < VD; ++v)
      cp_async16(stage + (((size_t)st * NV + gi * VD + v) * TPB + threadIdx.x) * 16,
                 traj + (((size_t)g * VD + v) * mloc + lm) * VW);
  }
  const int lane = threadIdx.x & 31;
  if (lane < XB / 16 && c * CH + CH <= Nt)
    cp_async16(stage + AdjStage<R, D>::STATES + ((size_t)st * (TPB / 32) + (threadIdx.x >> 5)) * XB + lane * 16,
               reinterpret_cast<const unsigned char *>(xd + (size_t)c * CH * D) + lane * 16);
  cp_async_commit();
}

// The state X_k of step j of the chunk in stage st (the components of a step are adjacent
// within their vectors).
template <typename R, int D>
__device__ __forceinline__ void stage_step(const unsigned char *stage, int st, int j, R (&x)[D]) {
  constexpr int NV = AdjChunk<R, D>::NV, SV = TS<R, D>::SV, VD = TS<R, D>::VD;
  const unsigned char *base = stage + (((size_t)st * NV + (j / SV) * VD) * TPB + threadIdx.x) * 16;
  if constexpr (D * sizeof(R) == 4) {
    x[0] = reinterpret_cast<const R *>(base)[j % SV];
  } else if constexpr (D * sizeof(R) == 8 && sizeof(R) == 4) {
    const float2 t = reinterpret_cast<const float2 *>(base)[j % SV];
    x[0] = t.x;
    x[1] = t.y;
  } else if constexpr (D * sizeof(R) == 8) {
    x[0] = reinterpret_cast<const R *>(base)[j % SV];
  } else {
#pragma unroll
    for (int v = 0; v < VD; ++v) {
      if constexpr (sizeof(R) == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(base + (size_t)v * TPB * 16);
        x[4 * v] = t.x; x[4 * v + 1] = t.y; x[4 * v + 2] = t.z; x[4 * v + 3] = t.w;
      } else {
        const double2 t = *reinterpret_cast<const double2 *>(base + (size_t)v * TPB * 16);
        x[2 * v] = t.x; x[2 * v + 1] = t.y;
      }
    }
  }
}

// The warp's staged target rows of the chunk in stage st.
template <typename R, int D>
__device__ __forceinline__ const R *staged_rows(const unsigned char *stage, int st) {
  return reinterpret_cast<const R *>(stage + AdjStage<R, D>::STATES +
                                     ((size_t)st * (TPB / 32) + (threadIdx.x >> 5)) * AdjStage<R, D>::XB);
}

template <typename R, int D, int DU, bool THETA>
__device__ __forceinline__ void finish_theta(const KParams<R, D, DU> &kp, R (&th)[D + 2], bool active,
                                             double *__restrict__ partT, Pair<R> *red, int64_t bid) {
  if constexpr (THETA) {
    // unrolled: a runtime index into th would keep the accumulators in local memory
#pragma unroll
  for (int t = 0; t < D + 2; ++t) {
    Pair<R> v = {active ? th[t] : R(0), R(0)};
    const double s = block_sum_to_double(v, red);
    if (threadIdx.x == 0) partT[(size_t)t * kp.nblk + bid] = s;
  }
  }
}

// Stored adjoint.  The states arrive in chunks of CH steps, staged in shared memory one
// chunk ahead; every step's contribution B^T lambda' delta goes to the warp's gradient
// rows, reduced every 16 steps (GradRows).  A chunk runs the fast form when no lane of the
// warp meets a step the jump log does not cover (the log is a prefix of the path's jump
// steps, jcnt[mloc + m]): steps without jumps and logged jump steps in one code path, with
// a warp-uniform test per step (the OR of the chunk's jump flags over the warp) before the
// log is consulted.  Other chunks (the first and the last, a closed log, the parameter
// gradients, the adjoint-state output) check every step's flag and regenerate what the
// log does not hold.
// LAM: write the adjoint states to lam_out (jd_sample_paths); a compile-time switch, since
// a run-time test leaves its stores and their address arithmetic in every step.
// CUB: the drift family as a compile-time constant (0, 1) for the pinned coefficients of
// d <= 2, or read at run time (-1).
// Dynamic shared memory: grad_rows_bytes<R, DU, 16>() + adj_stage_bytes<R, D>().
template <typename R, int D, int DU, bool THETA, bool LAM, int CUB>
__device__ __forceinline__ void stored_sweep(const KParams<R, D, DU> &kp, const R *__restrict__ u,
                                             const R *__restrict__ xd, const R *__restrict__ traj,
                                             const uint32_t *__restrict__ flags, const JLog<R, D> &jl,
                                             const int *__restrict__ jcnt, double *__restrict__ partG,
                                             double *__restrict__ partT, R *__restrict__ lam_out, int64_t mloc,
                                             unsigned char *dsm, Pair<R> *red1, int64_t bid) {
  using M = Ar<R>;
  constexpr int CH = AdjChunk<R, D>::CH, SV = TS<R, D>::SV, NR = 16, LD = RowGeom<R>::LD;
  constexpr bool FAST = !THETA && !LAM, PIN = pin_coef<D>();
  GradRows<R, DU, NR> rows;
  rows.init(reinterpret_cast<R *>(dsm));
  unsigned char *stage = dsm + grad_rows_bytes<R, DU, NR>();
  const int64_t npart = kp.npart;
  const int64_t lm = bid * TPB + threadIdx.x;
  const bool active = lm < mloc;
  // inactive threads of the last block replay path 0 (its stored data and its random
  // streams must belong to the same path) and discard the result
  const int64_t lmc = active ? lm : 0;
  const uint32_t m = (uint32_t)(kp.m_begin + lmc);
  const int Nt = kp.Nt;
  const int ng = (Nt + SV) / SV;
  const int nch = (Nt + CH - 1) / CH;
  issue_chunk<R, D>(traj, xd, nch - 1, ng, Nt, mloc, lmc, stage, (nch - 1) & 1);
  // the parameter-gradient sweep regenerates every jump step (it needs the sub-steps'
  // normals), so it reads no log
  LogReader2<R, D> lr;
  lr.init(jl, lmc, THETA ? 0 : min(__ldg(jcnt + lmc), jl.cap));
  const int kovf = THETA ? 0 : __ldg(jcnt + mloc + lmc);
  LogReader<R, D> lr0;   // an empty log for backward_step (parameter gradients)
  lr0.L = jl;
  lr0.idx = lmc;
  lr0.init(0);
  R mu[D], th[D + 2];
#pragma unroll
  for (int t = 0; t < D + 2; ++t) th[t] = R(0);
  {
    R x[D], xN[D];
    load_state<R, D>(traj, Nt, mloc, lmc, x);
    load_row<R, D>(xd + (size_t)Nt * D, xN);
#pragma unroll
    for (int c = 0; c < D; ++c) mu[c] = M::mul(kp.qdt[c], M::sub(x[c], xN[c]));
    if (LAM && active)
#pragma unroll
      for (int c = 0; c < D; ++c) lam_out[((size_t)Nt * D + c) * mloc + lm] = mu[c];
  }
  // pinned coefficients (d <= 2); the fast form zeroes B on inactive threads
  using KH = typename std::conditional<PIN, HotCoef<R, D, DU, CUB>, KParams<R, D, DU>>::type;
  HotCoef<R, D, DU, CUB> khv;
  if constexpr (PIN) khv = hot_coef<CUB>(kp, !FAST || active);
  const KH &kh = coef_src<PIN>(kp, khv);
  const int colw = GradRows<R, DU, NR>::col(threadIdx.x & 31);
  uint32_t fwn = __ldg(flags + (size_t)(((nch - 1) * CH) >> 5) * mloc + lmc);
#pragma unroll 1
  for (int c = nch - 1; c >= 0; --c) {
    const int k0 = c * CH;
    const uint32_t fw = fwn;
    if (c > 0) {
      issue_chunk<R, D>(traj, xd, c - 1, ng, Nt, mloc, lmc, stage, (c - 1) & 1);
      fwn = __ldg(flags + (size_t)((k0 - CH) >> 5) * mloc + lmc);
    } else {
      cp_async_commit();   // an empty group keeps the wait count uniform
    }
    cp_async_wait<1>();   // this chunk's copies (all groups but the newest) have landed
    __syncwarp();         // ... and the target rows that other lanes of the warp copied
    bool slow = true;
    if constexpr (FAST) slow = __any_sync(0xffffffffu, c == 0 || k0 + CH > Nt || k0 + CH > kovf);
    if (FAST && !slow) {
      // warp-uniform: bit j set when some lane of the warp has a jump at step k0 + j
      const uint32_t jw = __reduce_or_sync(0xffffffffu, (fw >> (k0 & 31)) & ((1u << CH) - 1u));
      const R *xdc = staged_rows<R, D>(stage, c & 1);
      R *rp = rows.w + (k0 & (NR - 1)) * LD + colw;
#pragma unroll
      for (int j = CH - 1; j >= 0; --j) {
        R g[DU], xk[D], xdk[D];
        stage_step<R, D>(stage, c & 1, j, xk);
#pragma unroll
        for (int cc = 0; cc < D; ++cc) xdk[cc] = xdc[j * D + cc];
        backward_logged(kh, xk, mu, g, lr, (jw >> j) & 1u, (fw >> ((k0 + j) & 31)) & 1u);
        cost_gradient(kh, xk, xdk, mu);
#pragma unroll
        for (int l = 0; l < DU; ++l) rp[(l * NR + j) * LD] = (PIN || active) ? g[l] : R(0);
      }
    } else {
      const uint32_t jw = __reduce_or_sync(0xffffffffu, (fw >> (k0 & 31)) & ((1u << CH) - 1u));
#pragma unroll 1
      for (int j = CH - 1; j >= 0; --j) {
        const int k = k0 + j;
        R g[DU];
#pragma unroll
        for (int l = 0; l < DU; ++l) g[l] = R(0);
        if (k < Nt) {
          R xk[D];
          stage_step<R, D>(stage, c & 1, j, xk);
          const bool jumped = (fw >> (k & 31)) & 1u;
          if constexpr (THETA) {
            backward_step<R, D, DU, true, LogReader<R, D>, false, KH>(kp, kh, k, m, jumped, xk, u, xd, mu, g, th,
                                                                      lr0);
          } else {
            backward_checked(kp, kh, k, m, (jw >> j) & 1u, jumped, k < kovf, xk, u, mu, g, lr);
            if (k >= 1) {
              R xdk[D];
              load_row<R, D>(xd + (size_t)k * D, xdk);
              cost_gradient(kh, xk, xdk, mu);
            }
          }
          if (LAM && active)
#pragma unroll
            for (int cc = 0; cc < D; ++cc) lam_out[((size_t)k * D + cc) * mloc + lm] = mu[cc];
        }
        rows.put(k & (NR - 1), g, active);
      }
    }
    if ((k0 & (NR - 1)) == 0) rows.flush(k0, Nt, partG, npart, bid);
  }
  finish_theta<R, D, DU, THETA>(kp, th, active, partT, red1, bid);
}

template <typename R, int D, int DU, bool THETA, bool LAM = false>
__global__ void __launch_bounds__(TPB)
adj_stored_kernel(const __grid_constant__ KParams<R, D, DU> kp, const R *__restrict__ u,
                  const R *__restrict__ xd, const R *__restrict__ traj,
                  const uint32_t *__restrict__ flags, JLog<R, D> jl, const int *__restrict__ jcnt,
                  double *__restrict__ partG, double *__restrict__ partT, R *__restrict__ lam_out,
                  int64_t mloc) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ Pair<R> red1[TPB / 32];
  if constexpr (pin_coef<D>() && !THETA && !LAM) {   // the drift family decided once
    if (kp.cubic)
      stored_sweep<R, D, DU, THETA, LAM, 1>(kp, u, xd, traj, flags, jl, jcnt, partG, partT, lam_out, mloc, dsm, red1,
                                            blockIdx.x);
    else
      stored_sweep<R, D, DU, THETA, LAM, 0>(kp, u, xd, traj, flags, jl, jcnt, partG, partT, lam_out, mloc, dsm, red1,
                                            blockIdx.x);
  } else {
    stored_sweep<R, D, DU, THETA, LAM, -1>(kp, u, xd, traj, flags, jl, jcnt, partG, partT, lam_out, mloc, dsm, red1,
                                           blockIdx.x);
  }
}

// Jump-log records per path and checkpoint segment in the recompute adjoint's shared
// memory (a segment whose jumps do not fit regenerates them).  Four records hold a
// 16-step segment's jumps except with probability below 1e-5 at lambda dt = 0.01.
template <int D>
__host__ __device__ constexpr int seg_log_cap() {
  return 4;
}


// The parameter-gradient variant of the recompute adjoint keeps each step's normals
// from the forward replay (instead of drawing them again) when the doubled segment
// buffer still leaves room for two or more blocks per SM.
template <typename R, int D, bool THETA>
__host__ __device__ constexpr bool recompute_zbuf() {
  return THETA && (size_t)seg_len<D>() * D * TPB * sizeof(R) * 2 +
                          (size_t)seg_log_cap<D>() * (2 + D) * TPB * sizeof(R) <= 100 * 1024;
}

// Recompute adjoint.  Per segment of S steps (a multiple of 8): replay the forward from
// the checkpoint into shared memory (states, a short jump log, and for the parameter
// gradients the main-stream normals), then sweep the segment backwards in chunks of 8
// steps, each in the fast form of the stored adjoint when no lane of the warp meets a
// jump step the segment's log does not hold.  Same step arithmetic and the same gradient
// tree as the stored adjoint (with 8-step rows, half the shared memory): the same bits.
template <typename R, int D, int DU, bool THETA>
__device__ __forceinline__ void adj_recompute_body(const KParams<R, D, DU> &kp, const R *__restrict__ u,
                                                   const R *__restrict__ xd, const R *__restrict__ ckpt,
                                                   double *__restrict__ partG, double *__restrict__ partT,
                                                   int64_t mloc) {
  using M = Ar<R>;
  constexpr int CH = 8;
  // the parameter-gradient backward regenerates every jump step (it needs the sub-steps'
  // normals), so its replay keeps no jump log: no shared log, more blocks per SM
  constexpr int JS = THETA ? 0 : seg_log_cap<D>();
  using LWR = typename std::conditional<THETA, NoLog, LogWriter<R, D>>::type;
  extern __shared__ __align__(16) unsigned char dsm[];
  constexpr bool ZBUF = recompute_zbuf<R, D, THETA>();
  R *sbuf = reinterpret_cast<R *>(dsm);   // [S * D][TPB] segment states
  const int S = kp.S;
  R *zbuf = sbuf + (size_t)S * D * TPB;   // ZBUF: [S * D][TPB] main-stream normals
  auto *skt = reinterpret_cast<typename V2<R>::T *>(zbuf + (ZBUF ? (size_t)S * D * TPB : 0));   // [JS][TPB]
  R *sy = reinterpret_cast<R *>(skt + JS * TPB);                                    // [JS * D][TPB]
  constexpr int NR = 8;
  GradRows<R, DU, NR> rows;
  rows.init(sy + (size_t)JS * D * TPB);
  __shared__ Pair<R> red1[TPB / 32];
  const int64_t npart = kp.npart;
  const int64_t lm = (int64_t)blockIdx.x * TPB + threadIdx.x;
  const bool active = lm < mloc;
  const int64_t lmc = active ? lm : 0;   // inactive threads replay path 0
  const uint32_t m = (uint32_t)(kp.m_begin + lmc);
  const int Nt = kp.Nt, tid = threadIdx.x;
  const int nseg = (Nt + S - 1) / S;
  const JLog<R, D> sl{skt, sy, TPB, JS};
  R mu[D], th[D + 2];
#pragma unroll
  for (int t = 0; t < D + 2; ++t) th[t] = R(0);
  {
    R xN[D];
    load_row<R, D>(xd + (size_t)Nt * D, xN);
#pragma unroll
    for (int c = 0; c < D; ++c)
      mu[c] = M::mul(kp.qdt[c], M::sub(__ldg(ckpt + ((size_t)nseg * D + c) * mloc + lmc), xN[c]));
  }
#pragma unroll 1
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int k0 = seg * S, len = min(S, Nt - k0);
    R x[D];
#pragma unroll
    for (int c = 0; c < D; ++c) x[c] = __ldg(ckpt + ((size_t)seg * D + c) * mloc + lmc);
    uint64_t jm = 0;   // bit i: step k0 + i had a jump (S <= 64)
    LWR lw;
    if constexpr (!THETA) {
      lw.L = sl;
      lw.idx = tid;
    }
#pragma unroll 1
    for (int i = 0; i < len; ++i) {
#pragma unroll
      for (int c = 0; c < D; ++c) sbuf[(i * D + c) * TPB + tid] = x[c];
      if (forward_step<R, D, DU, LWR, ZBUF, !THETA>(kp, k0 + i, m, u, x, lw, zbuf + (size_t)i * D * TPB + tid,
                                                    TPB))
        jm |= 1ull << i;
    }
    LogReader2<R, D> lr;
    int kovf = 0;
    if constexpr (THETA) {
      lr.init(sl, tid, 0);
    } else {
      lr.init(sl, tid, lw.r);
      kovf = lw.kovf;
    }
    LogReader<R, D> lr0;   // an empty log for backward_step (parameter gradients)
    lr0.L = sl;
    lr0.idx = tid;
    lr0.init(0);
    const int nch = (len + CH - 1) / CH;
#pragma unroll 1
    for (int cc = nch - 1; cc >= 0; --cc) {
      const int i0 = cc * CH;
      bool slow = true;
      if constexpr (!THETA) slow = __any_sync(0xffffffffu, k0 + i0 == 0 || i0 + CH > len || k0 + i0 + CH > kovf);
      // warp-uniform: bit j set when some lane of the warp has a jump at step k0 + i0 + j
      const uint32_t jwm = __reduce_or_sync(0xffffffffu, (jm >> i0) & ((1u << CH) - 1u));
      if (!THETA && !slow) {
        const R *xdc = xd + (size_t)(k0 + i0) * D;
        // rolled (the states come from shared memory anyway; measured faster than unrolled)
#pragma unroll 1
        for (int j = CH - 1; j >= 0; --j) {
          const int i = i0 + j;
          R g[DU], xk[D], xdk[D];
#pragma unroll
          for (int c = 0; c < D; ++c) xk[c] = sbuf[(i * D + c) * TPB + tid];
          load_row<R, D>(xdc + j * D, xdk);
          backward_logged(kp, xk, mu, g, lr, (jwm >> j) & 1u, (jm >> i) & 1u);
          cost_gradient(kp, xk, xdk, mu);
          rows.put((k0 + i) & (NR - 1), g, active);
        }
      } else {
        // rolled (the parameter-gradient step is large and these chunks are rare)
#pragma unroll 1
        for (int j = CH - 1; j >= 0; --j) {
          const int i = i0 + j, k = k0 + i;
          R g[DU];
#pragma unroll
          for (int l = 0; l < DU; ++l) g[l] = R(0);
          if (i < len) {
            R xk[D];
#pragma unroll
            for (int c = 0; c < D; ++c) xk[c] = sbuf[(i * D + c) * TPB + tid];
            const bool jumped = (jm >> i) & 1u;
            if constexpr (THETA) {
              backward_step<R, D, DU, true, LogReader<R, D>, ZBUF>(kp, kp, k, m, jumped, xk, u, xd, mu, g, th, lr0,
                                                                   zbuf + (size_t)i * D * TPB + tid, TPB);
            } else {
              backward_checked(kp, kp, k, m, (jwm >> j) & 1u, jumped, k < kovf, xk, u, mu, g, lr);
              if (k >= 1) {
                R xdk[D];
                load_row<R, D>(xd + (size_t)k * D, xdk);
                cost_gradient(kp, xk, xdk, mu);
              }
            }
          }
          rows.put(k & (NR - 1), g, active);
        }
      }
      if (((k0 + i0) & (NR - 1)) == 0) rows.flush(k0 + i0, Nt, partG, npart, blockIdx.x);
    }
  }
  finish_theta<R, D, DU, THETA>(kp, th, active, partT, red1, blockIdx.x);
}

template <typename R, int D, int DU, bool THETA>
__global__ void __launch_bounds__(TPB)
adj_recompute_kernel(const __grid_constant__ KParams<R, D, DU> kp, const R *__restrict__ u,
                     const R *__restrict__ xd, const R *__restrict__ ckpt,
                     double *__restrict__ partG, double *__restrict__ partT, int64_t mloc) {
  adj_recompute_body<R, D, DU, THETA>(kp, u, xd, ckpt, partG, partT, mloc);
}

// The parameter-gradient form for FP32 d <= 2 with at least 5 blocks per SM: the default
// allocation took 80 registers and spilled; 94 registers without spills run 20.4 -> 17.7
// ms per launch at M = 2^20, N_t = 1024 (the u-gradient form keeps its own allocation).
template <typename R, int D, int DU>
__global__ void __launch_bounds__(TPB, 5)
adj_recompute_theta5_kernel(const __grid_constant__ KParams<R, D, DU> kp, const R *__restrict__ u,
                            const R *__restrict__ xd, const R *__restrict__ ckpt,
                            double *__restrict__ partG, double *__restrict__ partT, int64_t mloc) {
  adj_recompute_body<R, D, DU, true>(kp, u, xd, ckpt, partG, partT, mloc);
}

template <typename R, int D>
constexpr bool theta5() {
  return sizeof(R) == 4 && D <= 2;
}

// The parameter-gradient recompute kernel an instantiation launches.
template <typename R, int D, int DU>
const void *theta_recompute_fn() {
  if constexpr (theta5<R, D>())
    return (const void *)adj_recompute_theta5_kernel<R, D, DU>;
  else
    return (const void *)adj_recompute_kernel<R, D, DU, true>;
}

// ---------------------------------------------------------------------------
// Host-side launch ops for one (precision, D, DU)
// ---------------------------------------------------------------------------
// Poisson thresholds floor(2^32 F(n; mu)) with the pmf accumulated in order
// p_0 = exp(-mu), p_n = p_{n-1} mu / n; clamped to [0, 2^32].
inline void poisson_thresholds(double mu, unsigned long long *thr) {
  double pn = std::exp(-mu), F = pn;
  for (int n = 0; n < NMAX; ++n) {
    if (n > 0) {
      pn = pn * mu / (double)n;
      F = F + pn;
    }
    double t = std::floor(F * 4294967296.0);
    t = t < 0.0 ? 0.0 : (t > 4294967296.0 ? 4294967296.0 : t);
    thr[n] = (unsigned long long)t;
  }
}

// The generator's key (seed mod 2^32, seed >> 32) and its ten round keys.
template <typename R, int D, int DU>
void set_philox_key(KParams<R, D, DU> &kp, unsigned long long seed) {
  kp.key0 = (uint32_t)(seed & 0xffffffffull);
  kp.key1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    kp.rk0[r] = kp.key0 + (uint32_t)r * 0x9E3779B9u;
    kp.rk1[r] = kp.key1 + (uint32_t)r * 0xBB67AE85u;
  }
}

template <typename R, int D, int DU>
void make_kparams(const jd_problem *p, int64_t m_begin, int64_t mloc, KParams<R, D, DU> &kp) {
  const jd_problem_desc &q = p->desc;
  const int d = q.d, du = q.du;
  const double dt = q.T / (double)q.Nt, sqdt = std::sqrt(dt);
  for (int i = 0; i < D * D; ++i) kp.A[i] = kp.C[i] = kp.dA[i] = R(0);
  for (int i = 0; i < D * DU; ++i) kp.B[i] = R(0);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      kp.A[i * D + j] = (R)p->A[(size_t)i * d + j];
      if (q.drift == JD_DRIFT_CUBIC) kp.C[i * D + j] = (R)p->C[(size_t)i * d + j];
      if (!p->dA.empty()) kp.dA[i * D + j] = (R)p->dA[(size_t)i * d + j];
    }
  for (int i = 0; i < d; ++i)
    for (int l = 0; l < du; ++l) kp.B[i * DU + l] = (R)p->B[(size_t)i * du + l];
  for (int c = 0; c < D; ++c) {
    const bool in = c < d;
    kp.sigma[c] = in ? (R)p->sigma[c] : R(0);
    kp.sig_sqdt[c] = in ? (R)(p->sigma[c] * sqdt) : R(0);
    kp.qdt[c] = in ? (R)(p->q[c] * dt) : R(0);
    kp.hqdt[c] = in ? (R)(0.5 * p->q[c] * dt) : R(0);
    kp.x0[c] = in ? (R)p->x0[c] : R(0);
    const bool reset = q.jump_law == JD_JUMP_KS && c >= d / 2, moved = q.jump_law != JD_JUMP_KS || reset;
    kp.jgain[c] = reset ? (R)q.jump_gain : R(1);
    kp.jscl[c] = moved ? (R)q.jump_scale : R(0);
  }
  kp.dt = (R)dt;
  kp.sqdt = (R)sqdt;
  kp.jump_scale = (R)q.jump_scale;
  kp.kvel = q.jump_law == JD_JUMP_KS ? d / 2 : 0;
  poisson_thresholds(q.lambda * dt, kp.thr);
  set_philox_key(kp, q.seed);
  kp.epoch = q.epoch;
  kp.d = d;
  kp.npair = (d + 1) / 2;
  kp.Nt = q.Nt;
  kp.cubic = q.drift == JD_DRIFT_CUBIC;
  kp.jump_law = (int)q.jump_law;
  kp.jumps_on = q.jump_law != JD_JUMP_NONE && q.lambda > 0.0;
  kp.has_dA = !p->dA.empty();
  kp.S = p->S;   // checkpoint spacing of the recompute plan (a power of two, 16 .. 64)
  kp.nblk = (int)ceil_div(mloc, TPB);
  kp.m_begin = q.m_offset + m_begin;   // global path index (a shard starts at m_offset)
  kp.npart = grad_parts(mloc);
}

// Key of the pre-drawn draws of a launch: everything they depend on (the generator's key
// and epoch, the first path and the path count, N_t, d, the jump law and its Poisson
// thresholds), mixed into 64 bits; never 0 (the key of empty buffers).
template <typename R, int D, int DU>
unsigned long long draws_key(const KParams<R, D, DU> &kp, int64_t mloc) {
  unsigned long long h = 0x9e3779b97f4a7c15ull;
  auto mix = [&h](unsigned long long v) {
    h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
  };
  mix(kp.key0);
  mix(kp.key1);
  mix(kp.epoch);
  mix((unsigned long long)kp.m_begin);
  mix((unsigned long long)mloc);
  mix((unsigned long long)kp.Nt);
  mix((unsigned long long)kp.d);
  mix((unsigned long long)kp.jump_law);
  mix((unsigned long long)kp.jumps_on);
  for (int n = 0; n < NMAX; ++n) mix(kp.thr[n]);
  return h | 1ull;
}

template <typename R, int D, int DU>
cudaError_t op_fwd(const jd_problem *p, int mode, int64_t m_begin, int64_t mloc, const void *uk,
                   const PathBufs &b, cudaStream_t s) {
  KParams<R, D, DU> kp;   // passed by value to the kernel (copied at the launch)
  make_kparams<R, D, DU>(p, m_begin, mloc, kp);
  if (b.npart) kp.npart = b.npart;
  const dim3 grid((unsigned)ceil_div(mloc, TPB));
  const R *u = static_cast<const R *>(uk);
  const R *xd = static_cast<const R *>(p->xdk);
  R *pc = static_cast<R *>(b.pcost);
  const JLog<R, D> jl{static_cast<typename V2<R>::T *>(b.log_kt), static_cast<R *>(b.log_y), mloc, b.log_cap};
  PairOut<R, D> p2{};
  if (mode & FWD_PAIR)
    p2 = PairOut<R, D>{static_cast<const R *>(b.uk2), b.partC2, static_cast<R *>(b.traj2), static_cast<R *>(b.ckpt2),
                       JLog<R, D>{static_cast<typename V2<R>::T *>(b.log_kt2), static_cast<R *>(b.log_y2), mloc,
                                  b.log_cap}};
  if constexpr (D <= 2) {
    if (b.pre_w) {   // a small problem: all main-stream draws in one parallel pass first
      R *pz = static_cast<R *>(b.pre_z), *ps = pz + (size_t)kp.Nt * D * mloc;
      Pair<R> *cw = reinterpret_cast<Pair<R> *>(ps + (size_t)kp.Nt * (1 + 2 * D) * mloc);
      const unsigned long long key = draws_key(kp, mloc);
      draws_kernel<R, D, DU><<<(unsigned)ceil_div((int64_t)kp.Nt * mloc, 256), 256, 0, s>>>(
          kp, mloc, b.pre_w, pz, ps, b.pre_key, key);
      count_launch();
      const PreDraws<R, D> pd{b.pre_w, pz, ps, cw, cw + mloc, b.pre_key, key};
      // blocks of one warp with SPREAD_LANES paths; a pair's controls on separate blocks
      const dim3 sgrid((unsigned)(ceil_div(mloc, SPREAD_LANES) * ((mode & FWD_PAIR) ? 2 : 1)));
      switch (mode) {
        case FWD_COST:
          fwd_kernel<R, D, DU, FWD_COST, false, true><<<sgrid, SPREAD_TPB, 0, s>>>(
              kp, u, xd, b.partC, nullptr, nullptr, nullptr, pc, jl, nullptr, mloc, p2, pd);
          break;
        case FWD_STORE:
          fwd_kernel<R, D, DU, FWD_STORE, false, true><<<sgrid, SPREAD_TPB, 0, s>>>(
              kp, u, xd, b.partC, static_cast<R *>(b.traj), b.flags, nullptr, pc, jl, b.jcnt, mloc, p2, pd);
          break;
        case FWD_STORE | FWD_PAIR:
          fwd_kernel<R, D, DU, FWD_STORE, true, true><<<sgrid, SPREAD_TPB, 0, s>>>(
              kp, u, xd, b.partC, static_cast<R *>(b.traj), b.flags, nullptr, nullptr, jl, b.jcnt, mloc, p2, pd);
          break;
        case FWD_CKPT | FWD_PAIR:
          fwd_kernel<R, D, DU, FWD_CKPT, true, true><<<sgrid, SPREAD_TPB, 0, s>>>(
              kp, u, xd, b.partC, nullptr, nullptr, static_cast<R *>(b.ckpt), nullptr, jl, nullptr, mloc, p2, pd);
          break;
        default:
          fwd_kernel<R, D, DU, FWD_CKPT, false, true><<<sgrid, SPREAD_TPB, 0, s>>>(
              kp, u, xd, b.partC, nullptr, nullptr, static_cast<R *>(b.ckpt), pc, jl, nullptr, mloc, p2, pd);
          break;
      }
      const bool pair = (mode & FWD_PAIR) != 0;
      spread_combine_kernel<R><<<grid, TPB, 0, s>>>(cw, pair ? cw + mloc : nullptr, mloc, b.partC,
                                                    pair ? b.partC2 : nullptr);
      count_launch(2);
      return cudaGetLastError();
    }
  }
  switch (mode) {
    case FWD_COST:
      fwd_kernel<R, D, DU, FWD_COST><<<grid, TPB, 0, s>>>(kp, u, xd, b.partC, nullptr, nullptr, nullptr, pc,
                                                          jl, nullptr, mloc, p2);
      break;
    case FWD_STORE:
      fwd_kernel<R, D, DU, FWD_STORE><<<grid, TPB, 0, s>>>(kp, u, xd, b.partC, static_cast<R *>(b.traj),
                                                           b.flags, nullptr, pc, jl, b.jcnt, mloc, p2);
      break;
    case FWD_STORE | FWD_PAIR:
    case FWD_CKPT | FWD_PAIR:
      if constexpr (PAIR_SWEEPS<D>) {   // the host asks for pairs only where they are built
        if (mode & FWD_STORE)
          fwd_kernel<R, D, DU, FWD_STORE, true><<<grid, TPB, 0, s>>>(kp, u, xd, b.partC, static_cast<R *>(b.traj),
                                                                     b.flags, nullptr, nullptr, jl, b.jcnt, mloc, p2);
        else
          fwd_kernel<R, D, DU, FWD_CKPT, true><<<grid, TPB, 0, s>>>(kp, u, xd, b.partC, nullptr, nullptr,
                                                                    static_cast<R *>(b.ckpt), nullptr, jl, nullptr,
                                                                    mloc, p2);
      } else {
        return cudaErrorNotSupported;
      }
      break;
    default:
      fwd_kernel<R, D, DU, FWD_CKPT><<<grid, TPB, 0, s>>>(kp, u, xd, b.partC, nullptr, nullptr,
                                                          static_cast<R *>(b.ckpt), pc, jl, nullptr, mloc, p2);
      break;
  }
  count_launch();
  return cudaGetLastError();
}

// Shared memory of the recompute adjoint for segments of S steps.
template <typename R, int D, int DU>
size_t recompute_smem(bool theta, int S) {
  return (size_t)S * D * TPB * sizeof(R) * (theta && recompute_zbuf<R, D, true>() ? 2 : 1) +
         (theta ? 0 : (size_t)seg_log_cap<D>() * (2 + D) * TPB * sizeof(R)) + grad_rows_bytes<R, DU, 8>();
}

// The dynamic shared-memory limit of a kernel is an attribute of the function on the
// current device: raised once per (kernel, device) where a launch needs more than the
// default 48 KB (not before every launch: it is not a stream operation).
inline cudaError_t ensure_dyn_smem(const void *fn, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, size_t> done;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(fn, dev);
  const auto it = done.find(key);
  if (it != done.end() && it->second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done[key] = bytes;
  return e;
}

template <typename R, int D, int DU>
cudaError_t op_adj(const jd_problem *p, int variant, bool theta, int64_t m_begin, int64_t mloc,
                   const void *uk, const PathBufs &b, cudaStream_t s) {
  KParams<R, D, DU> kp;   // passed by value to the kernel (copied at the launch)
  make_kparams<R, D, DU>(p, m_begin, mloc, kp);
  if (b.npart) kp.npart = b.npart;
  const dim3 grid((unsigned)ceil_div(mloc, TPB));
  const R *u = static_cast<const R *>(uk);
  const R *xd = static_cast<const R *>(p->xdk);
  cudaError_t err = cudaSuccess;
  if (variant == ADJ_STORED_V) {
    const R *tr = static_cast<const R *>(b.traj);
    R *lo = static_cast<R *>(b.lam_out);
    const JLog<R, D> jl{static_cast<typename V2<R>::T *>(b.log_kt), static_cast<R *>(b.log_y), mloc, b.log_cap};
    const size_t smem = grad_rows_bytes<R, DU, 16>() + adj_stage_bytes<R, D>();
    if (theta) {
      err = ensure_dyn_smem((const void *)adj_stored_kernel<R, D, DU, true>, smem);
      if (err == cudaSuccess)
        adj_stored_kernel<R, D, DU, true><<<grid, TPB, smem, s>>>(kp, u, xd, tr, b.flags, jl, b.jcnt, b.partG,
                                                                  b.partT, lo, mloc);
    } else if (lo) {
      err = ensure_dyn_smem((const void *)adj_stored_kernel<R, D, DU, false, true>, smem);
      if (err == cudaSuccess)
        adj_stored_kernel<R, D, DU, false, true><<<grid, TPB, smem, s>>>(kp, u, xd, tr, b.flags, jl, b.jcnt,
                                                                         b.partG, b.partT, lo, mloc);
    } else {
      err = ensure_dyn_smem((const void *)adj_stored_kernel<R, D, DU, false>, smem);
      if (err == cudaSuccess)
        adj_stored_kernel<R, D, DU, false><<<grid, TPB, smem, s>>>(kp, u, xd, tr, b.flags, jl, b.jcnt, b.partG,
                                                                   b.partT, nullptr, mloc);
    }
  } else {
    const size_t smem = recompute_smem<R, D, DU>(theta, kp.S);
    const R *ck = static_cast<const R *>(b.ckpt);
    if (theta) {
      if constexpr (theta5<R, D>()) {
        err = ensure_dyn_smem((const void *)adj_recompute_theta5_kernel<R, D, DU>, smem);
        if (err == cudaSuccess)
          adj_recompute_theta5_kernel<R, D, DU><<<grid, TPB, smem, s>>>(kp, u, xd, ck, b.partG, b.partT, mloc);
      } else {
        err = ensure_dyn_smem((const void *)adj_recompute_kernel<R, D, DU, true>, smem);
        if (err == cudaSuccess)
          adj_recompute_kernel<R, D, DU, true><<<grid, TPB, smem, s>>>(kp, u, xd, ck, b.partG, b.partT, mloc);
      }
    } else {
      err = ensure_dyn_smem((const void *)adj_recompute_kernel<R, D, DU, false>, smem);
      if (err == cudaSuccess)
        adj_recompute_kernel<R, D, DU, false><<<grid, TPB, smem, s>>>(kp, u, xd, ck, b.partG, b.partT, mloc);
    }
  }
  count_launch();
  if (err != cudaSuccess) return err;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched stored-plan sweeps (serving): up to kBatchMax problems of one instantiation in
// one launch.  The table of the problems is the kernel's parameter; problem i owns the
// launch's blocks first[i] .. first[i + 1] - 1, and each block runs the single-problem
// body with its index within its problem, so a problem's states, logs and partials are
// those of its own launch bit for bit.
// ---------------------------------------------------------------------------
template <typename R, int D, int DU>
struct SweepItem {
  KParams<R, D, DU> kp;
  const R *u, *xd;
  double *partC, *partG;
  R *traj;
  uint32_t *flags;
  JLog<R, D> jl;
  int *jcnt;
  int64_t mloc;
  PairOut<R, D> p2;
};
template <typename R, int D, int DU>
struct SweepBatch {
  int n;
  int first[kBatchMax + 1];
  SweepItem<R, D, DU> it[kBatchMax];
};

__device__ __forceinline__ int sweep_item(const int *first, int n) {
  int i = 0;
  while (i + 1 < n && (int)blockIdx.x >= first[i + 1]) ++i;
  return i;
}

template <typename R, int D, int DU, bool PAIR>
__global__ void __launch_bounds__(TPB) fwd_batch_kernel(const __grid_constant__ SweepBatch<R, D, DU> t) {
  __shared__ Pair<R> red[TPB / 32];
  const int i = sweep_item(t.first, t.n);
  const SweepItem<R, D, DU> &f = t.it[i];
  fwd_body<R, D, DU, FWD_STORE, PAIR, false>(f.kp, blockIdx.x - t.first[i], f.u, f.xd, f.partC, f.traj, f.flags,
                                             nullptr, nullptr, f.jl, f.jcnt, f.mloc, f.p2, PreDraws<R, D>{}, red);
}

template <typename R, int D, int DU>
__global__ void __launch_bounds__(TPB) adj_batch_kernel(const __grid_constant__ SweepBatch<R, D, DU> t) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ Pair<R> red1[TPB / 32];
  const int i = sweep_item(t.first, t.n);
  const SweepItem<R, D, DU> &f = t.it[i];
  const int64_t bid = blockIdx.x - t.first[i];
  if constexpr (pin_coef<D>()) {   // as adj_stored_kernel: the drift family decided once
    if (f.kp.cubic)
      stored_sweep<R, D, DU, false, false, 1>(f.kp, f.u, f.xd, f.traj, f.flags, f.jl, f.jcnt, f.partG, nullptr,
                                              nullptr, f.mloc, dsm, red1, bid);
    else
      stored_sweep<R, D, DU, false, false, 0>(f.kp, f.u, f.xd, f.traj, f.flags, f.jl, f.jcnt, f.partG, nullptr,
                                              nullptr, f.mloc, dsm, red1, bid);
  } else {
    stored_sweep<R, D, DU, false, false, -1>(f.kp, f.u, f.xd, f.traj, f.flags, f.jl, f.jcnt, f.partG, nullptr,
                                             nullptr, f.mloc, dsm, red1, bid);
  }
}

template <typename R, int D, int DU>
int sweep_table(const BatchSweep *items, int n, bool pair, SweepBatch<R, D, DU> &t) {
  static_assert(sizeof(SweepBatch<R, D, DU>) <= 32000, "the table is one kernel parameter (at most 32764 bytes)");
  t.n = n;
  int nb = 0;
  for (int i = 0; i < n; ++i) {
    const jd_problem *p = items[i].p;
    const PathBufs &b = items[i].b;
    const int64_t M = p->desc.M;
    SweepItem<R, D, DU> &f = t.it[i];
    make_kparams<R, D, DU>(p, 0, M, f.kp);
    f.u = static_cast<const R *>(items[i].uk);
    f.xd = static_cast<const R *>(p->xdk);
    f.partC = b.partC;
    f.partG = b.partG;
    f.traj = static_cast<R *>(b.traj);
    f.flags = b.flags;
    f.jl = JLog<R, D>{static_cast<typename V2<R>::T *>(b.log_kt), static_cast<R *>(b.log_y), M, b.log_cap};
    f.jcnt = b.jcnt;
    f.mloc = M;
    f.p2 = PairOut<R, D>{};
    if (pair)
      f.p2 = PairOut<R, D>{static_cast<const R *>(b.uk2), b.partC2, static_cast<R *>(b.traj2), nullptr,
                           JLog<R, D>{static_cast<typename V2<R>::T *>(b.log_kt2), static_cast<R *>(b.log_y2), M,
                                      b.log_cap}};
    t.first[i] = nb;
    nb += (int)ceil_div(M, TPB);
  }
  t.first[n] = nb;
  return nb;
}

template <typename R, int D, int DU>
cudaError_t op_fwd_batch(const BatchSweep *items, int n, int mode, cudaStream_t s) {
  if (n < 1 || n > kBatchMax) return cudaErrorInvalidValue;
  static thread_local SweepBatch<R, D, DU> t;   // a large table: kept off the stack
  const bool pair = (mode & FWD_PAIR) != 0;
  const int nb = sweep_table<R, D, DU>(items, n, pair, t);
  if constexpr (PAIR_SWEEPS<D>) {
    if (pair)
      fwd_batch_kernel<R, D, DU, true><<<nb, TPB, 0, s>>>(t);
    else
      fwd_batch_kernel<R, D, DU, false><<<nb, TPB, 0, s>>>(t);
  } else {
    if (pair) return cudaErrorNotSupported;
    fwd_batch_kernel<R, D, DU, false><<<nb, TPB, 0, s>>>(t);
  }
  count_launch();
  return cudaGetLastError();
}

template <typename R, int D, int DU>
cudaError_t op_adj_batch(const BatchSweep *items, int n, cudaStream_t s) {
  if (n < 1 || n > kBatchMax) return cudaErrorInvalidValue;
  static thread_local SweepBatch<R, D, DU> t;
  const int nb = sweep_table<R, D, DU>(items, n, false, t);
  const size_t smem = grad_rows_bytes<R, DU, 16>() + adj_stage_bytes<R, D>();
  cudaError_t err = ensure_dyn_smem((const void *)adj_batch_kernel<R, D, DU>, smem);
  if (err == cudaSuccess) adj_batch_kernel<R, D, DU><<<nb, TPB, smem, s>>>(t);
  count_launch();
  if (err != cudaSuccess) return err;
  return cudaGetLastError();
}

template <typename R, int D, int DU>
constexpr bool batch_built() {
  return D <= 2 && DU == 1;
}

template <typename R, int D, int DU>
size_t op_stack_bytes() {
  size_t need = 2 * sizeof(JumpStep<R, D>) + 2048;
  const void *ks[] = {
      (const void *)fwd_kernel<R, D, DU, FWD_COST>, (const void *)fwd_kernel<R, D, DU, FWD_STORE>,
      (const void *)fwd_kernel<R, D, DU, FWD_CKPT>, (const void *)adj_stored_kernel<R, D, DU, false>,
      (const void *)adj_stored_kernel<R, D, DU, false, true>,
      (const void *)adj_stored_kernel<R, D, DU, true>, (const void *)adj_recompute_kernel<R, D, DU, false>,
      theta_recompute_fn<R, D, DU>()};
  for (const void *k : ks) {
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, k) == cudaSuccess && a.localSizeBytes + 1024 > need)
      need = a.localSizeBytes + 1024;
  }
  if constexpr (PAIR_SWEEPS<D>) {
    for (const void *k : {(const void *)fwd_kernel<R, D, DU, FWD_STORE, true>,
                          (const void *)fwd_kernel<R, D, DU, FWD_CKPT, true>}) {
      cudaFuncAttributes a;
      if (cudaFuncGetAttributes(&a, k) == cudaSuccess && a.localSizeBytes + 1024 > need)
        need = a.localSizeBytes + 1024;
    }
  }
  if constexpr (batch_built<R, D, DU>()) {
    for (const void *k : {(const void *)fwd_batch_kernel<R, D, DU, false>, (const void *)fwd_batch_kernel<R, D, DU, true>,
                          (const void *)adj_batch_kernel<R, D, DU>}) {
      cudaFuncAttributes a;
      if (cudaFuncGetAttributes(&a, k) == cudaSuccess && a.localSizeBytes + 1024 > need)
        need = a.localSizeBytes + 1024;
    }
  }
  return (need + 255) & ~(size_t)255;
}

template <typename R, int D, int DU>
constexpr PathOps make_ops() {
  if constexpr (batch_built<R, D, DU>())
    return PathOps{D, DU, seg_len<D>(), (int)sizeof(R), 0, &op_stack_bytes<R, D, DU>, &op_fwd<R, D, DU>,
                   &op_adj<R, D, DU>, &recompute_smem<R, D, DU>, &op_fwd_batch<R, D, DU>, &op_adj_batch<R, D, DU>};
  else
    return PathOps{D, DU, seg_len<D>(), (int)sizeof(R), 0, &op_stack_bytes<R, D, DU>, &op_fwd<R, D, DU>,
                   &op_adj<R, D, DU>, &recompute_smem<R, D, DU>, nullptr, nullptr};
}

}  // namespace jd
