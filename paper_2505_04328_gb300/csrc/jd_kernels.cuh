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
//   traj  [ceil((Nt+1)/4)][D][mloc][4]  states X_k, k = 4g + j, 16-byte vector stores
//   flags [ceil(Nt/32)][mloc]           bit k%32 set when step k had a jump
//   ckpt  [nseg+1][D][mloc]              X_{sS} for s < nseg, X_Nt at s = nseg
//   partC [nblk]                          FP64 block sums of the per-path cost
//   partG [Nt][DU][nblk * TPB/32]         FP64 warp sums of the control sensitivities
//   partT [D+2][nblk]                     FP64 block sums of the parameter sensitivities
#pragma once

#include <atomic>
#include <type_traits>

#include "jd_device.cuh"

namespace jd {

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
// grid in time order (one record per jump: step index k, time fraction theta, state
// Y right after the jump).  A step is logged only when all its records fit, so a
// backward sweep that finds record k == step k has the step's whole sub-grid; any
// other jump step is regenerated from the counter-based streams.
//   kt[r * stride + idx] = (k, theta),   y[(r * D + c) * stride + idx] = Y_c
// ---------------------------------------------------------------------------
template <typename R>
struct V2;
template <>
struct V2<float> {
  using T = float2;
  static __device__ __forceinline__ T make(float a, float b) { return make_float2(a, b); }
};
template <>
struct V2<double> {
  using T = double2;
  static __device__ __forceinline__ T make(double a, double b) { return make_double2(a, b); }
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
  __device__ __forceinline__ bool fits(int n) const { return r + n <= L.cap; }
  __device__ __forceinline__ void put(int k, R theta, const R (&y)[D]) {
    L.kt[(int64_t)r * L.stride + idx] = V2<R>::make((R)k, theta);
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
  __device__ __forceinline__ void init(int count) {
    rec = count - 1;
    rk = rec >= 0 ? L.kt[(int64_t)rec * L.stride + idx].x : R(-1);
  }
  __device__ __forceinline__ bool has(int k) const { return rk == (R)k; }
  __device__ __forceinline__ void pop(R &theta, R (&y)[D]) {
    theta = L.kt[(int64_t)rec * L.stride + idx].y;
#pragma unroll
    for (int c = 0; c < D; ++c) y[c] = L.y[((int64_t)rec * D + c) * L.stride + idx];
    --rec;
    rk = rec >= 0 ? L.kt[(int64_t)rec * L.stride + idx].x : R(-1);
  }
};

struct NoLog {};

// Recompute variant: steps per checkpoint segment.
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
    if (lw.fits(1)) lw.put(k, th, x);
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
// (kp itself or a HotFwd); the jump paths read kp.
template <typename R, int D, int DU, typename LW, bool INLINE_JUMP = true, typename KH = KParams<R, D, DU>>
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
      if (lw.fits(1)) lw.put(k, th, y1);
    }
    return 1;
  }
  if (INLINE_JUMP && one_jump(kp, w0)) {
    R xih[D], z1[D];
    const R th = slot0_draws(kp, k, m, xih, z1);
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
    if (lw.fits(S.n)) {
      for (int i = 0; i < S.n; ++i) {
        R y[D];
#pragma unroll
        for (int c = 0; c < D; ++c) y[c] = S.Y[i + 1][c];
        lw.put(k, S.th[i], y);
      }
    }
  }
  return S.n;
}

// One uniform step k from x (in place); returns the number of jumps.  With a LogWriter
// the post-jump states of the step are recorded.  zo (optional, stride zs) receives the
// step's main-stream normals Z_{k,0}.
template <typename R, int D, int DU, typename LW, bool ZOUT = false, bool INLINE_JUMP = true,
          typename KH = KParams<R, D, DU>>
__device__ __forceinline__ int forward_step_h(const KParams<R, D, DU> &kp, const KH &kh, int k, uint32_t m,
                                              const R *__restrict__ u, R (&x)[D], LW &lw,
                                              R *zo = nullptr, int zs = 0) {
  R z[D];
  const uint32_t w0 = main_draws(kp, k, m, z);
  if constexpr (ZOUT) {
#pragma unroll
    for (int c = 0; c < D; ++c) zo[c * zs] = z[c];
  }
  R uk[DU];
#pragma unroll
  for (int l = 0; l < DU; ++l) uk[l] = __ldg(u + (size_t)k * DU + l);
  return step_from_draws<R, D, DU, LW, INLINE_JUMP, KH>(kp, kh, k, m, w0, z, uk, x, lw);
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
template <typename R, int D, int DU, typename LW, typename KH>
__device__ __forceinline__ int forward_step2(const KParams<R, D, DU> &kp, const KH &kh, int k, uint32_t m,
                                             const R *__restrict__ u, R (&x)[D], LW &lw,
                                             const R *__restrict__ u2, R (&x2)[D], LW &lw2) {
  R z[D];
  const uint32_t w0 = main_draws(kp, k, m, z);
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
    const R th = slot0_draws(kp, k, m, xih, z1);
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
// rematerialise it from the parameter bank at every use inside the loop.
template <typename R, int D, int DU>
struct HotCoef {
  R A[D * D], C[D * D], B[D * DU], qdt[D];
  R dt;
  int cubic;
};

__device__ __forceinline__ float reg_pin(float v) {
  asm volatile("" : "+f"(v));
  return v;
}
__device__ __forceinline__ double reg_pin(double v) {
  asm volatile("" : "+d"(v));
  return v;
}

template <typename R, int D, int DU>
__device__ __forceinline__ HotCoef<R, D, DU> hot_coef(const KParams<R, D, DU> &kp) {
  HotCoef<R, D, DU> h;
#pragma unroll
  for (int i = 0; i < D * D; ++i) {
    h.A[i] = reg_pin(kp.A[i]);
    h.C[i] = kp.cubic ? reg_pin(kp.C[i]) : R(0);
  }
#pragma unroll
  for (int i = 0; i < D * DU; ++i) h.B[i] = reg_pin(kp.B[i]);
#pragma unroll
  for (int c = 0; c < D; ++c) h.qdt[c] = reg_pin(kp.qdt[c]);
  h.dt = reg_pin(kp.dt);
  h.cubic = kp.cubic;
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

// Store mode: the last three states of the current group of four ride in registers
// (b0, b1, b2) and the group leaves as one 16-byte vector per component.
template <typename R, int D>
__device__ __forceinline__ void stage_state(R *__restrict__ traj, int k, int Nt, int64_t mloc, int64_t lm,
                                            bool active, const R (&x)[D], R (&b0)[D], R (&b1)[D], R (&b2)[D]) {
  const int j = k & 3;
  if (j == 3 || k == Nt) {
    if (active) {
#pragma unroll
      for (int c = 0; c < D; ++c)
        Vec4<R>::store(traj + (((size_t)(k >> 2) * D + c) * mloc + lm) * 4, j == 0 ? x[c] : b0[c],
                       j == 1 ? x[c] : b1[c], j == 2 ? x[c] : b2[c], x[c]);
    }
  } else {
#pragma unroll
    for (int c = 0; c < D; ++c) {
      b0[c] = j == 0 ? x[c] : b0[c];
      b1[c] = j == 1 ? x[c] : b1[c];
      b2[c] = j == 2 ? x[c] : b2[c];
    }
  }
}

template <typename R, int D, int DU, int MODE, bool PAIR = false>
__global__ void __launch_bounds__(TPB)
fwd_kernel(const __grid_constant__ KParams<R, D, DU> kp, const R *__restrict__ u,
           const R *__restrict__ xd, double *__restrict__ partC, R *__restrict__ traj,
           uint32_t *__restrict__ flags, R *__restrict__ ckpt, R *__restrict__ pcost,
           JLog<R, D> jl, int *__restrict__ jcnt, int64_t mloc, PairOut<R, D> p2) {
  __shared__ Pair<R> red[TPB / 32];
  const int64_t lm = (int64_t)blockIdx.x * TPB + threadIdx.x;
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
  R b0[D], b1[D], b2[D], c0[D], c1[D], c2[D];
#pragma unroll
  for (int c = 0; c < D; ++c) b0[c] = b1[c] = b2[c] = c0[c] = c1[c] = c2[c] = R(0);
  constexpr int UNR = ((PAIR || MODE == FWD_CKPT) && D <= 2) ? 2 : 1;
#pragma unroll UNR
  for (int k = 0; k <= Nt; ++k) {
    if (MODE == FWD_STORE) {
      stage_state<R, D>(traj, k, Nt, mloc, lm, active, x, b0, b1, b2);
      if constexpr (PAIR) stage_state<R, D>(p2.traj, k, Nt, mloc, lm, active, x2, c0, c1, c2);
    }
    if (k == Nt) break;
    if (MODE == FWD_CKPT && active && (k % seg_len<D>()) == 0) {   // S is a power of two
#pragma unroll
      for (int c = 0; c < D; ++c) {
        ckpt[((size_t)(k / seg_len<D>()) * D + c) * mloc + lm] = x[c];
        if constexpr (PAIR) p2.ckpt[((size_t)(k / seg_len<D>()) * D + c) * mloc + lm] = x2[c];
      }
    }
    int nj;
    if constexpr (PAIR)
      nj = forward_step2(kp, kh, k, m, u, x, lw, p2.u, x2, lw2);
    else
      nj = forward_step_h<R, D, DU, LW, false, true, KH>(kp, kh, k, m, u, x, lw);
    if (nj) fw |= 1u << (k & 31);
    cost.add(cost_term(kh, x, xd + (size_t)(k + 1) * D));
    if constexpr (PAIR) cost2.add(cost_term(kh, x2, xd + (size_t)(k + 1) * D));
    if (MODE == FWD_STORE && ((k & 31) == 31 || k == Nt - 1)) {
      if (active) flags[(size_t)(k >> 5) * mloc + lm] = fw;
      fw = 0;
    }
  }
  if constexpr (MODE == FWD_STORE) {
    if (active) jcnt[lm] = lw.r;   // the same count for the second control
  }
  if (MODE == FWD_CKPT && active) {
    const int nseg = (Nt + seg_len<D>() - 1) / seg_len<D>();
#pragma unroll
    for (int c = 0; c < D; ++c) {
      ckpt[((size_t)nseg * D + c) * mloc + lm] = x[c];
      if constexpr (PAIR) p2.ckpt[((size_t)nseg * D + c) * mloc + lm] = x2[c];
    }
  }
  Pair<R> v = cost.pair();
  if (!active) v = {R(0), R(0)};
  if (pcost && active) pcost[lm] = Ar<R>::add(v.s, v.e);
  const double s = block_sum_to_double(v, red);
  if (threadIdx.x == 0) partC[blockIdx.x] = s;
  if constexpr (PAIR) {
    Pair<R> v2 = cost2.pair();
    if (!active) v2 = {R(0), R(0)};
    const double s2 = block_sum_to_double(v2, red);
    if (threadIdx.x == 0) p2.partC[blockIdx.x] = s2;
  }
}

template <typename R, int D>
__device__ __forceinline__ void load_state(const R *__restrict__ traj, int k, int64_t mloc,
                                           int64_t lm, R (&x)[D]) {
  const int g = k >> 2, j = k & 3;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    R v[4];
    Vec4<R>::load(traj + (((size_t)g * D + c) * mloc + lm) * 4, v);
    x[c] = j == 0 ? v[0] : (j == 1 ? v[1] : (j == 2 ? v[2] : v[3]));
  }
}

template <typename R, int D, int DU, bool THETA>
__device__ __forceinline__ void finish_theta(const KParams<R, D, DU> &kp, R (&th)[D + 2], bool active,
                                             double *__restrict__ partT, Pair<R> *red) {
  if constexpr (THETA) {
    // unrolled: a runtime index into th would keep the accumulators in local memory
#pragma unroll
  for (int t = 0; t < D + 2; ++t) {
    Pair<R> v = {active ? th[t] : R(0), R(0)};
    const double s = block_sum_to_double(v, red);
    if (threadIdx.x == 0) partT[(size_t)t * kp.nblk + blockIdx.x] = s;
  }
  }
}

// LAM: write the adjoint states to lam_out (jd_sample_paths); a compile-time switch, since
// a run-time test leaves its stores and their address arithmetic in every step.
template <typename R, int D, int DU, bool THETA, bool LAM = false>
__global__ void __launch_bounds__(TPB)
adj_stored_kernel(const __grid_constant__ KParams<R, D, DU> kp, const R *__restrict__ u,
                  const R *__restrict__ xd, const R *__restrict__ traj,
                  const uint32_t *__restrict__ flags, JLog<R, D> jl, const int *__restrict__ jcnt,
                  double *__restrict__ partG, double *__restrict__ partT, R *__restrict__ lam_out,
                  int64_t mloc) {
  using M = Ar<R>;
  __shared__ Pair<R> red1[TPB / 32];
  const int64_t npart = kp.npart;
  const int64_t lm = (int64_t)blockIdx.x * TPB + threadIdx.x;
  const bool active = lm < mloc;
  // inactive threads of the last block replay path 0 (its stored data and its random
  // streams must belong to the same path) and discard the result
  const int64_t lmc = active ? lm : 0;
  const uint32_t m = (uint32_t)(kp.m_begin + lmc);
  const int Nt = kp.Nt;
  LogReader<R, D> lr;
  lr.L = jl;
  lr.idx = lmc;
  lr.init(min(__ldg(jcnt + lmc), jl.cap));
  R mu[D], th[D + 2];
#pragma unroll
  for (int t = 0; t < D + 2; ++t) th[t] = R(0);
  {
    R x[D];
    load_state<R, D>(traj, Nt, mloc, lmc, x);
#pragma unroll
    for (int c = 0; c < D; ++c) mu[c] = M::mul(kp.qdt[c], M::sub(x[c], __ldg(xd + (size_t)Nt * D + c)));
    if (LAM && active)
#pragma unroll
      for (int c = 0; c < D; ++c) lam_out[((size_t)Nt * D + c) * mloc + lm] = mu[c];
  }
  constexpr bool PIN = pin_coef<D>();
  using KH = typename std::conditional<PIN, HotCoef<R, D, DU>, KParams<R, D, DU>>::type;
  HotCoef<R, D, DU> khv;
  if constexpr (PIN) khv = hot_coef(kp);
  const KH &kh = coef_src<PIN>(kp, khv);
  const int nbatch = (Nt + BATCH - 1) / BATCH;
  const int ng = (Nt + 4) / 4;   // groups of 4 stored states
#pragma unroll 1
  for (int b = nbatch - 1; b >= 0; --b) {
    R xs[BATCH][D];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g = 2 * b + h;
      if (g >= ng) {   // the top batch may end inside group 2b
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
          for (int j = 0; j < 4; ++j) xs[4 * h + j][c] = R(0);
        continue;
      }
#pragma unroll
      for (int c = 0; c < D; ++c) {
        R v[4];
        Vec4<R>::load(traj + (((size_t)g * D + c) * mloc + lmc) * 4, v);
#pragma unroll
        for (int j = 0; j < 4; ++j) xs[4 * h + j][c] = v[j];
      }
    }
    const uint32_t fw = __ldg(flags + (size_t)((BATCH * b) >> 5) * mloc + lmc);
    Pair<R> gb[BATCH][DU];
#pragma unroll
    for (int j = BATCH - 1; j >= 0; --j) {
      const int k = BATCH * b + j;
      R g[DU];
#pragma unroll
      for (int l = 0; l < DU; ++l) g[l] = R(0);
      if (k < Nt) {
        backward_step<R, D, DU, THETA, LogReader<R, D>, false, KH>(
            kp, kh, k, m, (fw >> (k & 31)) & 1u, xs[j], u, xd, mu, g, th, lr);
        if (LAM && active)
#pragma unroll
          for (int c = 0; c < D; ++c) lam_out[((size_t)k * D + c) * mloc + lm] = mu[c];
      }
#pragma unroll
      for (int l = 0; l < DU; ++l) gb[j][l] = {active ? g[l] : R(0), R(0)};
    }
    reduce_batch<R, DU>(gb, BATCH * b, Nt, partG, npart);
  }
  finish_theta<R, D, DU, THETA>(kp, th, active, partT, red1);
}

// Jump-log records per path and checkpoint segment in the recompute adjoint's shared
// memory (a segment whose jumps do not fit regenerates them).  Four records hold a
// 16-step segment's jumps except with probability below 1e-5 at lambda dt = 0.01, and
// keep the d = 2 block at 24 KB (8 blocks per SM, the register limit).
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

template <typename R, int D, int DU, bool THETA>
__global__ void __launch_bounds__(TPB)
adj_recompute_kernel(const __grid_constant__ KParams<R, D, DU> kp, const R *__restrict__ u,
                     const R *__restrict__ xd, const R *__restrict__ ckpt,
                     double *__restrict__ partG, double *__restrict__ partT, int64_t mloc) {
  using M = Ar<R>;
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
  R *gcol = sy + (size_t)JS * D * TPB;   // THETA: [BATCH * DU][TPB] per-step contributions
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
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const R xN = __ldg(ckpt + ((size_t)nseg * D + c) * mloc + lmc);
    mu[c] = M::mul(kp.qdt[c], M::sub(xN, __ldg(xd + (size_t)Nt * D + c)));
  }
#pragma unroll 1
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int k0 = seg * S, len = min(S, Nt - k0);
    R x[D];
#pragma unroll
    for (int c = 0; c < D; ++c) x[c] = __ldg(ckpt + ((size_t)seg * D + c) * mloc + lmc);
    uint32_t jm = 0;
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
        jm |= 1u << i;
    }
    LogReader<R, D> lr;
    lr.L = sl;
    lr.idx = tid;
    if constexpr (THETA)
      lr.init(0);   // empty: every jump step is regenerated
    else
      lr.init(lw.r);
    const int nb = (len + BATCH - 1) / BATCH;
#pragma unroll 1
    for (int bb = nb - 1; bb >= 0; --bb) {
      Pair<R> gb[BATCH][DU];
      if constexpr (THETA) {
        // rolled over the batch (the parameter-gradient step is large): each step's
        // contribution waits in the thread's shared column gcol[(j DU + l) TPB]
#pragma unroll 1
        for (int j = BATCH - 1; j >= 0; --j) {
          const int i = BATCH * bb + j, k = k0 + i;
          R g[DU];
#pragma unroll
          for (int l = 0; l < DU; ++l) g[l] = R(0);
          if (i < len) {
            R xk[D];
#pragma unroll
            for (int c = 0; c < D; ++c) xk[c] = sbuf[(i * D + c) * TPB + tid];
            backward_step<R, D, DU, THETA, LogReader<R, D>, ZBUF>(kp, kp, k, m, (jm >> i) & 1u, xk, u, xd, mu, g, th,
                                                                  lr, zbuf + (size_t)i * D * TPB + tid, TPB);
          }
#pragma unroll
          for (int l = 0; l < DU; ++l) gcol[(j * DU + l) * TPB + tid] = active ? g[l] : R(0);
        }
#pragma unroll
        for (int j = 0; j < BATCH; ++j)
#pragma unroll
          for (int l = 0; l < DU; ++l) gb[j][l] = {gcol[(j * DU + l) * TPB + tid], R(0)};
      } else {
#pragma unroll
        for (int j = BATCH - 1; j >= 0; --j) {
          const int i = BATCH * bb + j, k = k0 + i;
          R g[DU];
#pragma unroll
          for (int l = 0; l < DU; ++l) g[l] = R(0);
          if (i < len) {
            R xk[D];
#pragma unroll
            for (int c = 0; c < D; ++c) xk[c] = sbuf[(i * D + c) * TPB + tid];
            backward_step<R, D, DU, THETA, LogReader<R, D>, ZBUF>(kp, kp, k, m, (jm >> i) & 1u, xk, u, xd, mu, g, th,
                                                                  lr, zbuf + (size_t)i * D * TPB + tid, TPB);
          }
#pragma unroll
          for (int l = 0; l < DU; ++l) gb[j][l] = {active ? g[l] : R(0), R(0)};
        }
      }
      reduce_batch<R, DU>(gb, k0 + BATCH * bb, Nt, partG, npart);
    }
  }
  finish_theta<R, D, DU, THETA>(kp, th, active, partT, red1);
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
  kp.key0 = (uint32_t)(q.seed & 0xffffffffull);
  kp.key1 = (uint32_t)(q.seed >> 32);
  kp.epoch = q.epoch;
  kp.d = d;
  kp.npair = (d + 1) / 2;
  kp.Nt = q.Nt;
  kp.cubic = q.drift == JD_DRIFT_CUBIC;
  kp.jump_law = (int)q.jump_law;
  kp.jumps_on = q.jump_law != JD_JUMP_NONE && q.lambda > 0.0;
  kp.has_dA = !p->dA.empty();
  kp.S = seg_len<D>();
  kp.nblk = (int)ceil_div(mloc, TPB);
  kp.m_begin = m_begin;
  kp.npart = grad_parts(mloc);
}

template <typename R, int D, int DU>
cudaError_t op_fwd(const jd_problem *p, int mode, int64_t m_begin, int64_t mloc, const void *uk,
                   const PathBufs &b, cudaStream_t s) {
  auto *kp = new KParams<R, D, DU>();
  make_kparams<R, D, DU>(p, m_begin, mloc, *kp);
  if (b.npart) kp->npart = b.npart;
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
  switch (mode) {
    case FWD_COST:
      fwd_kernel<R, D, DU, FWD_COST><<<grid, TPB, 0, s>>>(*kp, u, xd, b.partC, nullptr, nullptr, nullptr, pc,
                                                          jl, nullptr, mloc, p2);
      break;
    case FWD_STORE:
      fwd_kernel<R, D, DU, FWD_STORE><<<grid, TPB, 0, s>>>(*kp, u, xd, b.partC, static_cast<R *>(b.traj),
                                                           b.flags, nullptr, pc, jl, b.jcnt, mloc, p2);
      break;
    case FWD_STORE | FWD_PAIR:
    case FWD_CKPT | FWD_PAIR:
      if constexpr (PAIR_SWEEPS<D>) {   // the host asks for pairs only where they are built
        if (mode & FWD_STORE)
          fwd_kernel<R, D, DU, FWD_STORE, true><<<grid, TPB, 0, s>>>(*kp, u, xd, b.partC, static_cast<R *>(b.traj),
                                                                     b.flags, nullptr, nullptr, jl, b.jcnt, mloc, p2);
        else
          fwd_kernel<R, D, DU, FWD_CKPT, true><<<grid, TPB, 0, s>>>(*kp, u, xd, b.partC, nullptr, nullptr,
                                                                    static_cast<R *>(b.ckpt), nullptr, jl, nullptr,
                                                                    mloc, p2);
      } else {
        delete kp;
        return cudaErrorNotSupported;
      }
      break;
    default:
      fwd_kernel<R, D, DU, FWD_CKPT><<<grid, TPB, 0, s>>>(*kp, u, xd, b.partC, nullptr, nullptr,
                                                          static_cast<R *>(b.ckpt), pc, jl, nullptr, mloc, p2);
      break;
  }
  delete kp;
  count_launch();
  return cudaGetLastError();
}

template <typename R, int D, int DU>
constexpr size_t recompute_smem(bool theta) {
  return (size_t)seg_len<D>() * D * TPB * sizeof(R) * (theta && recompute_zbuf<R, D, true>() ? 2 : 1) +
         (theta ? (size_t)BATCH * DU * TPB * sizeof(R) : (size_t)seg_log_cap<D>() * (2 + D) * TPB * sizeof(R));
}

template <typename R, int D, int DU>
cudaError_t op_adj(const jd_problem *p, int variant, bool theta, int64_t m_begin, int64_t mloc,
                   const void *uk, const PathBufs &b, cudaStream_t s) {
  auto *kp = new KParams<R, D, DU>();
  make_kparams<R, D, DU>(p, m_begin, mloc, *kp);
  if (b.npart) kp->npart = b.npart;
  const dim3 grid((unsigned)ceil_div(mloc, TPB));
  const R *u = static_cast<const R *>(uk);
  const R *xd = static_cast<const R *>(p->xdk);
  cudaError_t err = cudaSuccess;
  if (variant == ADJ_STORED_V) {
    const R *tr = static_cast<const R *>(b.traj);
    R *lo = static_cast<R *>(b.lam_out);
    const JLog<R, D> jl{static_cast<typename V2<R>::T *>(b.log_kt), static_cast<R *>(b.log_y), mloc, b.log_cap};
    if (theta)
      adj_stored_kernel<R, D, DU, true><<<grid, TPB, 0, s>>>(*kp, u, xd, tr, b.flags, jl, b.jcnt, b.partG,
                                                             b.partT, lo, mloc);
    else if (lo)
      adj_stored_kernel<R, D, DU, false, true><<<grid, TPB, 0, s>>>(*kp, u, xd, tr, b.flags, jl, b.jcnt, b.partG,
                                                                    b.partT, lo, mloc);
    else
      adj_stored_kernel<R, D, DU, false><<<grid, TPB, 0, s>>>(*kp, u, xd, tr, b.flags, jl, b.jcnt, b.partG,
                                                              b.partT, nullptr, mloc);
  } else {
    const size_t smem = recompute_smem<R, D, DU>(theta);
    const R *ck = static_cast<const R *>(b.ckpt);
    // the dynamic shared-memory limit is a property of the function: set once per process
    // (one device per process)
    // (it is not a stream operation, and a call per launch sat between the phases)
    static std::atomic<bool> set_theta{false}, set_plain{false};
    std::atomic<bool> &done = theta ? set_theta : set_plain;
    if (!done.load(std::memory_order_acquire)) {
      err = theta ? cudaFuncSetAttribute(adj_recompute_kernel<R, D, DU, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                  : cudaFuncSetAttribute(adj_recompute_kernel<R, D, DU, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err == cudaSuccess) done.store(true, std::memory_order_release);
    }
    if (err == cudaSuccess) {
      if (theta)
        adj_recompute_kernel<R, D, DU, true><<<grid, TPB, smem, s>>>(*kp, u, xd, ck, b.partG, b.partT, mloc);
      else
        adj_recompute_kernel<R, D, DU, false><<<grid, TPB, smem, s>>>(*kp, u, xd, ck, b.partG, b.partT, mloc);
    }
  }
  delete kp;
  count_launch();
  if (err != cudaSuccess) return err;
  return cudaGetLastError();
}

template <typename R, int D, int DU>
size_t op_stack_bytes() {
  size_t need = 2 * sizeof(JumpStep<R, D>) + 2048;
  const void *ks[] = {
      (const void *)fwd_kernel<R, D, DU, FWD_COST>, (const void *)fwd_kernel<R, D, DU, FWD_STORE>,
      (const void *)fwd_kernel<R, D, DU, FWD_CKPT>, (const void *)adj_stored_kernel<R, D, DU, false>,
      (const void *)adj_stored_kernel<R, D, DU, false, true>,
      (const void *)adj_stored_kernel<R, D, DU, true>, (const void *)adj_recompute_kernel<R, D, DU, false>,
      (const void *)adj_recompute_kernel<R, D, DU, true>};
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
  return (need + 255) & ~(size_t)255;
}

template <typename R, int D, int DU>
constexpr PathOps make_ops() {
  return PathOps{D, DU, seg_len<D>(), (int)sizeof(R), 0, &op_stack_bytes<R, D, DU>, &op_fwd<R, D, DU>,
                 &op_adj<R, D, DU>};
}

}  // namespace jd
