// jd_feedback.cuh -- path kernels of the feedback control u(z, t) = mu(t)^T phi(z)
// (Sec. 2 eq:control_structure) on the phase space z = (x, v) (d = 2, du = 1):
//
//  phi_{i,l}(z) = phi(x - x^i) phi(v - v^l), the bump of Sec. 5.2 eq:Gaussian_RBF,
//  phi(r) = exp(-1 / (1 - (eps r)^2)) on |r| < 1/eps, centred on the cell centres of
//  Sec. 5.1.  The control enters the drift as B u(z) and is evaluated at the left end
//  of every sub-step of the jump-adapted grid (Algorithm 5.1); the path cost is
//  sum_k dt l(X_{k+1}) + sum over sub-steps (alpha/2) delta u(Y)^2 with the quadratic
//  or the Gaussian tracking term l (Sec. 6 eq:tracking_cost).
//
//  fb_fwd_kernel     forward sweep, one thread per path; per-block FP64 cost partials;
//                    optionally stores X_k and the jump flags for the adjoint.
//  fb_adj_kernel     backward sweep over the stored states (steps with jumps are
//                    regenerated from X_k and the counter-based streams) with
//                    a <- a + delta [J_f^T a + w grad u],  w = alpha u + B^T a
//                    (Sec. 5.5 eq:adjoint_eq_approximation); the gradient
//                    dJ/dmu_{k,i,l} = (1/M) sum over paths and sub-steps of
//                    delta w phi_x,i phi_v,l (eq:definition_Gradient) is, per step, a
//                    sum of outer products over paths: each warp exchanges its 32 paths'
//                    factors through shared memory and forms 32-path dot products
//                    (paired FMAs), one partial per warp, step and weight.
//  fb_reduce_kernel  FP64 sums of the warp partials over groups of warps (fixed order).
//
// No block barrier inside the sweeps: the weights are read through L1 (every thread of
// a step reads the same 4 NX NV bytes), the exchange is per warp.  FP32 paths use the
// SFU for the bumps (rcp.approx, ex2.approx with e^y = 2^(y log2 e)) and paired
// FFMA2/FMUL2 arithmetic; FP64 paths use IEEE division and exp.
//
// The kernels work on padded sizes NX x NV (instances 4x4, 10x10, 16x16): the weights
// beyond nx x nv are 0, so the bumps of the padding centres do not reach u.
//
// A step with jumps runs its sub-steps in the same loop as a step without (forward: one
// sub-step per iteration; adjoint: one backward sub-step and one warp exchange per
// round), so a warp in which one path jumps pays one more pass of the same code rather
// than a separate, serialized jump routine.
//
// Layouts (mloc paths, nwarp = ceil(mloc / 32)):
//   mu    [Nt][NX/2][NV][2]        kernel precision, weights of rows i, i+1 interleaved
//   traj  [Nt+1][2][mloc]          states X_k
//   flags [ceil(Nt/32)][mloc]      bit k%32 set when step k had a jump
//   partC [nblk]                   FP64 block sums of the path costs
//   partW [nwarp][Nt][NX/2][NV][2] kernel-precision warp sums of the gradient (weight
//                                  (i, l) at 2 (i/2 NV + l) + i%2)
//   partG [ngroup][Nt][NX/2][NV][2] FP64 sums of partW over groups of FB_GROUP_WARPS warps
#pragma once

#include <cooperative_groups.h>

#include "jd_kernels.cuh"

namespace jd {

constexpr int FB_AROW = 68;   // exchange buffer: pitch of a pair row (2 x 32 values + 4)

template <typename R>
struct FbParams {
  R xc0, dxc, vc0, dvc;     // centres x^i = xc0 + i dxc, v^l = vc0 + l dvc
  R eps2, m2eps2;           // eps^2, -2 eps^2
  R alpha, halpha;          // alpha, alpha / 2
  R q[2];                   // tracking weights
  R hinv_s2, inv_s2;        // Gaussian: 1 / (2 sigma_J^2), 1 / sigma_J^2
  R srate_dt;               // surrogate adjoint (Sec. 6.5): variance of step k is srate_dt k
  R omega;                  // interacting particles (Sec. 6.4): ring coupling
  R iax2, iav2;             // ellipse cost: 1 / A_x^2, 1 / A_v^2
  const R *z0;              // interacting particles: initial states [2][S] (on the ellipse)
  int gauss, ellipse, N, Nt;   // N: particles per ring, 0 = independent paths
  int S;                    // lanes (path indices) per ring: particle i of ring r is lane S r + i
  int64_t mloc;
};

// ---------------------------------------------------------------------------
// Rings of interacting particles (Sec. 6.4): particle i of a ring needs a value of its
// neighbours i - 1 and i + 1 (cyclic over the ring's N particles) once per step.  The ring
// occupies S consecutive lanes (S = 32 for N <= 32, the next power of two up to 256, then
// 256 per block of a thread-block cluster), by its size:
//   RING 1: one warp per ring, two shuffles;
//   RING 2: rings of 64, 128 or 256 lanes within a block: shared memory, one block barrier;
//   RING 3: a ring of C = S / 256 blocks forming one thread-block cluster (N <= 2048): each
//           block's shared memory, read across the cluster (distributed shared memory),
//           one cluster barrier.
// Every lane of a ring (idle ones too) calls get() once per step; the buffers alternate,
// so one barrier per exchange suffices.
// ---------------------------------------------------------------------------
template <typename R, int RING>
struct RingX {
  R *sv;        // RING >= 2: [2][FB_TPB] shared buffer of this block
  int i, N;     // particle index in the ring, particles per ring
  int par = 0;  // buffer in use
  __device__ __forceinline__ int left() const { return i == 0 ? N - 1 : i - 1; }
  __device__ __forceinline__ int right() const { return i == N - 1 ? 0 : i + 1; }
  __device__ __forceinline__ void get(R v, R &vl, R &vr) {
    if constexpr (RING == 1) {
      const int l = i < N ? left() : 0, r = i < N ? right() : 0;
      vl = __shfl_sync(0xffffffffu, v, l);
      vr = __shfl_sync(0xffffffffu, v, r);
    } else if constexpr (RING == 2) {
      R *b = sv + par * FB_TPB;
      b[threadIdx.x] = v;
      __syncthreads();
      const int base = threadIdx.x - i;
      vl = i < N ? b[base + left()] : R(0);
      vr = i < N ? b[base + right()] : R(0);
      par ^= 1;
    } else if constexpr (RING == 3) {
      namespace cg = cooperative_groups;
      cg::cluster_group cl = cg::this_cluster();
      R *b = sv + par * FB_TPB;
      b[threadIdx.x] = v;
      cl.sync();
      vl = vr = R(0);
      if (i < N) {
        const int l = left(), r = right();
        vl = *cl.map_shared_rank(b + l % FB_TPB, (unsigned)(l / FB_TPB));
        vr = *cl.map_shared_rank(b + r % FB_TPB, (unsigned)(r / FB_TPB));
      }
      par ^= 1;
    }
  }
};



// ---------------------------------------------------------------------------
// Bumps.  phi = exp(-t), t = 1 / (1 - eps^2 r^2) on the support;
// d phi / dr = phi t^2 (-2 eps^2 r).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float sfu_rcp(float a) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ float sfu_ex2(float a) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
constexpr float kNegLog2e = -1.4426950408889634f;   // -log2(e): exp(-t) = 2^(-t log2 e)

// FP64: one bump (IEEE division and exp)
template <bool GRAD>
__device__ __forceinline__ double bump(double r, const FbParams<double> &fp, double &dphi) {
  using M = Ar<double>;
  const double s1 = M::fma(-fp.eps2, M::mul(r, r), 1.0);   // 1 - eps^2 r^2
  if (!(s1 > 0.0)) {
    dphi = 0.0;
    return 0.0;
  }
  const double t = 1.0 / s1;
  const double ph = ::exp(-t);
  if (GRAD) dphi = M::mul(M::mul(ph, M::mul(t, t)), M::mul(fp.m2eps2, r));
  return ph;
}

// FP32: two bumps at once (distances r0, r1 to their centres): paired arithmetic, SFU
// reciprocal and 2^y.  1 - eps^2 r^2 is clamped below at 2^-40 instead of branching on
// the support: off it (and where 1 - eps^2 r^2 < 2^-40, inside) t = 2^40 makes
// 2^(-t log2 e) exactly 0, and t^2 = 2^80 stays finite, so phi and phi' are 0.
template <bool GRAD>
__device__ __forceinline__ void bump2(float r0, float r1, const FbParams<float> &fp, float &p0, float &p1,
                                      float &d0, float &d1) {
  float q0, q1, s0 = 1.f, s1 = 1.f;
  Pr<float>::mul(r0, r1, r0, r1, q0, q1);
  Pr<float>::fma(-fp.eps2, -fp.eps2, q0, q1, s0, s1);   // 1 - eps^2 r^2
  const float t0 = sfu_rcp(fmaxf(s0, 0x1p-40f)), t1 = sfu_rcp(fmaxf(s1, 0x1p-40f));
  float y0, y1;
  Pr<float>::mul(t0, t1, kNegLog2e, kNegLog2e, y0, y1);
  p0 = sfu_ex2(y0);
  p1 = sfu_ex2(y1);
  if (GRAD) {
    float tt0, tt1, w0, w1, z0, z1;
    Pr<float>::mul(t0, t1, t0, t1, tt0, tt1);
    Pr<float>::mul(p0, p1, tt0, tt1, w0, w1);
    Pr<float>::mul(r0, r1, fp.m2eps2, fp.m2eps2, z0, z1);
    Pr<float>::mul(w0, w1, z0, z1, d0, d1);
  }
}

// The N bumps at x of the centres c0 + i dc (distances r_i = (x - c0) - i dc; FP32 steps
// them down two at a time).  Centres beyond nx / nv give bumps whose weights are 0.
template <typename R, int N, bool GRAD>
__device__ __forceinline__ void bumps(R x, R c0, R dc, const FbParams<R> &fp, R (&p)[N], R (&d)[N]) {
  using M = Ar<R>;
  const R r0 = M::sub(x, c0);
  if constexpr (Pr<R>::on) {
    R a0 = r0, a1 = M::sub(r0, dc);
    const R st = M::add(dc, dc);
#pragma unroll
    for (int i = 0; i < N; i += 2) {
      bump2<GRAD>(a0, a1, fp, p[i], p[i + 1], d[i], d[i + 1]);
      if (i + 2 < N) Pr<R>::sub(a0, a1, st, st, a0, a1);
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) p[i] = bump<GRAD>(M::fma(R(-i), dc, r0), fp, d[i]);
  }
}

// Two values of mu, rows i and i+1 at column l, and the next column (one 16-byte load
// in FP32).
template <typename R>
struct Mu4 {
  R a0, a1, b0, b1;   // (i, l), (i+1, l), (i, l+1), (i+1, l+1)
};
template <typename R>
__device__ __forceinline__ Mu4<R> load_mu4(const R *p);
template <>
__device__ __forceinline__ Mu4<float> load_mu4<float>(const float *p) {
  const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
  return {v.x, v.y, v.z, v.w};
}
template <>
__device__ __forceinline__ Mu4<double> load_mu4<double>(const double *p) {
  const double2 v = __ldg(reinterpret_cast<const double2 *>(p)), w = __ldg(reinterpret_cast<const double2 *>(p) + 1);
  return {v.x, v.y, w.x, w.y};
}

// u(z) = sum_i phi_x,i sum_l mu_k[i][l] phi_v,l with the shape-function values, and with
// GRAD also (u_x, u_v).  mk: the step's interleaved weights (global, read through L1).
template <typename R, int NX, int NV, bool GRAD>
__device__ __forceinline__ R fb_eval(const FbParams<R> &fp, const R *__restrict__ mk, R x, R v, R (&px)[NX],
                                     R (&pv)[NV], R &ux, R &uv) {
  using M = Ar<R>;
  R dpx[NX], dpv[NV];
  bumps<R, NX, GRAD>(x, fp.xc0, fp.dxc, fp, px, dpx);
  bumps<R, NV, GRAD>(v, fp.vc0, fp.dvc, fp, pv, dpv);
  // t_i = sum_l mu[i][l] phi_v,l (and tv_i with phi_v'), rows i, i+1 together
  R t[NX], tv[NX];
#pragma unroll
  for (int i = 0; i < NX; i += 2) {
    R a0 = R(0), a1 = R(0), b0 = R(0), b1 = R(0);
#pragma unroll
    for (int l = 0; l < NV; l += 2) {
      const Mu4<R> m = load_mu4<R>(mk + ((i / 2) * NV + l) * 2);
      if constexpr (Pr<R>::on) {
        Pr<R>::fma(m.a0, m.a1, pv[l], pv[l], a0, a1);
        Pr<R>::fma(m.b0, m.b1, pv[l + 1], pv[l + 1], a0, a1);
        if (GRAD) {
          Pr<R>::fma(m.a0, m.a1, dpv[l], dpv[l], b0, b1);
          Pr<R>::fma(m.b0, m.b1, dpv[l + 1], dpv[l + 1], b0, b1);
        }
      } else {
        a0 = M::fma(m.a0, pv[l], a0);
        a1 = M::fma(m.a1, pv[l], a1);
        a0 = M::fma(m.b0, pv[l + 1], a0);
        a1 = M::fma(m.b1, pv[l + 1], a1);
        if (GRAD) {
          b0 = M::fma(m.a0, dpv[l], b0);
          b1 = M::fma(m.a1, dpv[l], b1);
          b0 = M::fma(m.b0, dpv[l + 1], b0);
          b1 = M::fma(m.b1, dpv[l + 1], b1);
        }
      }
    }
    t[i] = a0;
    t[i + 1] = a1;
    tv[i] = b0;
    tv[i + 1] = b1;
  }
  // u = sum_i phi_x,i t_i, u_x = sum_i phi_x,i' t_i, u_v = sum_i phi_x,i tv_i (even and
  // odd i in two halves)
  R u0 = R(0), u1 = R(0), x0 = R(0), x1 = R(0), v0 = R(0), v1 = R(0);
#pragma unroll
  for (int i = 0; i < NX; i += 2) {
    if constexpr (Pr<R>::on) {
      Pr<R>::fma(px[i], px[i + 1], t[i], t[i + 1], u0, u1);
      if (GRAD) {
        Pr<R>::fma(dpx[i], dpx[i + 1], t[i], t[i + 1], x0, x1);
        Pr<R>::fma(px[i], px[i + 1], tv[i], tv[i + 1], v0, v1);
      }
    } else {
      u0 = M::fma(px[i], t[i], u0);
      u1 = M::fma(px[i + 1], t[i + 1], u1);
      if (GRAD) {
        x0 = M::fma(dpx[i], t[i], x0);
        x1 = M::fma(dpx[i + 1], t[i + 1], x1);
        v0 = M::fma(px[i], tv[i], v0);
        v1 = M::fma(px[i + 1], tv[i + 1], v1);
      }
    }
  }
  ux = M::add(x0, x1);
  uv = M::add(v0, v1);
  return M::add(u0, u1);
}

// dt l(z, t_k) and (with GRAD) its gradient dt grad l: quadratic (1/2) sum q_c e_c^2 or
// Gaussian -exp(-sum q_c e_c^2 / (2 sigma_J^2)), e = z - z_d(t_k).
template <typename R, bool GRAD>
__device__ __forceinline__ R fb_track(const FbParams<R> &fp, R dt, const R (&z)[2],
                                      const R *__restrict__ xdk, R (&g)[2]) {
  using M = Ar<R>;
  if (fp.ellipse) {   // -exp(-E^2 / (2 sigma_J^2)), E = x^2/A_x^2 + v^2/A_v^2 - 1 (Sec. 6.4)
    const R E = M::sub(M::fma(M::mul(z[1], z[1]), fp.iav2, M::mul(M::mul(z[0], z[0]), fp.iax2)), R(1));
    const R X = exp(-M::mul(M::mul(E, E), fp.hinv_s2));
    if (GRAD) {
      const R c = M::mul(dt, M::mul(M::mul(X, M::mul(E, fp.inv_s2)), R(2)));
      g[0] = M::mul(c, M::mul(z[0], fp.iax2));
      g[1] = M::mul(c, M::mul(z[1], fp.iav2));
    }
    return -M::mul(dt, X);
  }
  const R e0 = M::sub(z[0], __ldg(xdk)), e1 = M::sub(z[1], __ldg(xdk + 1));
  const R w0 = M::mul(fp.q[0], e0), w1 = M::mul(fp.q[1], e1);
  const R Q = M::fma(w1, e1, M::mul(w0, e0));
  if (fp.gauss) {
    const R E = exp(-M::mul(Q, fp.hinv_s2));
    if (GRAD) {
      const R c = M::mul(dt, M::mul(E, fp.inv_s2));
      g[0] = M::mul(c, w0);
      g[1] = M::mul(c, w1);
    }
    return -M::mul(dt, E);
  }
  if (GRAD) {
    g[0] = M::mul(dt, w0);
    g[1] = M::mul(dt, w1);
  }
  return M::mul(M::mul(R(0.5), dt), Q);
}

// One Euler sub-step of length de from y under the feedback control (plus, for
// interacting particles, the neighbours' force cin on the velocity); returns the
// sub-step's control cost (alpha/2) de u(y)^2.
template <typename R, int NX, int NV, bool CPL>
__device__ __forceinline__ R fb_substep(const KParams<R, 2, 1> &kp, const FbParams<R> &fp,
                                        const R *__restrict__ mk, R de, R sqde, const R (&z)[2], R (&y)[2],
                                        R cin) {
  using M = Ar<R>;
  R px[NX], pv[NV], ux, uv;
  const R u = fb_eval<R, NX, NV, false>(fp, mk, y[0], y[1], px, pv, ux, uv);
  const R uu[1] = {u};
  R f[2];
  drift(kp, y, uu, f);
  if (CPL) f[1] = M::add(f[1], cin);   // interacting particles: the neighbours' force
#pragma unroll
  for (int c = 0; c < 2; ++c) y[c] = M::fma(M::mul(kp.sigma[c], sqde), z[c], M::fma(de, f[c], y[c]));
  return M::mul(M::mul(fp.halpha, de), M::mul(u, u));
}

// Jump plan of a step with jumps (the per-step draws of Algorithm 5.2, as in
// build_jump_step): the Poisson count n from w0, the time fractions of the n slots
// sorted stably, and the slot of each jump in time order.
template <typename R>
struct FbPlan {
  R th[NMAX];
  int order[NMAX];
};

template <typename R>
__device__ __forceinline__ int fb_plan(const KParams<R, 2, 1> &kp, int k, uint32_t m, uint32_t w0, FbPlan<R> &P) {
  using M = Ar<R>;
  int n = 0;
#pragma unroll 1
  for (int i = 0; i < NMAX; ++i) n += ((unsigned long long)w0 >= kp.thr[i]) ? 1 : 0;
  R theta[NMAX];
#pragma unroll 1
  for (int i = 0; i < n; ++i) {
    const uint4 o = philox10((uint32_t)k, m, (1u << 24) | ((uint32_t)(i + 1) << 16), kp.epoch,
                             kp.key0, kp.key1);
    theta[i] = M::u01(o.x);
    P.order[i] = i;
  }
#pragma unroll 1
  for (int i = 1; i < n; ++i) {
    const int cur = P.order[i];
    int j = i - 1;
    while (j >= 0 && theta[P.order[j]] > theta[cur]) {
      P.order[j + 1] = P.order[j];
      --j;
    }
    P.order[j + 1] = cur;
  }
#pragma unroll 1
  for (int i = 0; i < n; ++i) P.th[i] = theta[P.order[i]];
  return n;
}

// Length of sub-step i of a step with n >= 1 jumps.
template <typename R>
__device__ __forceinline__ R fb_delta(const KParams<R, 2, 1> &kp, const FbPlan<R> &P, int n, int i) {
  using M = Ar<R>;
  if (i == 0) return M::mul(kp.dt, P.th[0]);
  if (i < n) return M::mul(kp.dt, M::sub(P.th[i], P.th[i - 1]));
  return M::mul(kp.dt, M::sub(R(1), P.th[n - 1]));
}

// Block sum of one compensated pair per thread (FB_TPB threads) into a double.
template <typename R>
__device__ __forceinline__ double fb_block_sum(Pair<R> v, Pair<R> *red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double out = 0.0;
  if (threadIdx.x == 0) {
    Pair<R> s = red[0];
    for (int w = 1; w < FB_TPB / 32; ++w) s = padd(s, red[w]);
    out = (double)s.s + (double)s.e;
  }
  return out;
}

template <typename R, int NX, int NV, bool STORE, int RING>
__global__ void __launch_bounds__(FB_TPB)
fb_fwd_kernel(const __grid_constant__ KParams<R, 2, 1> kp, const __grid_constant__ FbParams<R> fp,
              const R *__restrict__ mu, const R *__restrict__ xd, R *__restrict__ traj,
              uint32_t *__restrict__ flags, double *__restrict__ partC) {
  using M = Ar<R>;
  constexpr int LP = NX * NV;
  constexpr bool CPL = RING > 0;
  __shared__ Pair<R> red[FB_TPB / 32];
  __shared__ R ringbuf[RING >= 2 ? 2 * FB_TPB : 1];
  const int64_t mloc = fp.mloc, m = (int64_t)blockIdx.x * FB_TPB + threadIdx.x;
  // interacting particles: lane i < N of each S-lane ring is particle i (M is a multiple of
  // S, and of 256 for rings beyond a warp, so rings and blocks are whole); every lane of
  // the ring runs the step loop for the exchange
  RingX<R, RING> rx;
  rx.sv = ringbuf;
  rx.i = CPL ? (int)(m % fp.S) : 0;
  rx.N = fp.N;
  const bool in_range = m < mloc, active = in_range && (!CPL || rx.i < fp.N);
  const uint32_t mg = (uint32_t)(kp.m_begin + m);
  const int Nt = fp.Nt;
  Kahan<R> cost;
  if (in_range) {
    R z[2] = {kp.x0[0], kp.x0[1]};
    if (CPL && active) {
      z[0] = fp.z0[rx.i];
      z[1] = fp.z0[fp.S + rx.i];
    }
    uint32_t fw = 0;
    if (STORE && active) {
      traj[m] = z[0];
      traj[mloc + m] = z[1];
    }
#pragma unroll 1
    for (int k = 0; k < Nt; ++k) {
      R cin = R(0);
      if constexpr (CPL) {   // omega (x_{i-1} + x_{i+1}) at t_k, fixed over the step
        R xl, xr;
        rx.get(z[0], xl, xr);
        cin = M::mul(fp.omega, M::add(xl, xr));
        if (!active) continue;
      }
      const R *mk = mu + (size_t)k * LP;
      R zs[2];
      const uint32_t w0 = main_draws<true>(kp, k, mg, zs);   // round keys of the parameter block
      int n = 0;
      FbPlan<R> P;
      if (has_jump(kp, w0)) {
        n = fb_plan(kp, k, mg, w0, P);
        fw |= 1u << (k & 31);
      }
      // sub-steps 0..n (one when the step has no jump) in one loop, so that a warp with
      // a jumping path runs the same code for every sub-step (Algorithm 5.1)
#pragma unroll 1
      for (int i = 0;; ++i) {
        R de = kp.dt, sq = kp.sqdt;
        if (n > 0) {
          de = fb_delta(kp, P, n, i);
          sq = Ar<R>::sqrt(de);
        }
        cost.add(fb_substep<R, NX, NV, CPL>(kp, fp, mk, de, sq, zs, z, cin));
        if (i >= n) break;
        R xih[2];
        slot_draws(kp, k, mg, P.order[i], xih, zs);   // the jump's size and the next normals
        apply_jump(kp, z, xih);
      }
      R g[2];
      cost.add(fb_track<R, false>(fp, kp.dt, z, xd + (size_t)(k + 1) * 2, g));
      if (STORE) {
        traj[((size_t)(k + 1) * 2) * mloc + m] = z[0];
        traj[((size_t)(k + 1) * 2 + 1) * mloc + m] = z[1];
        if ((k & 31) == 31 || k == Nt - 1) {
          flags[(size_t)(k >> 5) * mloc + m] = fw;
          fw = 0;
        }
      }
    }
  }
  const double bs = fb_block_sum(active ? cost.pair() : Pair<R>{R(0), R(0)}, red);
  if (threadIdx.x == 0) partC[blockIdx.x] = bs;
}

// 32-path dot products of a 2 x 2 block of weights: pa is the pair row of rows i, i+1 of
// the delta w phi_x factors, pb the pair row of phi_v at l, l+1 (both [path][2]):
// q += sum_m (A_i,m B_l,m, A_i+1,m B_l,m, A_i,m B_l+1,m, A_i+1,m B_l+1,m).  FP32: the
// even and odd paths in separate chains, added at the end.
template <typename R>
__device__ __forceinline__ void quad_dot32(const R *pa, const R *pb, R (&q)[4]);
template <>
__device__ __forceinline__ void quad_dot32<float>(const float *pa, const float *pb, float (&q)[4]) {
  float e[4] = {0.f, 0.f, 0.f, 0.f}, o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int j = 0; j < 64; j += 4) {   // paths j/2 and j/2 + 1
    const float4 a = *reinterpret_cast<const float4 *>(pa + j);
    const float4 b = *reinterpret_cast<const float4 *>(pb + j);
    Pr<float>::fma(a.x, a.y, b.x, b.x, e[0], e[1]);
    Pr<float>::fma(a.x, a.y, b.y, b.y, e[2], e[3]);
    Pr<float>::fma(a.z, a.w, b.z, b.z, o[0], o[1]);
    Pr<float>::fma(a.z, a.w, b.w, b.w, o[2], o[3]);
  }
  float t0, t1;
  Pr<float>::add(e[0], e[1], o[0], o[1], t0, t1);
  Pr<float>::add(q[0], q[1], t0, t1, q[0], q[1]);
  Pr<float>::add(e[2], e[3], o[2], o[3], t0, t1);
  Pr<float>::add(q[2], q[3], t0, t1, q[2], q[3]);
}
template <>
__device__ __forceinline__ void quad_dot32<double>(const double *pa, const double *pb, double (&q)[4]) {
#pragma unroll
  for (int j = 0; j < 64; j += 2) {
    const double2 a = *reinterpret_cast<const double2 *>(pa + j);
    const double2 b = *reinterpret_cast<const double2 *>(pb + j);
    q[0] = __fma_rn(a.x, b.x, q[0]);
    q[1] = __fma_rn(a.y, b.x, q[1]);
    q[2] = __fma_rn(a.x, b.y, q[2]);
    q[3] = __fma_rn(a.y, b.y, q[3]);
  }
}

// 2 x 2 weight blocks per lane in the warp exchange.
template <int NX, int NV>
constexpr int fb_qpl() {
  return ((NX / 2) * (NV / 2) + 31) / 32;
}

// One round of the warp exchange: each lane's record (ra = delta w phi_x, rb = phi_v) goes
// into the warp's buffer (pair rows: values of rows c, c+1 interleaved per path), then
// lane p adds the 32-path dot products of its 2 x 2 block of weights (i, i+1) x (l, l+1),
// i/2 = p / (NV/2), l/2 = p % (NV/2), to sq.  Eight consecutive lanes read at most three
// phi_x pair rows and distinct phi_v pair rows (4-bank offsets apart).
template <typename R, int NX, int NV>
__device__ __forceinline__ void fb_exchange_add(R *wa, R *wb, int lane, const R (&ra)[NX], const R (&rb)[NV],
                                                R (&sq)[fb_qpl<NX, NV>()][4]) {
  constexpr int NQ = (NX / 2) * (NV / 2), QPL = fb_qpl<NX, NV>();
#pragma unroll
  for (int c = 0; c < NX; ++c) wa[(c / 2) * FB_AROW + 2 * lane + (c & 1)] = ra[c];
#pragma unroll
  for (int c = 0; c < NV; ++c) wb[(c / 2) * FB_AROW + 2 * lane + (c & 1)] = rb[c];
  __syncwarp();
#pragma unroll
  for (int t = 0; t < QPL; ++t) {
    const int p = lane + 32 * t;
    if (p < NQ) quad_dot32<R>(wa + (p / (NV / 2)) * FB_AROW, wb + (p % (NV / 2)) * FB_AROW, sq[t]);
  }
  __syncwarp();
}

// The warp's partial of one step: block (i/2, l/2) = (p / (NV/2), p % (NV/2)) holds
// weights (i, l), (i+1, l), (i, l+1), (i+1, l+1), contiguous in the pair layout (one
// 16-byte store in FP32).
template <typename R, int NX, int NV>
__device__ __forceinline__ void fb_store_partial(R *dst, int lane, const R (&sq)[fb_qpl<NX, NV>()][4]) {
  constexpr int NQ = (NX / 2) * (NV / 2), QPL = fb_qpl<NX, NV>();
#pragma unroll
  for (int t = 0; t < QPL; ++t) {
    const int p = lane + 32 * t;
    if (p < NQ) {
      R *o = dst + 2 * ((p / (NV / 2)) * NV + 2 * (p % (NV / 2)));
      if constexpr (sizeof(R) == 4) {
        *reinterpret_cast<float4 *>(o) = make_float4(sq[t][0], sq[t][1], sq[t][2], sq[t][3]);
      } else {
        o[0] = sq[t][0];
        o[1] = sq[t][1];
        o[2] = sq[t][2];
        o[3] = sq[t][3];
      }
    }
  }
}

// Shared memory of fb_adj_kernel: per warp NX/2 pair rows of phi_x factors and NV/2 of phi_v.
template <typename R, int NX, int NV>
constexpr size_t fb_adj_smem() {
  return sizeof(R) * (size_t)(FB_TPB / 32) * ((NX / 2) + (NV / 2)) * FB_AROW;
}

template <typename R, int NX, int NV, int RING>
__global__ void __launch_bounds__(FB_TPB)
fb_adj_kernel(const __grid_constant__ KParams<R, 2, 1> kp, const __grid_constant__ FbParams<R> fp,
              const R *__restrict__ mu, const R *__restrict__ xd, const R *__restrict__ traj,
              const uint32_t *__restrict__ flags, R *__restrict__ partW) {
  using M = Ar<R>;
  constexpr int LP = NX * NV, QPL = fb_qpl<NX, NV>();   // 2 x 2 blocks per lane
  constexpr bool CPL = RING > 0;
  extern __shared__ __align__(16) unsigned char fb_smem[];
  __shared__ R ringbuf[RING >= 2 ? 2 * FB_TPB : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  R *wa = reinterpret_cast<R *>(fb_smem) + warp * ((NX / 2) + (NV / 2)) * FB_AROW;
  R *wb = wa + (NX / 2) * FB_AROW;
  const int64_t mloc = fp.mloc, m = (int64_t)blockIdx.x * FB_TPB + threadIdx.x;
  const int64_t wid = (int64_t)blockIdx.x * (FB_TPB / 32) + warp;
  RingX<R, RING> rx;
  rx.sv = ringbuf;
  rx.i = CPL ? (int)(m % fp.S) : 0;
  rx.N = fp.N;
  const bool active = m < mloc && (!CPL || rx.i < fp.N);
  // lanes of the neighbours (their stored states give the coupling force of each step)
  const int64_t mleft = CPL ? m - rx.i + rx.left() : m, mright = CPL ? m - rx.i + rx.right() : m;
  const uint32_t mg = (uint32_t)(kp.m_begin + m);
  const int Nt = fp.Nt;
  R a[2] = {R(0), R(0)};
  if (active) {
    const R zT[2] = {traj[((size_t)Nt * 2) * mloc + m], traj[((size_t)Nt * 2 + 1) * mloc + m]};
    fb_track<R, true>(fp, kp.dt, zT, xd + (size_t)Nt * 2, a);
  }
  // X_k and the flag word of step k are loaded one step ahead (the loop waits on nothing
  // but its own arithmetic)
  R zn[2] = {R(0), R(0)};
  uint32_t fword = 0;
  if (active && Nt > 0) {
    zn[0] = traj[((size_t)(Nt - 1) * 2) * mloc + m];
    zn[1] = traj[((size_t)(Nt - 1) * 2 + 1) * mloc + m];
    fword = flags[(size_t)((Nt - 1) >> 5) * mloc + m];
  }
#pragma unroll 1
  for (int k = Nt - 1; k >= 0; --k) {
    const R *mk = mu + (size_t)k * LP;
    R zk[2] = {zn[0], zn[1]};
    const uint32_t fk = fword;
    if (active && k >= 1) {
      zn[0] = traj[((size_t)(k - 1) * 2) * mloc + m];
      zn[1] = traj[((size_t)(k - 1) * 2 + 1) * mloc + m];
      if ((k & 31) == 0) fword = flags[(size_t)((k - 1) >> 5) * mloc + m];
    }
    int n = 0;
    FbPlan<R> P;
    R Ys[NMAX + 1][2];   // sub-step start states of a step with jumps (Ys[0] = X_k)
    R cin = R(0);
    if constexpr (RING == 1) {   // interacting particles: the neighbours' force of step k
      R xl, xr;
      rx.get(zk[0], xl, xr);
      cin = M::mul(fp.omega, M::add(xl, xr));
    } else if constexpr (CPL) {   // the same from the neighbours' stored states
      if (active)
        cin = M::mul(fp.omega, M::add(traj[((size_t)k * 2) * mloc + mleft], traj[((size_t)k * 2) * mloc + mright]));
    }
    if (active) {
      if ((fk >> (k & 31)) & 1u) {
        // regenerate the step's sub-states from X_k with the forward's arithmetic
        R zs[2], y[2] = {zk[0], zk[1]};
        const uint32_t w0 = main_draws<true>(kp, k, mg, zs);   // round keys of the parameter block
        n = fb_plan(kp, k, mg, w0, P);
#pragma unroll 1
        for (int i = 0; i < n; ++i) {
          const R de = fb_delta(kp, P, n, i);
          fb_substep<R, NX, NV, CPL>(kp, fp, mk, de, Ar<R>::sqrt(de), zs, y, cin);
          R xih[2];
          slot_draws(kp, k, mg, P.order[i], xih, zs);
          apply_jump(kp, y, xih);
          Ys[i + 1][0] = y[0];
          Ys[i + 1][1] = y[1];
        }
      }
    }
    // sub-steps n..0 backwards, round r = sub-step n - r of every path (paths with fewer
    // sub-steps contribute zeros); each round's records (delta w phi_x, phi_v) are summed
    // over the warp's 32 paths through the exchange buffer
    R sq[QPL][4];
#pragma unroll
    for (int t = 0; t < QPL; ++t) sq[t][0] = sq[t][1] = sq[t][2] = sq[t][3] = R(0);
    const int rounds = (int)__reduce_max_sync(0xffffffffu, active ? (unsigned)(n + 1) : 0u);
    R sn = R(0);   // interacting particles: sum over sub-steps of delta a_v (d/d neighbour force)
#pragma unroll 1
    for (int r = 0; r < rounds; ++r) {
      R ra[NX], rb[NV];
      if (active && r <= n) {
        const int i = n - r;
        if (i < n) jump_adjoint(kp, a);   // across the jump that ends sub-step i
        R y[2] = {zk[0], zk[1]};
        R de = kp.dt;
        if (n > 0) {
          de = fb_delta(kp, P, n, i);
          if (i > 0) {
            y[0] = Ys[i][0];
            y[1] = Ys[i][1];
          }
        }
        R ux, uv;
        const R u = fb_eval<R, NX, NV, true>(fp, mk, y[0], y[1], ra, rb, ux, uv);
        const R w = M::fma(kp.B[1], a[1], M::fma(kp.B[0], a[0], M::mul(fp.alpha, u)));
        const R dw = M::mul(de, w);
#pragma unroll
        for (int c = 0; c < NX; ++c) ra[c] = M::mul(dw, ra[c]);
        if (CPL) sn = M::fma(de, a[1], sn);
        adjoint_update(kp, y, de, a);
        a[0] = M::fma(dw, ux, a[0]);
        a[1] = M::fma(dw, uv, a[1]);
      } else {
#pragma unroll
        for (int c = 0; c < NX; ++c) ra[c] = R(0);
#pragma unroll
        for (int c = 0; c < NV; ++c) rb[c] = R(0);
      }
      fb_exchange_add<R, NX, NV>(wa, wb, lane, ra, rb, sq);
    }
    if constexpr (CPL) {   // the neighbour force of particle j drove particles j-1 and j+1
      R sl, sr;
      rx.get(sn, sl, sr);
      if (active) a[0] = M::fma(fp.omega, M::add(sl, sr), a[0]);
    }
    if (active && k >= 1) {
      R g[2];
      fb_track<R, true>(fp, kp.dt, zk, xd + (size_t)k * 2, g);
      a[0] = M::add(a[0], g[0]);
      a[1] = M::add(a[1], g[1]);
    }
    fb_store_partial<R, NX, NV>(partW + ((size_t)wid * Nt + k) * LP, lane, sq);
  }
}

// ---------------------------------------------------------------------------
// Surrogate-state adjoint (Sec. 6.5): the costates run backwards along states drawn
// around the target, zs_k = z_d(t_k) + sqrt(rate t_k) xi (xi: the Box-Muller pair of
// Philox words 0, 1 of counter (k, m, 2 << 24, epoch)), never along the forward's.  The
// adjoint runs first and keeps bhat_k = B^T r (after the Jacobian of the path's own jumps
// of step k) per path and step; the forward sweep then forms the gradient records
// delta phi(Y) (alpha u(Y) + bhat_k) on its own sub-steps, so no state is stored.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void fb_surrogate_state(const KParams<R, 2, 1> &kp, const FbParams<R> &fp, int k,
                                                   uint32_t m, const R *__restrict__ xd, R (&zs)[2]) {
  using M = Ar<R>;
  const uint4 o = philox10((uint32_t)k, m, 2u << 24, kp.epoch, kp.key0, kp.key1);
  R x0, x1;
  normal_pair<R>(o.x, o.y, x0, x1);
  const R sd = M::sqrt(M::mul(fp.srate_dt, (R)k));
  zs[0] = M::fma(sd, x0, __ldg(xd + (size_t)k * 2));
  zs[1] = M::fma(sd, x1, __ldg(xd + (size_t)k * 2 + 1));
}

template <typename R, int NX, int NV>
__global__ void __launch_bounds__(FB_TPB)
fb_sur_adj_kernel(const __grid_constant__ KParams<R, 2, 1> kp, const __grid_constant__ FbParams<R> fp,
                  const R *__restrict__ mu, const R *__restrict__ xd, R *__restrict__ bhat) {
  using M = Ar<R>;
  constexpr int LP = NX * NV;
  const int64_t mloc = fp.mloc, m = (int64_t)blockIdx.x * FB_TPB + threadIdx.x;
  if (m >= mloc) return;
  const uint32_t mg = (uint32_t)(kp.m_begin + m);
  const int Nt = fp.Nt;
  R zs[2], a[2];
  fb_surrogate_state(kp, fp, Nt, mg, xd, zs);
  fb_track<R, true>(fp, kp.dt, zs, xd + (size_t)Nt * 2, a);
#pragma unroll 1
  for (int k = Nt - 1; k >= 0; --k) {
    if (kp.jumps_on) {   // the Jacobian of the step's jumps (gamma per reset on v)
      const uint32_t w0 = philox10((uint32_t)k, mg, 0u, kp.epoch, kp.key0, kp.key1).x;
#pragma unroll 1
      for (int i = 0; i < NMAX && (unsigned long long)w0 >= kp.thr[i]; ++i) jump_adjoint(kp, a);
    }
    const R b = M::fma(kp.B[1], a[1], M::mul(kp.B[0], a[0]));
    bhat[(size_t)k * mloc + m] = b;
    fb_surrogate_state(kp, fp, k, mg, xd, zs);
    R px[NX], pv[NV], ux, uv;
    const R u = fb_eval<R, NX, NV, true>(fp, mu + (size_t)k * LP, zs[0], zs[1], px, pv, ux, uv);
    const R dw = M::mul(kp.dt, M::fma(fp.alpha, u, b));
    adjoint_update(kp, zs, kp.dt, a);
    a[0] = M::fma(dw, ux, a[0]);
    a[1] = M::fma(dw, uv, a[1]);
    if (k >= 1) {
      R g[2];
      fb_track<R, true>(fp, kp.dt, zs, xd + (size_t)k * 2, g);
      a[0] = M::add(a[0], g[0]);
      a[1] = M::add(a[1], g[1]);
    }
  }
}

// Forward sweep of the surrogate gradient: the path cost as fb_fwd_kernel, and per step
// the records delta_i phi(Y_i) (alpha u(Y_i) + bhat_k) of every sub-step, summed over the
// warp by the exchange into partW.  Sub-steps run in rounds across the warp (a path with
// n jumps takes n + 1 rounds).
template <typename R, int NX, int NV>
__global__ void __launch_bounds__(FB_TPB)
fb_fwd_sur_kernel(const __grid_constant__ KParams<R, 2, 1> kp, const __grid_constant__ FbParams<R> fp,
                  const R *__restrict__ mu, const R *__restrict__ xd, const R *__restrict__ bhat,
                  double *__restrict__ partC, R *__restrict__ partW) {
  using M = Ar<R>;
  constexpr int LP = NX * NV, QPL = fb_qpl<NX, NV>();
  extern __shared__ __align__(16) unsigned char fb_smem[];
  __shared__ Pair<R> red[FB_TPB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  R *wa = reinterpret_cast<R *>(fb_smem) + warp * ((NX / 2) + (NV / 2)) * FB_AROW;
  R *wb = wa + (NX / 2) * FB_AROW;
  const int64_t mloc = fp.mloc, m = (int64_t)blockIdx.x * FB_TPB + threadIdx.x;
  const int64_t wid = (int64_t)blockIdx.x * (FB_TPB / 32) + warp;
  const bool active = m < mloc;
  const uint32_t mg = (uint32_t)(kp.m_begin + m);
  const int Nt = fp.Nt;
  Kahan<R> cost;
  R z[2] = {kp.x0[0], kp.x0[1]};
#pragma unroll 1
  for (int k = 0; k < Nt; ++k) {
    const R *mk = mu + (size_t)k * LP;
    R zs[2] = {R(0), R(0)};
    int n = 0;
    FbPlan<R> P;
    R bk = R(0);
    if (active) {
      const uint32_t w0 = main_draws<true>(kp, k, mg, zs);   // round keys of the parameter block
      if (has_jump(kp, w0)) n = fb_plan(kp, k, mg, w0, P);
      bk = bhat[(size_t)k * mloc + m];
    }
    R sq[QPL][4];
#pragma unroll
    for (int t = 0; t < QPL; ++t) sq[t][0] = sq[t][1] = sq[t][2] = sq[t][3] = R(0);
    const int rounds = (int)__reduce_max_sync(0xffffffffu, active ? (unsigned)(n + 1) : 0u);
#pragma unroll 1
    for (int r = 0; r < rounds; ++r) {
      R ra[NX], rb[NV];
      if (active && r <= n) {
        R de = kp.dt, sqd = kp.sqdt;
        if (n > 0) {
          de = fb_delta(kp, P, n, r);
          sqd = M::sqrt(de);
        }
        R ux, uv;
        const R u = fb_eval<R, NX, NV, false>(fp, mk, z[0], z[1], ra, rb, ux, uv);
        const R dw = M::mul(de, M::fma(fp.alpha, u, bk));
#pragma unroll
        for (int c = 0; c < NX; ++c) ra[c] = M::mul(dw, ra[c]);
        cost.add(M::mul(M::mul(fp.halpha, de), M::mul(u, u)));
        const R uu[1] = {u};
        R f[2];
        drift(kp, z, uu, f);
#pragma unroll
        for (int c = 0; c < 2; ++c) z[c] = M::fma(M::mul(kp.sigma[c], sqd), zs[c], M::fma(de, f[c], z[c]));
        if (r < n) {
          R xih[2];
          slot_draws(kp, k, mg, P.order[r], xih, zs);
          apply_jump(kp, z, xih);
        }
      } else {
#pragma unroll
        for (int c = 0; c < NX; ++c) ra[c] = R(0);
#pragma unroll
        for (int c = 0; c < NV; ++c) rb[c] = R(0);
      }
      fb_exchange_add<R, NX, NV>(wa, wb, lane, ra, rb, sq);
    }
    if (active) {
      R g[2];
      cost.add(fb_track<R, false>(fp, kp.dt, z, xd + (size_t)(k + 1) * 2, g));
    }
    fb_store_partial<R, NX, NV>(partW + ((size_t)wid * Nt + k) * LP, lane, sq);
  }
  const double bs = fb_block_sum(active ? cost.pair() : Pair<R>{R(0), R(0)}, red);
  if (threadIdx.x == 0) partC[blockIdx.x] = bs;
}

// partG[g][c] = sum over warps w of group g (in order) of partW[w][c]; one thread per
// group and four consecutive columns (16-byte loads in FP32), consecutive threads on
// consecutive columns.  FP32 partials are added as compensated FP32 pairs (TwoSum: FP64
// adds are scarce on this part) and the pair is rounded to FP64 once per group; FP64
// partials are added in FP64.  ncol is a multiple of 4 (NX NV is 16, 100 or 256).
template <typename R>
__global__ void fb_reduce_kernel(const R *__restrict__ partW, int64_t nwarp, int64_t ncol,
                                 double *__restrict__ partG) {
  const int64_t ngroup = (nwarp + FB_GROUP_WARPS - 1) / FB_GROUP_WARPS, nc4 = ncol / 4;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ngroup * nc4;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = t / nc4, c = 4 * (t - g * nc4);
    const int64_t w1 = std::min<int64_t>(nwarp, (g + 1) * FB_GROUP_WARPS);
    double *o = partG + g * ncol + c;
    if constexpr (sizeof(R) == 4) {
      Pair<float> s0{0.f, 0.f}, s1{0.f, 0.f}, s2{0.f, 0.f}, s3{0.f, 0.f};
#pragma unroll 8
      for (int64_t w = g * FB_GROUP_WARPS; w < w1; ++w) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(partW + w * ncol + c));
        s0 = padd(s0, Pair<float>{v.x, 0.f});
        s1 = padd(s1, Pair<float>{v.y, 0.f});
        s2 = padd(s2, Pair<float>{v.z, 0.f});
        s3 = padd(s3, Pair<float>{v.w, 0.f});
      }
      o[0] = (double)s0.s + (double)s0.e;
      o[1] = (double)s1.s + (double)s1.e;
      o[2] = (double)s2.s + (double)s2.e;
      o[3] = (double)s3.s + (double)s3.e;
    } else {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll 4
      for (int64_t w = g * FB_GROUP_WARPS; w < w1; ++w) {
        const R *q = partW + w * ncol + c;
        const double2 v = __ldg(reinterpret_cast<const double2 *>(q)), u = __ldg(reinterpret_cast<const double2 *>(q) + 1);
        s0 += v.x;
        s1 += v.y;
        s2 += u.x;
        s3 += u.y;
      }
      o[0] = s0;
      o[1] = s1;
      o[2] = s2;
      o[3] = s3;
    }
  }
}

// mu (FP64, [Nt][nx][nv]) -> kernel precision [Nt][NX/2][NV][2] (rows i, i+1
// interleaved), zero beyond nx, nv.
template <typename R>
__global__ void fb_prep_mu_kernel(const double *__restrict__ mu, R *__restrict__ out, int Nt, int nx, int nv,
                                  int NX, int NV) {
  const int64_t n = (int64_t)Nt * NX * NV;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t / (NX * NV);
    const int r = (int)(t - k * NX * NV), e = r & 1, pl = r >> 1, ip = pl / NV, l = pl - ip * NV;
    const int i = 2 * ip + e;
    out[t] = (i < nx && l < nv) ? (R)mu[(k * nx + i) * nv + l] : R(0);
  }
}

// J = (1/M) sum_b partC[b];  grad[k][i][l] = (1/M) sum_g partG[g][k][2 (i/2 NV + l) + i%2],
// groups in order.
__global__ void fb_finalize_kernel(const double *__restrict__ partC, const double *__restrict__ partG,
                                   int64_t nblk, int64_t ngroup, int Nt, int nx, int nv, int NX, int NV,
                                   int64_t M, double *__restrict__ J, double *__restrict__ grad);

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
template <typename R>
void fb_make_params(const ::jd_problem *p, const jd_feedback_desc &fb, FbParams<R> &fp) {
  const double dx = 2.0 * fb.x_max / fb.nx, dv = 2.0 * fb.v_max / fb.nv;   // cell widths (Sec. 5.1)
  fp.xc0 = (R)(0.5 * dx - fb.x_max);
  fp.dxc = (R)dx;
  fp.vc0 = (R)(0.5 * dv - fb.v_max);
  fp.dvc = (R)dv;
  fp.eps2 = (R)(fb.eps * fb.eps);
  fp.m2eps2 = (R)(-2.0 * fb.eps * fb.eps);
  fp.alpha = (R)p->desc.nu;
  fp.halpha = (R)(0.5 * p->desc.nu);
  fp.q[0] = (R)p->q[0];
  fp.q[1] = (R)p->q[1];
  const double s2 = fb.track == JD_TRACK_GAUSS ? fb.sigma_J * fb.sigma_J : 1.0;
  fp.hinv_s2 = (R)(0.5 / s2);
  fp.inv_s2 = (R)(1.0 / s2);
  fp.gauss = fb.track == JD_TRACK_GAUSS;
  fp.srate_dt = (R)(fb.adjoint == JD_FB_SURROGATE ? fb.sur_rate * (p->desc.T / p->desc.Nt) : 0.0);
  fp.ellipse = fb.track == JD_TRACK_ELLIPSE;
  fp.iax2 = (R)(fb.track == JD_TRACK_ELLIPSE || fb.particles ? 1.0 / (fb.ax * fb.ax) : 0.0);
  fp.iav2 = (R)(fb.track == JD_TRACK_ELLIPSE || fb.particles ? 1.0 / (fb.av * fb.av) : 0.0);
  fp.N = fb.particles;
  fp.S = fb.particles ? ring_lanes(fb.particles) : 0;
  fp.omega = (R)fb.omega;
  fp.z0 = static_cast<const R *>(p->fb_z0);   // the ring's initial states (fb_upload_ring)
  fp.Nt = p->desc.Nt;
  fp.mloc = p->desc.M;
}

// Kernel coefficients of a feedback problem: for interacting particles the particle's own
// share of the ring coupling, -2 omega x_i, joins its drift matrix (A[1][0]).
template <typename R>
void fb_make_kparams(const ::jd_problem *p, const jd_feedback_desc &fb, KParams<R, 2, 1> &kp) {
  make_kparams<R, 2, 1>(p, 0, p->desc.M, kp);
  if (fb.particles) kp.A[2] = (R)(p->A[2] - 2.0 * fb.omega);
}

// Launch of a feedback kernel; a ring of more than 256 lanes (RING 3) runs as one
// thread-block cluster of S / 256 blocks.
template <typename... KArgs, typename... Args>
cudaError_t fb_launch(void (*kern)(KArgs...), int ring, int S, unsigned grid, size_t smem, cudaStream_t s,
                      Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(FB_TPB);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  if (ring == 3) {
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)(S / FB_TPB);
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
  }
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename R, int NX, int NV, bool STORE, int RING>
cudaError_t fb_fwd_ring(const KParams<R, 2, 1> &kp, const FbParams<R> &fp, const R *mu, const R *xd, R *traj,
                        uint32_t *flags, double *partC, unsigned grid, cudaStream_t s) {
  return fb_launch(fb_fwd_kernel<R, NX, NV, STORE, RING>, RING, fp.S, grid, 0, s, kp, fp, mu, xd, traj, flags,
                   partC);
}

template <typename R, int NX, int NV>
cudaError_t fb_fwd_launch(const ::jd_problem *p, const jd_feedback_desc &fb, bool store, const FbBufs &b,
                          cudaStream_t s) {
  KParams<R, 2, 1> kp;
  fb_make_kparams<R>(p, fb, kp);
  FbParams<R> fp;
  fb_make_params<R>(p, fb, fp);
  const unsigned grid = (unsigned)ceil_div(p->desc.M, FB_TPB);
  const R *mu = static_cast<const R *>(b.mu), *xd = static_cast<const R *>(p->xdk);
  R *traj = store ? static_cast<R *>(b.traj) : nullptr;
  uint32_t *flags = store ? b.flags : nullptr;
  switch (ring_kind(fb.particles) * 2 + (store ? 1 : 0)) {
    case 0: return fb_fwd_ring<R, NX, NV, false, 0>(kp, fp, mu, xd, traj, flags, b.partC, grid, s);
    case 1: return fb_fwd_ring<R, NX, NV, true, 0>(kp, fp, mu, xd, traj, flags, b.partC, grid, s);
    case 2: return fb_fwd_ring<R, NX, NV, false, 1>(kp, fp, mu, xd, traj, flags, b.partC, grid, s);
    case 3: return fb_fwd_ring<R, NX, NV, true, 1>(kp, fp, mu, xd, traj, flags, b.partC, grid, s);
    case 4: return fb_fwd_ring<R, NX, NV, false, 2>(kp, fp, mu, xd, traj, flags, b.partC, grid, s);
    case 5: return fb_fwd_ring<R, NX, NV, true, 2>(kp, fp, mu, xd, traj, flags, b.partC, grid, s);
    case 6: return fb_fwd_ring<R, NX, NV, false, 3>(kp, fp, mu, xd, traj, flags, b.partC, grid, s);
    default: return fb_fwd_ring<R, NX, NV, true, 3>(kp, fp, mu, xd, traj, flags, b.partC, grid, s);
  }
}

template <typename R, int NX, int NV, int RING>
cudaError_t fb_adj_ring(const KParams<R, 2, 1> &kp, const FbParams<R> &fp, const FbBufs &b, const R *xd,
                        unsigned grid, cudaStream_t s) {
  constexpr size_t smem = fb_adj_smem<R, NX, NV>();
  static_assert(smem <= 232448, "fb_adj_kernel shared memory");
  const cudaError_t e = ensure_dyn_smem((const void *)fb_adj_kernel<R, NX, NV, RING>, smem);
  if (e != cudaSuccess) return e;
  return fb_launch(fb_adj_kernel<R, NX, NV, RING>, RING, fp.S, grid, smem, s, kp, fp,
                   static_cast<const R *>(b.mu), xd, static_cast<const R *>(b.traj),
                   static_cast<const uint32_t *>(b.flags), static_cast<R *>(b.partW));
}

// The adjoint sweep (warp partials of the gradient).
template <typename R, int NX, int NV>
cudaError_t fb_adj_launch(const ::jd_problem *p, const jd_feedback_desc &fb, const FbBufs &b, cudaStream_t s) {
  KParams<R, 2, 1> kp;
  fb_make_kparams<R>(p, fb, kp);
  FbParams<R> fp;
  fb_make_params<R>(p, fb, fp);
  const unsigned grid = (unsigned)ceil_div(p->desc.M, FB_TPB);
  const R *xd = static_cast<const R *>(p->xdk);
  switch (ring_kind(fb.particles)) {
    case 0: return fb_adj_ring<R, NX, NV, 0>(kp, fp, b, xd, grid, s);
    case 1: return fb_adj_ring<R, NX, NV, 1>(kp, fp, b, xd, grid, s);
    case 2: return fb_adj_ring<R, NX, NV, 2>(kp, fp, b, xd, grid, s);
    default: return fb_adj_ring<R, NX, NV, 3>(kp, fp, b, xd, grid, s);
  }
}

// Surrogate gradient (Sec. 6.5): the surrogate adjoint writes bhat, then the forward
// sweep forms the cost and the warp partials of the gradient.
template <typename R, int NX, int NV>
cudaError_t fb_sur_launch(const ::jd_problem *p, const jd_feedback_desc &fb, const FbBufs &b, cudaStream_t s) {
  KParams<R, 2, 1> kp;
  make_kparams<R, 2, 1>(p, 0, p->desc.M, kp);
  FbParams<R> fp;
  fb_make_params<R>(p, fb, fp);
  const unsigned grid = (unsigned)ceil_div(p->desc.M, FB_TPB);
  const R *mu = static_cast<const R *>(b.mu), *xd = static_cast<const R *>(p->xdk);
  fb_sur_adj_kernel<R, NX, NV><<<grid, FB_TPB, 0, s>>>(kp, fp, mu, xd, static_cast<R *>(b.traj));
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  constexpr size_t smem = fb_adj_smem<R, NX, NV>();
  e = cudaFuncSetAttribute(fb_fwd_sur_kernel<R, NX, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fb_fwd_sur_kernel<R, NX, NV><<<grid, FB_TPB, smem, s>>>(kp, fp, mu, xd, static_cast<const R *>(b.traj), b.partC,
                                                          static_cast<R *>(b.partW));
  count_launch();
  return cudaGetLastError();
}

// First stage of the gradient reduction: warp partials -> FP64 group partials.
template <typename R, int NX, int NV>
cudaError_t fb_reduce_launch(const ::jd_problem *p, const FbBufs &b, cudaStream_t s) {
  const int64_t nwarp = ceil_div(p->desc.M, FB_TPB) * (FB_TPB / 32), ncol = (int64_t)p->desc.Nt * NX * NV;
  const int64_t n = fb_groups(nwarp) * (ncol / 4);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 152 * 16));
  fb_reduce_kernel<R><<<grid, 256, 0, s>>>(static_cast<const R *>(b.partW), nwarp, ncol, b.partG);
  count_launch();
  return cudaGetLastError();
}

template <typename R, int NX, int NV>
cudaError_t fb_prep_dims(const double *mu64, void *muR, int Nt, int nx, int nv, cudaStream_t s) {
  const int64_t n = (int64_t)Nt * NX * NV;
  const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n, 256), 4096);
  fb_prep_mu_kernel<R><<<grid, 256, 0, s>>>(mu64, static_cast<R *>(muR), Nt, nx, nv, NX, NV);
  count_launch();
  return cudaGetLastError();
}

template <typename R, int NX, int NV>
size_t fb_stack_bytes() {
  static const size_t bytes = [] {   // the kernels' attributes do not change: ask once
    size_t need = 0;
    const void *ks[] = {(const void *)fb_fwd_kernel<R, NX, NV, false, 0>, (const void *)fb_fwd_kernel<R, NX, NV, true, 0>,
                        (const void *)fb_fwd_kernel<R, NX, NV, false, 1>, (const void *)fb_fwd_kernel<R, NX, NV, true, 1>,
                        (const void *)fb_fwd_kernel<R, NX, NV, false, 2>, (const void *)fb_fwd_kernel<R, NX, NV, true, 2>,
                        (const void *)fb_fwd_kernel<R, NX, NV, false, 3>, (const void *)fb_fwd_kernel<R, NX, NV, true, 3>,
                        (const void *)fb_adj_kernel<R, NX, NV, 0>, (const void *)fb_adj_kernel<R, NX, NV, 1>,
                        (const void *)fb_adj_kernel<R, NX, NV, 2>, (const void *)fb_adj_kernel<R, NX, NV, 3>,
                        (const void *)fb_sur_adj_kernel<R, NX, NV>, (const void *)fb_fwd_sur_kernel<R, NX, NV>};
    for (const void *k : ks) {
      cudaFuncAttributes a;
      if (cudaFuncGetAttributes(&a, k) == cudaSuccess) need = std::max(need, a.localSizeBytes);
    }
    need += 2048;
    return (need + 255) & ~(size_t)255;
  }();
  return bytes;
}

template <typename R, int NX, int NV>
constexpr FbOps fb_make_ops() {
  return FbOps{NX, NV, (int)sizeof(R), &fb_stack_bytes<R, NX, NV>, &fb_fwd_launch<R, NX, NV>,
               &fb_adj_launch<R, NX, NV>, &fb_sur_launch<R, NX, NV>, &fb_reduce_launch<R, NX, NV>,
               &fb_prep_dims<R, NX, NV>};
}

}  // namespace jd
