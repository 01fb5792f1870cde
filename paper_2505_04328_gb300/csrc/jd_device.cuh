// jd_device.cuh -- device primitives of the path kernels (sm_103a).
//
//  * Philox4x32-10 (Salmon et al., SC'11), written from its published definition.
//  * Uniform ((w >> 9) + 1/2) 2^-23, exact in FP32 and FP64, never 0 or 1.
//  * Box-Muller pairs (first word: radius, second: angle) with the CUDA math
//    library's logf/sqrtf/sincospif (or the double versions).
//  * Compensated (TwoSum) pairs for every cross-path sum, reduced by a transposed
//    warp butterfly (one shuffle per path-step) and then across the block.
//  * One Euler-Maruyama step of the jump-adapted scheme (Algorithm 5.1) and its
//    exact adjoint (eq:AdjointModel read as the derivative of the discrete cost).
//
// All state arithmetic uses explicit round-to-nearest intrinsics (__fmaf_rn,
// __fmul_rn, __fadd_rn ...), so the compiler cannot contract or reorder it and the
// stored and recomputed sweeps produce the same bits.
#pragma once

#include <cstdint>

#include "jd_internal.h"

namespace jd {

// ---------------------------------------------------------------------------
// Philox4x32-10
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                          uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c0;   // one wide multiply
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c2;
    const uint32_t y0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0, y2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c0 = y0;
    c1 = (uint32_t)p1;
    c2 = y2;
    c3 = (uint32_t)p0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}

// The same generator with the ten round keys given (rk0[r] = k0 + r 0x9E3779B9, rk1[r] =
// k1 + r 0xBB67AE85): from a kernel's parameter block each XOR takes its key as a
// constant operand, and no key is bumped per block.
__device__ __forceinline__ uint4 philox10_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                             const uint32_t (&rk0)[10], const uint32_t (&rk1)[10]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c0;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c2;
    const uint32_t y0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk0[r], y2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk1[r];
    c0 = y0;
    c1 = (uint32_t)p1;
    c2 = y2;
    c3 = (uint32_t)p0;
  }
  return make_uint4(c0, c1, c2, c3);
}

// ---------------------------------------------------------------------------
// Precision-generic arithmetic with fixed rounding
// ---------------------------------------------------------------------------
template <typename R>
struct Ar;

template <>
struct Ar<float> {
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float sqrt(float a) { return __fsqrt_rn(a); }
  static __device__ __forceinline__ float log(float a) { return logf(a); }
  static __device__ __forceinline__ void sincospi(float a, float *s, float *c) { sincospif(a, s, c); }
  static __device__ __forceinline__ float u01(uint32_t w) {
    return __fmaf_rn(__uint2float_rn(w >> 9), 0x1p-23f, 0x1p-24f);
  }
};

template <>
struct Ar<double> {
  static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double sqrt(double a) { return __dsqrt_rn(a); }
  static __device__ __forceinline__ double log(double a) { return ::log(a); }
  static __device__ __forceinline__ void sincospi(double a, double *s, double *c) { ::sincospi(a, s, c); }
  static __device__ __forceinline__ double u01(uint32_t w) {
    return __fma_rn((double)(w >> 9), 0x1p-23, 0x1p-24);
  }
};

// ---------------------------------------------------------------------------
// Paired FP32 arithmetic: two independent lanes of a vector in one FFMA2 / FMUL2 (sm_100
// and later).  Per component the rounding is that of __fmaf_rn / __fmul_rn, so the
// paired and scalar forms give the same bits; FP64 stays scalar.
// ---------------------------------------------------------------------------
template <typename R>
struct Pr {
  static constexpr bool on = false;
};
template <>
struct Pr<float> {
  static constexpr bool on = true;
  static __device__ __forceinline__ void fma(float a0, float a1, float b0, float b1, float &c0, float &c1) {
    const float2 r = __ffma2_rn(make_float2(a0, a1), make_float2(b0, b1), make_float2(c0, c1));
    c0 = r.x;
    c1 = r.y;
  }
  static __device__ __forceinline__ void mul(float a0, float a1, float b0, float b1, float &r0, float &r1) {
    const float2 r = __fmul2_rn(make_float2(a0, a1), make_float2(b0, b1));
    r0 = r.x;
    r1 = r.y;
  }
  static __device__ __forceinline__ void add(float a0, float a1, float b0, float b1, float &r0, float &r1) {
    const float2 r = __fadd2_rn(make_float2(a0, a1), make_float2(b0, b1));
    r0 = r.x;
    r1 = r.y;
  }
  // a - b as a + (-b): the same IEEE operation, so the same bits as __fsub_rn
  static __device__ __forceinline__ void sub(float a0, float a1, float b0, float b1, float &r0, float &r1) {
    const float2 r = __fadd2_rn(make_float2(a0, a1), make_float2(-b0, -b1));
    r0 = r.x;
    r1 = r.y;
  }
};

template <typename R>
__device__ __forceinline__ void normal_pair(uint32_t wa, uint32_t wb, R &z0, R &z1) {
  using M = Ar<R>;
  const R ua = M::u01(wa), ub = M::u01(wb);
  const R r = M::sqrt(M::mul(R(-2), M::log(ua)));
  R s, c;
  M::sincospi(M::mul(R(2), ub), &s, &c);
  if constexpr (Pr<R>::on) {
    Pr<R>::mul(r, r, c, s, z0, z1);
  } else {
    z0 = M::mul(r, c);
    z1 = M::mul(r, s);
  }
}

// ---------------------------------------------------------------------------
// Compensated sums: (s, e) with the true value s + e; TwoSum keeps every addition
// exact up to the final rounding of e.
// ---------------------------------------------------------------------------
template <typename R>
struct Pair {
  R s, e;
};

template <typename R>
__device__ __forceinline__ Pair<R> padd(Pair<R> a, Pair<R> b) {
  using M = Ar<R>;
  const R s = M::add(a.s, b.s);
  const R bb = M::sub(s, a.s);
  const R err = M::add(M::sub(a.s, M::sub(s, bb)), M::sub(b.s, bb));
  return {s, M::add(M::add(a.e, b.e), err)};
}

template <typename R>
__device__ __forceinline__ Pair<R> shfl_xor(Pair<R> v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.s, o), __shfl_xor_sync(0xffffffffu, v.e, o)};
}

template <typename R>
__device__ __forceinline__ Pair<R> warp_sum(Pair<R> v) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v = padd(v, shfl_xor(v, o));
  return v;
}

// Kahan accumulator for one path's running cost (true sum s - c).
template <typename R>
struct Kahan {
  R s = R(0), c = R(0);
  __device__ __forceinline__ void add(R term) {
    using M = Ar<R>;
    const R y = M::sub(term, c);
    const R t = M::add(s, y);
    c = M::sub(M::sub(t, s), y);
    s = t;
  }
  __device__ __forceinline__ Pair<R> pair() const { return {s, -c}; }
};

// Block sum of one pair per thread into a double; thread 0 returns the result.
template <typename R>
__device__ __forceinline__ double block_sum_to_double(Pair<R> v, Pair<R> *smem /* >= TPB/32 */) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  double out = 0.0;
  if (threadIdx.x == 0) {
    Pair<R> s = smem[0];
    for (int w = 1; w < TPB / 32; ++w) s = padd(s, smem[w]);
    out = (double)s.s + (double)s.e;
  }
  __syncthreads();
  return out;
}

// Transposed warp reduction of B steps (B = BATCH = 8): every lane holds one value
// per step; after the butterfly lanes with (lane & 3) == 0 hold the 32-lane sum of
// step j = 4*bit4 + 2*bit3 + bit2 of the lane index.  Uses B - 1 + 2 shuffles for B
// steps (about one per path-step).
template <typename R>
__device__ __forceinline__ Pair<R> warp_transpose_sum8(Pair<R> (&v)[BATCH], int lane) {
#pragma unroll
  for (int c = BATCH, o = 16; c > 1; c >>= 1, o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < c / 2; ++i) {
      const Pair<R> send = upper ? v[i] : v[i + c / 2];
      const Pair<R> keep = upper ? v[i + c / 2] : v[i];
      v[i] = padd(keep, shfl_xor(send, o));
    }
  }
  Pair<R> r = v[0];
  r = padd(r, shfl_xor(r, 2));
  r = padd(r, shfl_xor(r, 1));
  return r;
}

__device__ __forceinline__ int transposed_step_of_lane(int lane) {
  return ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
}

// One batch of per-step gradient contributions gb[j][l] (steps kbase + j) summed over
// the warp's 32 paths (compensated) and written as one FP64 partial per warp:
// partG[(k*DU + l) * npart + warp_id], npart = blocks * TPB/32.  No block barrier.
template <typename R, int DU>
__device__ __forceinline__ void reduce_batch(Pair<R> (&gb)[BATCH][DU], int kbase, int Nt,
                                             double *__restrict__ partG, int64_t npart) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (int64_t)blockIdx.x * (TPB / 32) + (threadIdx.x >> 5);
#pragma unroll
  for (int l = 0; l < DU; ++l) {
    Pair<R> v[BATCH];
#pragma unroll
    for (int j = 0; j < BATCH; ++j) v[j] = gb[j][l];
    const Pair<R> r = warp_transpose_sum8(v, lane);
    const int k = kbase + transposed_step_of_lane(lane);
    if ((lane & 3) == 0 && k < Nt) partG[((int64_t)k * DU + l) * npart + wid] = (double)r.s + (double)r.e;
  }
}

// ---------------------------------------------------------------------------
// Per-warp rows of per-step gradient contributions (the adjoint kernels of d <= 8).
// Every lane writes its path's contribution of step k to row k mod NR (one shared store
// per step).  Every NR steps the rows become one FP64 partial per (step, control, warp),
// partG[(k DU + l) npart + warp_id], with no block barrier:
//   NR = 16: lane l sums row l/2 over lanes 16 (l % 2) .. +15, one shuffle joins the
//            halves (fewer instructions per step);
//   NR = 8:  lane l sums row l/4 over lanes 8 (l % 4) .. +7, two shuffles join the
//            quarters (half the shared memory).
// Both evaluate the same tree of compensated (TwoSum) pairs over the warp's lanes
// (L_i = lane i), so a kernel may take either and the gradient keeps its bits:
//     a_q = L4q + L4q+2, b_q = L4q+1 + L4q+3                      (q = 0..7)
//     c_h = a_4h + a_4h+1, d_h = b_4h + b_4h+1                   (quarters, h = 0..3)
//     e_H = c_2H + c_2H+1, f_H = d_2H + d_2H+1;  s_H = e_H + f_H   (halves, H = 0, 1)
//     sum = s_0 + s_1
// Row stride 36 values, the second half of a double row moved by 2 values: the row
// stores and the 16-byte row reads are free of bank conflicts.
// ---------------------------------------------------------------------------
template <typename R>
struct RowGeom {
  static constexpr int LD = 36;                          // values per row
  static constexpr int HALF = sizeof(R) == 8 ? 18 : 16;   // column of lane 16
};

template <typename R, int DU, int NR>
__host__ __device__ constexpr size_t grad_rows_bytes() {   // per block
  return (size_t)(TPB / 32) * DU * NR * RowGeom<R>::LD * sizeof(R);
}

// TwoSum of two pairs (a, b) with zero error terms, two lanes at once (FP32: one FADD2
// per operation; FP64: scalar).  Per component the operations of padd.
template <typename R>
__device__ __forceinline__ void two_sum2(R a0, R a1, R b0, R b1, Pair<R> &r0, Pair<R> &r1) {
  if constexpr (Pr<R>::on) {
    R s0, s1, bb0, bb1, t0, t1, u0, u1, v0, v1, e0, e1;
    Pr<R>::add(a0, a1, b0, b1, s0, s1);
    Pr<R>::sub(s0, s1, a0, a1, bb0, bb1);
    Pr<R>::sub(s0, s1, bb0, bb1, t0, t1);
    Pr<R>::sub(a0, a1, t0, t1, u0, u1);
    Pr<R>::sub(b0, b1, bb0, bb1, v0, v1);
    Pr<R>::add(u0, u1, v0, v1, e0, e1);
    r0 = {s0, e0};
    r1 = {s1, e1};
  } else {
    r0 = padd(Pair<R>{a0, R(0)}, Pair<R>{b0, R(0)});
    r1 = padd(Pair<R>{a1, R(0)}, Pair<R>{b1, R(0)});
  }
}

// padd of two independent pairs of pairs: r0 = a0 + b0, r1 = a1 + b1.
template <typename R>
__device__ __forceinline__ void padd2(Pair<R> a0, Pair<R> a1, Pair<R> b0, Pair<R> b1, Pair<R> &r0, Pair<R> &r1) {
  if constexpr (Pr<R>::on) {
    R s0, s1, bb0, bb1, t0, t1, u0, u1, v0, v1, e0, e1, w0, w1, x0, x1;
    Pr<R>::add(a0.s, a1.s, b0.s, b1.s, s0, s1);
    Pr<R>::sub(s0, s1, a0.s, a1.s, bb0, bb1);
    Pr<R>::sub(s0, s1, bb0, bb1, t0, t1);
    Pr<R>::sub(a0.s, a1.s, t0, t1, u0, u1);
    Pr<R>::sub(b0.s, b1.s, bb0, bb1, v0, v1);
    Pr<R>::add(u0, u1, v0, v1, e0, e1);
    Pr<R>::add(a0.e, a1.e, b0.e, b1.e, w0, w1);
    Pr<R>::add(w0, w1, e0, e1, x0, x1);
    r0 = {s0, x0};
    r1 = {s1, x1};
  } else {
    r0 = padd(a0, b0);
    r1 = padd(a1, b1);
  }
}

// Row values at cols c0 .. c0 + N - 1 (16-byte reads).
template <typename R, int N>
__device__ __forceinline__ void row_read(const R *src, R (&v)[N]) {
  if constexpr (sizeof(R) == 4) {
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
      const float4 t = reinterpret_cast<const float4 *>(src)[q];
      v[4 * q] = t.x;
      v[4 * q + 1] = t.y;
      v[4 * q + 2] = t.z;
      v[4 * q + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < N / 2; ++q) {
      const double2 t = reinterpret_cast<const double2 *>(src)[q];
      v[2 * q] = t.x;
      v[2 * q + 1] = t.y;
    }
  }
}

template <typename R, int DU, int NR = 16>
struct GradRows {
  static_assert(NR == 8 || NR == 16, "8 or 16 rows");
  R *w;   // this warp's rows [DU][NR][LD]
  __device__ __forceinline__ void init(R *block_rows) {
    w = block_rows + (size_t)(threadIdx.x >> 5) * DU * NR * RowGeom<R>::LD;
  }
  static __device__ __forceinline__ int col(int lane) { return lane + (lane >> 4) * (RowGeom<R>::HALF - 16); }
  // contribution g of the step in row j (= k mod NR); inactive lanes add 0
  __device__ __forceinline__ void put(int j, const R (&g)[DU], bool active) {
    const int c = col(threadIdx.x & 31);
#pragma unroll
    for (int l = 0; l < DU; ++l) w[(l * NR + j) * RowGeom<R>::LD + c] = active ? g[l] : R(0);
  }
  // rows of steps kbase .. kbase + NR - 1 (those < Nt) -> FP64 warp partials; bid: the
  // block's index within its problem's launch
  __device__ __forceinline__ void flush(int kbase, int Nt, double *__restrict__ partG, int64_t npart,
                                        int64_t bid) {
    __syncwarp();
    const int lane = threadIdx.x & 31;
    const int64_t wid = bid * (TPB / 32) + (threadIdx.x >> 5);
    constexpr int SPAN = 32 / (32 / NR);   // lanes summed by one reader: 16 or 8
    const int r = lane / (32 / NR), part = lane % (32 / NR);
#pragma unroll
    for (int l = 0; l < DU; ++l) {
      R v[SPAN];
      row_read<R, SPAN>(w + (l * NR + r) * RowGeom<R>::LD + col(part * SPAN), v);
      Pair<R> a[SPAN / 4], b[SPAN / 4];
#pragma unroll
      for (int q = 0; q < SPAN / 4; ++q) two_sum2(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3], a[q], b[q]);
      Pair<R> c0, d0, e, f;
      padd2(a[0], b[0], a[1], b[1], c0, d0);
      if constexpr (NR == 16) {
        Pair<R> c1, d1;
        padd2(a[2], b[2], a[3], b[3], c1, d1);
        padd2(c0, d0, c1, d1, e, f);
      } else {
        padd2(c0, d0, shfl_xor(c0, 1), shfl_xor(d0, 1), e, f);
      }
      Pair<R> s = padd(e, f);
      s = padd(s, shfl_xor(s, 32 / NR / 2));
      const int k = kbase + r;
      if (part == 0 && k < Nt) partG[((int64_t)k * DU + l) * npart + wid] = (double)s.s + (double)s.e;
    }
    __syncwarp();
  }
};

// ---------------------------------------------------------------------------
// Model: drift f = A x + C x^3 + B u and its transposed Jacobian
// ---------------------------------------------------------------------------
template <typename KP, typename R, int D, int DU>
__device__ __forceinline__ void drift(const KP &kp, const R (&y)[D], const R (&u)[DU],
                                      R (&f)[D]) {
  using M = Ar<R>;
  if constexpr (Pr<R>::on && D % 2 == 0) {
    // components i, i+1 together: the same operations in the same order as below
#pragma unroll
    for (int i = 0; i < D; i += 2) {
      R s0 = R(0), s1 = R(0);
#pragma unroll
      for (int l = 0; l < DU; ++l) Pr<R>::fma(kp.B[i * DU + l], kp.B[(i + 1) * DU + l], u[l], u[l], s0, s1);
#pragma unroll
      for (int j = 0; j < D; ++j) Pr<R>::fma(kp.A[i * D + j], kp.A[(i + 1) * D + j], y[j], y[j], s0, s1);
      f[i] = s0;
      f[i + 1] = s1;
    }
    if (kp.cubic) {
      R y2[D], y3[D];
#pragma unroll
      for (int j = 0; j < D; j += 2) {
        Pr<R>::mul(y[j], y[j + 1], y[j], y[j + 1], y2[j], y2[j + 1]);
        Pr<R>::mul(y2[j], y2[j + 1], y[j], y[j + 1], y3[j], y3[j + 1]);
      }
#pragma unroll
      for (int i = 0; i < D; i += 2)
#pragma unroll
        for (int j = 0; j < D; ++j) Pr<R>::fma(kp.C[i * D + j], kp.C[(i + 1) * D + j], y3[j], y3[j], f[i], f[i + 1]);
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < D; ++i) {
    R s = R(0);
#pragma unroll
    for (int l = 0; l < DU; ++l) s = M::fma(kp.B[i * DU + l], u[l], s);
#pragma unroll
    for (int j = 0; j < D; ++j) s = M::fma(kp.A[i * D + j], y[j], s);
    f[i] = s;
  }
  if (kp.cubic) {
    R y3[D];
#pragma unroll
    for (int j = 0; j < D; ++j) y3[j] = M::mul(M::mul(y[j], y[j]), y[j]);
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) f[i] = M::fma(kp.C[i * D + j], y3[j], f[i]);
  }
}

// mu <- mu + delta J_f(y)^T mu,  J_f = A + 3 C diag(y^2)
template <typename KP, typename R, int D>
__device__ __forceinline__ void adjoint_update(const KP &kp, const R (&y)[D], R delta,
                                               R (&mu)[D]) {
  using M = Ar<R>;
  R t[D];
  if constexpr (Pr<R>::on && D % 2 == 0) {
    // components j, j+1 together: the same operations in the same order as below
#pragma unroll
    for (int j = 0; j < D; j += 2) {
      R s0 = R(0), s1 = R(0);
#pragma unroll
      for (int i = 0; i < D; ++i) Pr<R>::fma(kp.A[i * D + j], kp.A[i * D + j + 1], mu[i], mu[i], s0, s1);
      t[j] = s0;
      t[j + 1] = s1;
    }
    if (kp.cubic) {
#pragma unroll
      for (int j = 0; j < D; j += 2) {
        R s0 = R(0), s1 = R(0);
#pragma unroll
        for (int i = 0; i < D; ++i) Pr<R>::fma(kp.C[i * D + j], kp.C[i * D + j + 1], mu[i], mu[i], s0, s1);
        R q0, q1, w0, w1;
        Pr<R>::mul(y[j], y[j + 1], y[j], y[j + 1], q0, q1);
        Pr<R>::mul(R(3), R(3), q0, q1, w0, w1);
        Pr<R>::fma(w0, w1, s0, s1, t[j], t[j + 1]);
      }
    }
#pragma unroll
    for (int j = 0; j < D; j += 2) Pr<R>::fma(delta, delta, t[j], t[j + 1], mu[j], mu[j + 1]);
    return;
  }
#pragma unroll
  for (int j = 0; j < D; ++j) {
    R s = R(0);
#pragma unroll
    for (int i = 0; i < D; ++i) s = M::fma(kp.A[i * D + j], mu[i], s);
    t[j] = s;
  }
  if (kp.cubic) {
#pragma unroll
    for (int j = 0; j < D; ++j) {
      R s = R(0);
#pragma unroll
      for (int i = 0; i < D; ++i) s = M::fma(kp.C[i * D + j], mu[i], s);
      t[j] = M::fma(M::mul(R(3), M::mul(y[j], y[j])), s, t[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < D; ++j) mu[j] = M::fma(delta, t[j], mu[j]);
}

// g += delta B^T mu
template <typename KP, typename R, int D, int DU>
__device__ __forceinline__ void control_sensitivity(const KP &kp, const R (&mu)[D],
                                                    R delta, R (&g)[DU]) {
  using M = Ar<R>;
#pragma unroll
  for (int l = 0; l < DU; ++l) {
    R s = R(0);
#pragma unroll
    for (int c = 0; c < D; ++c) s = M::fma(kp.B[c * DU + l], mu[c], s);
    g[l] = M::fma(delta, s, g[l]);
  }
}

// ---------------------------------------------------------------------------
// Random draws of one uniform step
// ---------------------------------------------------------------------------
template <int D>
struct MainWords {
  static constexpr int PD = (D + 1) / 2;            // normal pairs compiled
  static constexpr int NB = (1 + 2 * PD + 3) / 4;   // Philox blocks per step
};

// Main stream of step k, path m: word 0 decides the Poisson count, words 1..2P the
// sub-step-0 normals.
// Block (c0, c1, c2, epoch) of the problem's generator; RK: with the round keys of the
// parameter block (kernels whose kp is a __grid_constant__ parameter), else the keys are
// bumped round by round.  The same words either way.
template <bool RK, typename R, int D, int DU>
__device__ __forceinline__ uint4 philox_kp(const KParams<R, D, DU> &kp, uint32_t c0, uint32_t c1, uint32_t c2) {
  if constexpr (RK)
    return philox10_rk(c0, c1, c2, kp.epoch, kp.rk0, kp.rk1);
  else
    return philox10(c0, c1, c2, kp.epoch, kp.key0, kp.key1);
}

template <bool RK = false, typename R, int D, int DU>
__device__ __forceinline__ uint32_t main_draws(const KParams<R, D, DU> &kp, int k, uint32_t m,
                                               R (&z)[D]) {
  constexpr int NB = MainWords<D>::NB, PD = MainWords<D>::PD;
  uint32_t w[4 * NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const uint4 o = philox_kp<RK>(kp, (uint32_t)k, m, (uint32_t)b);
    w[4 * b] = o.x;
    w[4 * b + 1] = o.y;
    w[4 * b + 2] = o.z;
    w[4 * b + 3] = o.w;
  }
#pragma unroll
  for (int p = 0; p < PD; ++p) {
    R a, b;
    normal_pair<R>(w[1 + 2 * p], w[2 + 2 * p], a, b);
    z[2 * p] = a;
    if (2 * p + 1 < D) z[2 * p + 1] = b;
  }
  return w[0];
}

template <typename R, int D, int DU>
__device__ __forceinline__ bool has_jump(const KParams<R, D, DU> &kp, uint32_t w0) {
  return kp.jumps_on && (unsigned long long)w0 >= kp.thr[0];
}

// Sub-step structure of a step that has jumps: the time order of the jump slots,
// the sub-step lengths and the sub-step start states.  Sizes and normals are not
// stored; they are regenerated from the slot's Philox words when needed.
template <typename R, int D>
struct JumpStep {
  int n;
  int order[NMAX];        // slot (0-based) of the i-th jump in time order
  R th[NMAX];             // sorted jump-time fractions
  R delta[NMAX + 1];
  R Y[NMAX + 2][D];       // Y[i] = start of sub-step i, Y[n+1] = X_{k+1}
};

// Jump slot s of step k (counter (k, m, 1<<24 | (s+1)<<16 | b, epoch)): word 0 is the
// time fraction, words 1..2P the size, words 1+2P..4P the normals of the sub-step
// that starts at this jump.  Returns unit sizes xih and normals z (zero for c >= d).
template <typename R, int D, int DU>
__device__ __forceinline__ void slot_draws(const KParams<R, D, DU> &kp, int k, uint32_t m, int s,
                                           R *xih, R *z) {
  using M = Ar<R>;
  const int P = kp.npair, d = kp.d;
  const uint32_t tag = (1u << 24) | ((uint32_t)(s + 1) << 16);
#pragma unroll
  for (int c = 0; c < D; ++c) {
    xih[c] = R(0);
    z[c] = R(0);
  }
  uint4 blk = make_uint4(0, 0, 0, 0);
  int have = -1;
  auto word = [&](int j) -> uint32_t {
    if ((j >> 2) != have) {
      have = j >> 2;
      blk = philox10((uint32_t)k, m, tag | (uint32_t)have, kp.epoch, kp.key0, kp.key1);
    }
    const int r = j & 3;
    return r == 0 ? blk.x : (r == 1 ? blk.y : (r == 2 ? blk.z : blk.w));
  };
#pragma unroll 1
  for (int p = 0; p < P; ++p) {
    const uint32_t wa = word(1 + 2 * p), wb = word(2 + 2 * p);
    R a, b;
    if (kp.jump_law == JD_JUMP_UNIFORM) {
      a = M::sub(M::mul(R(2), M::u01(wa)), R(1));
      b = M::sub(M::mul(R(2), M::u01(wb)), R(1));
    } else {
      normal_pair<R>(wa, wb, a, b);
    }
    if (2 * p < d) xih[2 * p] = a;
    if (2 * p + 1 < d) xih[2 * p + 1] = b;
  }
#pragma unroll 1
  for (int p = 0; p < P; ++p) {
    const uint32_t wa = word(1 + 2 * P + 2 * p), wb = word(2 + 2 * P + 2 * p);
    R a, b;
    normal_pair<R>(wa, wb, a, b);
    if (2 * p < d) z[2 * p] = a;
    if (2 * p + 1 < d) z[2 * p + 1] = b;
  }
}

// Draws of jump slot 0 for a step with exactly one jump, with the word layout known at
// compile time (valid when kp.npair == ceil(D/2)): time fraction, unit size, and the
// normals of the sub-step after the jump.  Same values as slot_draws(kp, k, m, 0, ..).
template <bool RK = false, typename R, int D, int DU>
__device__ __forceinline__ R slot0_draws(const KParams<R, D, DU> &kp, int k, uint32_t m, R (&xih)[D],
                                         R (&z)[D]) {
  using M = Ar<R>;
  constexpr int PD = MainWords<D>::PD;
  constexpr int NB = (1 + 4 * PD + 3) / 4;
  uint32_t w[4 * NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const uint4 o = philox_kp<RK>(kp, (uint32_t)k, m, (1u << 24) | (1u << 16) | (uint32_t)b);
    w[4 * b] = o.x;
    w[4 * b + 1] = o.y;
    w[4 * b + 2] = o.z;
    w[4 * b + 3] = o.w;
  }
  const int d = kp.d;
#pragma unroll
  for (int p = 0; p < PD; ++p) {
    R a, b;
    if (kp.jump_law == JD_JUMP_UNIFORM) {
      a = M::sub(M::mul(R(2), M::u01(w[1 + 2 * p])), R(1));
      b = M::sub(M::mul(R(2), M::u01(w[2 + 2 * p])), R(1));
    } else {
      normal_pair<R>(w[1 + 2 * p], w[2 + 2 * p], a, b);
    }
    xih[2 * p] = 2 * p < d ? a : R(0);
    if (2 * p + 1 < D) xih[2 * p + 1] = 2 * p + 1 < d ? b : R(0);
    normal_pair<R>(w[1 + 2 * PD + 2 * p], w[2 + 2 * PD + 2 * p], a, b);
    z[2 * p] = 2 * p < d ? a : R(0);
    if (2 * p + 1 < D) z[2 * p + 1] = 2 * p + 1 < d ? b : R(0);
  }
  return M::u01(w[0]);
}

// The jump map applied at an arrival with unit sizes xih (Sec. 5.3 eq:jump_law):
// y_c <- jgain_c y_c + jscl_c xih_c.  Additive laws: jgain = 1, jscl = s (y + s xih, bit
// for bit).  Keilson-Storer: the velocity half z_c, c >= d/2, of the phase-space state
// is reset to gamma z_c + s xih_c; positions have jgain = 1, jscl = 0 and stay.  No
// branch on the law, so the inline one-jump step keeps its size.
template <typename R, int D, int DU>
__device__ __forceinline__ void apply_jump(const KParams<R, D, DU> &kp, R *y, const R *xih) {
  using M = Ar<R>;
#pragma unroll
  for (int c = 0; c < D; ++c) y[c] = M::add(M::mul(kp.jgain[c], y[c]), M::mul(kp.jscl[c], xih[c]));
}

// Adjoint across a jump: mu (derivative w.r.t. the post-jump state) times the map's
// Jacobian, the identity for the additive laws and gamma on the reset velocities.
// (jgain_c = 1 leaves mu_c unchanged bit for bit, so the additive laws need no branch)
template <typename KP, typename R>
__device__ __forceinline__ void jump_adjoint(const KP &kp, R *mu) {
  using M = Ar<R>;
  constexpr int D = sizeof(kp.jgain) / sizeof(kp.jgain[0]);
  if constexpr (Pr<R>::on && D % 2 == 0) {
#pragma unroll
    for (int c = 0; c < D; c += 2) Pr<R>::mul(kp.jgain[c], kp.jgain[c + 1], mu[c], mu[c + 1], mu[c], mu[c + 1]);
  } else {
#pragma unroll
    for (int c = 0; c < D; ++c) mu[c] = M::mul(kp.jgain[c], mu[c]);
  }
}

// One Euler sub-step y <- y + de f(y, u) + sigma sqrt(de) z (the form every jump path uses).
template <typename R, int D, int DU>
__device__ __forceinline__ void euler_substep(const KParams<R, D, DU> &kp, R de, const R (&z)[D],
                                              const R (&u)[DU], R (&y)[D]) {
  using M = Ar<R>;
  R f[D];
  drift(kp, y, u, f);
  const R sq = M::sqrt(de);
  if constexpr (Pr<R>::on && D % 2 == 0) {
#pragma unroll
    for (int c = 0; c < D; c += 2) {
      R a0, a1;
      Pr<R>::fma(de, de, f[c], f[c + 1], y[c], y[c + 1]);
      Pr<R>::mul(kp.sigma[c], kp.sigma[c + 1], sq, sq, a0, a1);
      Pr<R>::fma(a0, a1, z[c], z[c + 1], y[c], y[c + 1]);
    }
    return;
  }
#pragma unroll
  for (int c = 0; c < D; ++c) y[c] = M::fma(M::mul(kp.sigma[c], sq), z[c], M::fma(de, f[c], y[c]));
}

// Plan and integrate a step that has jumps (Algorithm 5.1 with the additive jump
// map): Poisson count from w0, jump times (word 0 of every slot) sorted stably,
// sub-step lengths, then the Euler sub-steps from x with the jump of slot order[i]
// applied after sub-step i.
template <typename R, int D, int DU>
__device__ __noinline__ void build_jump_step(const KParams<R, D, DU> &kp, int k, uint32_t m,
                                             uint32_t w0, const R *z0, const R *u, const R *x,
                                             JumpStep<R, D> *S) {
  using M = Ar<R>;
  int n = 0;
#pragma unroll 1
  for (int i = 0; i < NMAX; ++i) n += ((unsigned long long)w0 >= kp.thr[i]) ? 1 : 0;
  S->n = n;
  if (n == 0) {   // callers only come here after a jump was drawn; stay well defined
    R uu[DU], y[D], f[D];
#pragma unroll
    for (int l = 0; l < DU; ++l) uu[l] = u[l];
#pragma unroll
    for (int c = 0; c < D; ++c) y[c] = S->Y[0][c] = x[c];
    drift(kp, y, uu, f);
    S->delta[0] = kp.dt;
#pragma unroll
    for (int c = 0; c < D; ++c) S->Y[1][c] = M::fma(kp.sig_sqdt[c], z0[c], M::fma(kp.dt, f[c], y[c]));
    return;
  }
  R theta[NMAX];
#pragma unroll 1
  for (int i = 0; i < n; ++i) {
    const uint4 o = philox10((uint32_t)k, m, (1u << 24) | ((uint32_t)(i + 1) << 16), kp.epoch,
                             kp.key0, kp.key1);
    theta[i] = M::u01(o.x);
    S->order[i] = i;
  }
#pragma unroll 1
  for (int i = 1; i < n; ++i) {
    const int cur = S->order[i];
    int j = i - 1;
    while (j >= 0 && theta[S->order[j]] > theta[cur]) {
      S->order[j + 1] = S->order[j];
      --j;
    }
    S->order[j + 1] = cur;
  }
#pragma unroll 1
  for (int i = 0; i < n; ++i) S->th[i] = theta[S->order[i]];
  S->delta[0] = M::mul(kp.dt, S->th[0]);
#pragma unroll 1
  for (int i = 1; i < n; ++i) S->delta[i] = M::mul(kp.dt, M::sub(S->th[i], S->th[i - 1]));
  S->delta[n] = M::mul(kp.dt, M::sub(R(1), S->th[n - 1]));
  R uu[DU], y[D], z[D];
#pragma unroll
  for (int l = 0; l < DU; ++l) uu[l] = u[l];
#pragma unroll
  for (int c = 0; c < D; ++c) {
    y[c] = x[c];
    z[c] = z0[c];
    S->Y[0][c] = y[c];
  }
#pragma unroll 1
  for (int i = 0; i <= n; ++i) {
    R f[D];
    drift(kp, y, uu, f);
    const R de = S->delta[i], sq = M::sqrt(de);
#pragma unroll
    for (int c = 0; c < D; ++c) y[c] = M::fma(M::mul(kp.sigma[c], sq), z[c], M::fma(de, f[c], y[c]));
    if (i < n) {
      R xih[D];
      slot_draws(kp, k, m, S->order[i], xih, z);
      apply_jump(kp, y, xih);
    }
#pragma unroll
    for (int c = 0; c < D; ++c) S->Y[i + 1][c] = y[c];
  }
}

}  // namespace jd
