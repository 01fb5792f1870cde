// jd_tc32.cuh -- d = 32 linear-drift kernels (FP32 paths), one CTA per tile of 128 paths.
//
// The drift contraction A x of all 128 paths of a tile is one 128 x 32 x 32 matrix
// product per step.  TC = 0 runs it on the CUDA cores (coefficients as constant-bank
// operands); TC = 1 runs it on the tensor cores (tcgen05.mma, BF16 inputs, FP32
// accumulation in tensor memory, one TMEM lane per path); TC = 2 splits each input into
// a BF16 high part and a BF16 low part and issues three products (hi*hi + hi*lo + lo*hi),
// which keeps about 16 mantissa bits.  The adjoint's A^T lambda uses the same scheme.
// Everything else (noise, jumps, cost, reductions) is the same FP32 arithmetic as the
// generic kernels; steps with jumps run entirely on the CUDA cores through the generic
// jump routines.
//
// tcgen05 usage: warp 0 allocates 32 TMEM columns; every step all threads write their
// row of the operand tile (K-major, no swizzle: 8-row x 16-byte core matrices, 128 B
// apart along K, 512 B apart along rows), fence the writes for the async proxy,
// synchronize, thread 0 issues the MMAs and commits them to an mbarrier; the threads
// generate the step's noise meanwhile, then wait on the mbarrier (bounded: on timeout the
// CTA records JD_ERR_TIMEOUT in *status and stops), and read their lane with tcgen05.ld.
//
// Layouts: traj32 [Nt+1][8][mloc][4] (state X_k, components 4c..4c+3 in one 16-byte
// vector); flags, jump log and partials as in jd_kernels.cuh.
#pragma once

#include <cuda_bf16.h>

#include "jd_kernels.cuh"

namespace jd {

constexpr int D32 = 32, DU32 = 4;
using KP32 = KParams<float, D32, DU32>;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (row, k) in a rows x 32 BF16 tile, K-major core-matrix layout.
__device__ __forceinline__ uint32_t tc_tile_off(int row, int kblk) {
  return (uint32_t)((row >> 3) * 512 + kblk * 128 + (row & 7) * 16);
}

__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;   // leading (K) byte offset between core matrices
  d |= (uint64_t)(512 >> 4) << 32;   // stride (row) byte offset between core matrices
  d |= (uint64_t)1 << 46;            // descriptor version
  return d;                          // no swizzle, base offset 0
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128, N = 32.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint32_t a_addr, uint32_t b_addr, uint32_t acc) {
  const uint64_t da = tc_smem_desc(a_addr), db = tc_smem_desc(b_addr);
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(da), "l"(db), "r"(kTcIdesc), "r"(acc));
}

// One row (thread) of a 32-wide operand: BF16 high part, and the low part when SPLIT.
template <bool SPLIT>
__device__ __forceinline__ void tc_write_row(unsigned char *hi, unsigned char *lo, int row, const float (&v)[32]) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint32_t ph[4], pl[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float a = v[8 * j + 2 * q], b = v[8 * j + 2 * q + 1];
      const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
      ph[q] = *reinterpret_cast<const uint32_t *>(&h);
      if (SPLIT) {
        const __nv_bfloat162 l = __floats2bfloat162_rn(a - __low2float(h), b - __high2float(h));
        pl[q] = *reinterpret_cast<const uint32_t *>(&l);
      }
    }
    const uint32_t off = tc_tile_off(row, j);
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(smem_u32(hi + off)), "r"(ph[0]), "r"(ph[1]),
                 "r"(ph[2]), "r"(ph[3]));
    if (SPLIT)
      asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(smem_u32(lo + off)), "r"(pl[0]), "r"(pl[1]),
                   "r"(pl[2]), "r"(pl[3]));
  }
}

// Shared state of a tensor-core tile.
struct TcShared {
  unsigned char xhi[8192], xlo[8192];   // 128 x 32 BF16 operand tiles (rows = paths)
  unsigned char ahi[2048], alo[2048];   // 32 x 32 BF16 coefficient tiles
  unsigned long long mbar;
  uint32_t tmem;
  int stop;     // set when a wait timed out; read by every thread after the issue barrier
  int issued;   // products committed so far (thread 0)
};

// Write the coefficient tile: row n, column k holds coef(n, k) (A for the forward,
// A^T for the adjoint).  Threads 0..31 write one row each.
template <bool SPLIT>
__device__ __forceinline__ void tc_write_coef(TcShared &sh, const KP32 &kp, bool transpose) {
  if (threadIdx.x < 32) {
    float row[32];
    const int n = threadIdx.x;
#pragma unroll
    for (int k = 0; k < 32; ++k) row[k] = transpose ? kp.A[k * 32 + n] : kp.A[n * 32 + k];
    tc_write_row<SPLIT>(sh.ahi, sh.alo, n, row);
  }
}

__device__ __forceinline__ void tc_setup(TcShared &sh) {
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem)),
                 "r"(32));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sh.mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    sh.stop = 0;
    sh.issued = 0;
  }
}

// Bounded wait for mbarrier phase `parity`; true when it completed.
__device__ __forceinline__ bool tc_wait(TcShared &sh, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 24) && !done; ++it) {
    asm volatile(
        "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(&sh.mbar)), "r"(parity));
  }
  return done != 0;
}

// Free the tile's tensor memory.  A CTA that stopped after a timed-out wait first waits
// once more (bounded) for its last product so no MMA is in flight.
__device__ __forceinline__ void tc_teardown(TcShared &sh) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (sh.stop && threadIdx.x == 0 && sh.issued > 0) (void)tc_wait(sh, (uint32_t)((sh.issued - 1) & 1));
  __syncthreads();
  if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sh.tmem), "r"(32));
}

// Issue the step's product (thread 0) after all rows are written.  Returns false (in
// every thread, read after the barrier) once the tile has stopped.
template <bool SPLIT>
__device__ __forceinline__ bool tc_issue(TcShared &sh) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (sh.stop) return false;
  if (threadIdx.x == 0) {
    const uint32_t x0 = smem_u32(sh.xhi), xl = smem_u32(sh.xlo), a0 = smem_u32(sh.ahi), al = smem_u32(sh.alo);
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) tc_mma(sh.tmem, x0 + kk * 256, a0 + kk * 256, kk > 0);
    if (SPLIT) {
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) tc_mma(sh.tmem, xl + kk * 256, a0 + kk * 256, 1);
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) tc_mma(sh.tmem, x0 + kk * 256, al + kk * 256, 1);
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(&sh.mbar)));
    sh.issued++;
  }
  return true;
}

// Wait for the step's product (bounded) and read this thread's lane: out[n] = row . coef_n.
// Returns false when the wait timed out (the CTA then stops).
__device__ __forceinline__ bool tc_collect(TcShared &sh, uint32_t parity, float (&out)[32], int *status) {
  const bool done = tc_wait(sh, parity);
  if (!done) {
    sh.stop = 1;
    if (status) atomicExch(status, (int)JD_ERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  uint32_t r[32];
  const uint32_t addr = sh.tmem + ((uint32_t)((threadIdx.x >> 5) * 32) << 16);
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int n = 0; n < 32; ++n) out[n] = __uint_as_float(r[n]);
  return done;
}

// out = A x (transpose = false) or A^T x on the CUDA cores (constant-bank coefficients)
__device__ __forceinline__ void cc_matvec(const KP32 &kp, const float (&x)[32], float (&out)[32], bool transpose) {
#pragma unroll
  for (int n = 0; n < 32; ++n) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 32; ++k) s = __fmaf_rn(transpose ? kp.A[k * 32 + n] : kp.A[n * 32 + k], x[k], s);
    out[n] = s;
  }
}

// Main-stream noise of step k: block 0 first (its word 0 decides the Poisson count);
// when the step has no jump, x_c += sigma_c sqrt(dt) Z_c is added in place, block by
// block, so no copy of the state is kept.  Returns word 0.
__device__ __forceinline__ uint32_t main_noise_or_jump(const KP32 &kp, int k, uint32_t m, float (&x)[32],
                                                        bool &jump) {
  const uint4 o0 = philox10((uint32_t)k, m, 0u, kp.epoch, kp.key0, kp.key1);
  jump = has_jump(kp, o0.x);
  if (jump) return o0.x;
  uint32_t carry = o0.w;
  {
    float z0, z1;
    normal_pair<float>(o0.y, o0.z, z0, z1);   // words 1, 2 -> components 0, 1
    x[0] = __fmaf_rn(kp.sig_sqdt[0], z0, x[0]);
    x[1] = __fmaf_rn(kp.sig_sqdt[1], z1, x[1]);
  }
#pragma unroll
  for (int b = 1; b < 9; ++b) {
    const uint4 o = philox10((uint32_t)k, m, (uint32_t)b, kp.epoch, kp.key0, kp.key1);
    // words 4b..4b+3: pairs (4b-1, 4b) and (4b+1, 4b+2); word 4b+3 carries over
    const int c = 4 * b - 2;   // components of pair (4b-1, 4b)
    float z0, z1;
    normal_pair<float>(carry, o.x, z0, z1);
    x[c] = __fmaf_rn(kp.sig_sqdt[c], z0, x[c]);
    x[c + 1] = __fmaf_rn(kp.sig_sqdt[c + 1], z1, x[c + 1]);
    if (b < 8) {
      normal_pair<float>(o.y, o.z, z0, z1);
      x[c + 2] = __fmaf_rn(kp.sig_sqdt[c + 2], z0, x[c + 2]);
      x[c + 3] = __fmaf_rn(kp.sig_sqdt[c + 3], z1, x[c + 3]);
      carry = o.w;
    }
  }
  return o0.x;
}

template <int TC>
__global__ void __launch_bounds__(TPB)
fwd32_kernel(const __grid_constant__ KP32 kp, const float *__restrict__ u, const float *__restrict__ xd,
             double *__restrict__ partC, float *__restrict__ traj, uint32_t *__restrict__ flags,
             float *__restrict__ pcost, JLog<float, D32> jl, int *__restrict__ jcnt, int *status,
             int64_t mloc) {
  constexpr bool SPLIT = TC == 2;
  __shared__ __align__(1024) TcShared sh;
  __shared__ Pair<float> red[TPB / 32];
  const int64_t lm = (int64_t)blockIdx.x * TPB + threadIdx.x;
  const bool active = lm < mloc;
  const uint32_t m = (uint32_t)(kp.m_begin + lm);
  const int Nt = kp.Nt;
  const bool store = traj != nullptr;
  if (TC) {
    tc_setup(sh);
    tc_write_coef<SPLIT>(sh, kp, false);
  }
  float x[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) x[c] = kp.x0[c];
  Kahan<float> cost;
  uint32_t fw = 0;
  LogWriter<float, D32> lw;
  lw.L = jl;
  lw.idx = lm;
  if (!active || !store) lw.L.cap = 0;
#pragma unroll 1
  for (int k = 0; k <= Nt; ++k) {
    if (store && active) {
#pragma unroll
      for (int c4 = 0; c4 < 8; ++c4)
        Vec4<float>::store(traj + (((size_t)k * 8 + c4) * mloc + lm) * 4, x[4 * c4], x[4 * c4 + 1], x[4 * c4 + 2],
                           x[4 * c4 + 3]);
    }
    if (k == Nt) break;
    float f[32];
    if (TC) {
      tc_write_row<SPLIT>(sh.xhi, sh.xlo, threadIdx.x, x);
      if (!tc_issue<SPLIT>(sh)) break;
    } else {
      cc_matvec(kp, x, f, false);
    }
    bool jump;
    const uint32_t w0 = main_noise_or_jump(kp, k, m, x, jump);   // x += noise unless jump
    if (TC) tc_collect(sh, (uint32_t)(k & 1), f, status);
    if (!jump) {
      float uk[DU32];
#pragma unroll
      for (int l = 0; l < DU32; ++l) uk[l] = __ldg(u + (size_t)k * DU32 + l);
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        float bc = 0.f;
#pragma unroll
        for (int l = 0; l < DU32; ++l) bc = __fmaf_rn(kp.B[c * DU32 + l], uk[l], bc);
        x[c] = __fmaf_rn(kp.dt, __fadd_rn(f[c], bc), x[c]);
      }
    } else {
      // steps with jumps run on the CUDA cores through the generic routine (x is X_k)
      fw |= 1u << (k & 31);
      JumpStep<float, D32> S;
      float zl[32], ul[DU32], xl[32];
      (void)main_draws(kp, k, m, zl);
#pragma unroll
      for (int l = 0; l < DU32; ++l) ul[l] = __ldg(u + (size_t)k * DU32 + l);
#pragma unroll
      for (int c = 0; c < 32; ++c) xl[c] = x[c];
      build_jump_step(kp, k, m, w0, zl, ul, xl, &S);
#pragma unroll
      for (int c = 0; c < 32; ++c) x[c] = S.Y[S.n + 1][c];
      if (lw.fits(S.n)) {
        for (int i = 0; i < S.n; ++i) {
          float y[32];
#pragma unroll
          for (int c = 0; c < 32; ++c) y[c] = S.Y[i + 1][c];
          lw.put(k, S.th[i], y);
        }
      }
    }
    cost.add(cost_term(kp, x, xd + (size_t)(k + 1) * D32));
    if (store && ((k & 31) == 31 || k == Nt - 1)) {
      if (active) flags[(size_t)(k >> 5) * mloc + lm] = fw;
      fw = 0;
    }
  }
  if (store && active) jcnt[lm] = lw.r;
  Pair<float> v = cost.pair();
  if (!active) v = {0.f, 0.f};
  if (pcost && active) pcost[lm] = v.s + v.e;
  const double s = block_sum_to_double(v, red);
  if (threadIdx.x == 0) partC[blockIdx.x] = s;
  if (TC) tc_teardown(sh);
}

// Backward through a step that had jumps (rare), out of line so that its register
// needs do not weigh on the main loop: X_k is reloaded, the generic backward step runs on
// the CUDA cores (jump log or regeneration), and the cost gradient at t_k is added.
__device__ __noinline__ void adj32_jump_step(const KP32 &kp, int k, uint32_t m, const float *__restrict__ traj,
                                             int64_t mloc, int64_t lmc, const float *__restrict__ u,
                                             const float *__restrict__ xd, float *mu_io, float *g_out,
                                             LogReader<float, D32> *lr) {
  float xk[32], mu[32], g[DU32], th[D32 + 2];
#pragma unroll
  for (int c4 = 0; c4 < 8; ++c4) {
    float v[4];
    Vec4<float>::load(traj + (((size_t)k * 8 + c4) * mloc + lmc) * 4, v);
#pragma unroll
    for (int q = 0; q < 4; ++q) xk[4 * c4 + q] = v[q];
  }
#pragma unroll
  for (int c = 0; c < 32; ++c) mu[c] = mu_io[c];
  LogReader<float, D32> l = *lr;
  backward_step<float, D32, DU32, false>(kp, k, m, true, xk, u, xd, mu, g, th, l);
  *lr = l;
#pragma unroll
  for (int c = 0; c < 32; ++c) mu_io[c] = mu[c];
#pragma unroll
  for (int q = 0; q < DU32; ++q) g_out[q] = g[q];
}

template <int TC>
__global__ void __launch_bounds__(TPB)
adj32_kernel(const __grid_constant__ KP32 kp, const float *__restrict__ u, const float *__restrict__ xd,
             const float *__restrict__ traj, const uint32_t *__restrict__ flags, JLog<float, D32> jl,
             const int *__restrict__ jcnt, double *__restrict__ partG, float *__restrict__ lam_out,
             int *status, int64_t mloc) {
  constexpr bool SPLIT = TC == 2;
  __shared__ __align__(1024) TcShared sh;
  const int64_t npart = (int64_t)kp.nblk * (TPB / 32);
  const int64_t wid = (int64_t)blockIdx.x * (TPB / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int64_t lm = (int64_t)blockIdx.x * TPB + threadIdx.x;
  const bool active = lm < mloc;
  const int64_t lmc = active ? lm : 0;   // inactive threads replay path 0
  const uint32_t m = (uint32_t)(kp.m_begin + lmc);
  const int Nt = kp.Nt;
  if (TC) {
    tc_setup(sh);
    tc_write_coef<SPLIT>(sh, kp, true);
  }
  LogReader<float, D32> lr;
  lr.L = jl;
  lr.idx = lmc;
  lr.init(min(__ldg(jcnt + lmc), jl.cap));
  float mu[32];
  {
    float x[32];
#pragma unroll
    for (int c4 = 0; c4 < 8; ++c4) {
      float v[4];
      Vec4<float>::load(traj + (((size_t)Nt * 8 + c4) * mloc + lmc) * 4, v);
#pragma unroll
      for (int q = 0; q < 4; ++q) x[4 * c4 + q] = v[q];
    }
#pragma unroll
    for (int c = 0; c < 32; ++c) mu[c] = __fmul_rn(kp.qdt[c], __fsub_rn(x[c], __ldg(xd + (size_t)Nt * D32 + c)));
    if (lam_out && active)
#pragma unroll
      for (int c = 0; c < 32; ++c) lam_out[((size_t)Nt * D32 + c) * mloc + lm] = mu[c];
  }
#pragma unroll 1
  for (int k = Nt - 1; k >= 0; --k) {
    if (TC) {
      tc_write_row<SPLIT>(sh.xhi, sh.xlo, threadIdx.x, mu);
      if (!tc_issue<SPLIT>(sh)) break;
    }
    const bool jumped = (__ldg(flags + (size_t)(k >> 5) * mloc + lmc) >> (k & 31)) & 1u;
    float t[32];
    if (TC)
      tc_collect(sh, (uint32_t)((Nt - 1 - k) & 1), t, status);
    else
      cc_matvec(kp, mu, t, true);
    float g[DU32];
    if (!jumped) {
#pragma unroll
      for (int l = 0; l < DU32; ++l) g[l] = 0.f;
      control_sensitivity(kp, mu, kp.dt, g);
#pragma unroll
      for (int c = 0; c < 32; ++c) mu[c] = __fmaf_rn(kp.dt, t[c], mu[c]);
      if (k >= 1) {
        // cost gradient dt q (X_k - xd_k), the stored state streamed 4 components at a time
#pragma unroll
        for (int c4 = 0; c4 < 8; ++c4) {
          float v[4];
          Vec4<float>::load(traj + (((size_t)k * 8 + c4) * mloc + lmc) * 4, v);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = 4 * c4 + q;
            mu[c] = __fmaf_rn(kp.qdt[c], __fsub_rn(v[q], __ldg(xd + (size_t)k * D32 + c)), mu[c]);
          }
        }
      }
    } else {
      float ml[32], gl[DU32];
#pragma unroll
      for (int c = 0; c < 32; ++c) ml[c] = mu[c];
      adj32_jump_step(kp, k, m, traj, mloc, lmc, u, xd, ml, gl, &lr);
#pragma unroll
      for (int c = 0; c < 32; ++c) mu[c] = ml[c];
#pragma unroll
      for (int l = 0; l < DU32; ++l) g[l] = gl[l];
    }
    if (lam_out && active)
#pragma unroll
      for (int c = 0; c < 32; ++c) lam_out[((size_t)k * D32 + c) * mloc + lm] = mu[c];
    // per-step, per-warp compensated sums of the control sensitivities
#pragma unroll
    for (int l = 0; l < DU32; ++l) {
      const Pair<float> r = warp_sum(Pair<float>{active ? g[l] : 0.f, 0.f});
      if (lane == 0) partG[((int64_t)k * DU32 + l) * npart + wid] = (double)r.s + (double)r.e;
    }
  }
  if (TC) tc_teardown(sh);
}

}  // namespace jd
