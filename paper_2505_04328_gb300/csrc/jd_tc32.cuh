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
// The coefficient struct (13 KB) reaches the kernels through a device buffer and is
// staged into shared memory once per CTA; the kernels take no large parameters.
//
// Layouts: traj32 [Nt+1][8][mloc][4] (state X_k, components 4c..4c+3 in one 16-byte
// vector); flags, jump log and partials as in jd_kernels.cuh.
#pragma once

#include <cuda_bf16.h>

#include <cstddef>

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

// Coefficients of a tile in shared memory: the parameter struct (13 KB, beyond what the
// constant bank serves directly) plus A^T, copied once per CTA.
struct CcShared {
  float at[32 * 32];   // at[k * 32 + n] = A[n][k]; first, so its 16-byte rows stay aligned
  KP32 kp;             // kp.A at byte 4096 + 0: 16-byte aligned too
};
static_assert(offsetof(CcShared, kp) % 16 == 0 && offsetof(KP32, A) == 0, "16-byte aligned coefficient rows");

__device__ __forceinline__ void stage_params(CcShared &cs, const KP32 *__restrict__ kpg) {
  const uint32_t *src = reinterpret_cast<const uint32_t *>(kpg);
  uint32_t *dst = reinterpret_cast<uint32_t *>(&cs.kp);
  for (int i = threadIdx.x; i < (int)(sizeof(KP32) / 4); i += blockDim.x) dst[i] = __ldg(src + i);
  for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) cs.at[(i & 31) * 32 + (i >> 5)] = __ldg(kpg->A + i);
  __syncthreads();
}

// out_n = sum_k M[k][n] v_k on the CUDA cores, M row-major in shared memory (M = A^T
// gives A v, M = A gives A^T v).  v goes through the thread's own shared-memory column
// (vcol[k * TPB]) so the loop over k stays rolled; the rows of M are broadcast reads.
__device__ __forceinline__ void cc_matvec(const float *M, float *vcol, const float (&v)[32], float (&out)[32]) {
#pragma unroll
  for (int k = 0; k < 32; ++k) vcol[k * TPB] = v[k];
#pragma unroll
  for (int n = 0; n < 32; ++n) out[n] = 0.f;
#pragma unroll 2
  for (int k = 0; k < 32; ++k) {
    const float vk = vcol[k * TPB];
    const float4 *row = reinterpret_cast<const float4 *>(M + k * 32);
#pragma unroll
    for (int q = 0; q < 8; ++q) {   // paired FMAs: per component the rounding of __fmaf_rn
      const float4 a = row[q];
      Pr<float>::fma(a.x, a.y, vk, vk, out[4 * q], out[4 * q + 1]);
      Pr<float>::fma(a.z, a.w, vk, vk, out[4 * q + 2], out[4 * q + 3]);
    }
  }
}

// Main-stream noise of step k: block 0 first (its word 0 decides the Poisson count);
// when the step has no jump, x_c += sigma_c sqrt(dt) Z_c.  Blocks 1..8 run in a loop
// unrolled four times (four independent Philox chains for the scheduler) that parks the
// 30 normals in the thread's shared-memory column zcol[c * TPB]; the fully unrolled form,
// 9 Philox blocks and 16 Box-Muller pairs of straight-line code, overflowed the
// instruction cache.  Returns word 0.
// rk: the Philox round keys as a kernel parameter (constant operands of the rounds' XORs;
// the staged copy in shared memory would cost a load per key).
struct RoundKeys {
  uint32_t k0[10], k1[10];
};

__device__ __forceinline__ uint32_t main_noise_or_jump(const KP32 &kp, const RoundKeys &rk, int k, uint32_t m,
                                                        float (&x)[32], float *zcol, bool &jump) {
  const uint4 o0 = philox10_rk((uint32_t)k, m, 0u, kp.epoch, rk.k0, rk.k1);
  jump = has_jump(kp, o0.x);
  if (jump) return o0.x;
  uint32_t carry = o0.w;
  {
    float z0, z1;
    normal_pair<float>(o0.y, o0.z, z0, z1);   // words 1, 2 -> components 0, 1
    x[0] = __fmaf_rn(kp.sig_sqdt[0], z0, x[0]);
    x[1] = __fmaf_rn(kp.sig_sqdt[1], z1, x[1]);
  }
#pragma unroll 4
  for (int b = 1; b < 9; ++b) {
    const uint4 o = philox10_rk((uint32_t)k, m, (uint32_t)b, kp.epoch, rk.k0, rk.k1);
    // words 4b..4b+3: pairs (4b-1, 4b) and (4b+1, 4b+2); word 4b+3 carries over
    const int c = 4 * b - 2;   // components of pair (4b-1, 4b)
    float z0, z1;
    normal_pair<float>(carry, o.x, z0, z1);
    zcol[c * TPB] = z0;
    zcol[(c + 1) * TPB] = z1;
    if (b < 8) {
      normal_pair<float>(o.y, o.z, z0, z1);
      zcol[(c + 2) * TPB] = z0;
      zcol[(c + 3) * TPB] = z1;
      carry = o.w;
    }
  }
#pragma unroll
  for (int c = 2; c < 32; c += 2)
    Pr<float>::fma(kp.sig_sqdt[c], kp.sig_sqdt[c + 1], zcol[c * TPB], zcol[(c + 1) * TPB], x[c], x[c + 1]);
  return o0.x;
}

// ---------------------------------------------------------------------------
// Steps with jumps at d = 32 (linear drift)
// ---------------------------------------------------------------------------

// y += de * (f + B u_k)
__device__ __forceinline__ void add_drift(const KP32 &kp, const float *__restrict__ u, int k, float de,
                                          const float (&f)[32], float (&y)[32]) {
  float uk[DU32];
#pragma unroll
  for (int l = 0; l < DU32; ++l) uk[l] = __ldg(u + (size_t)k * DU32 + l);
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    float bc = 0.f;
#pragma unroll
    for (int l = 0; l < DU32; ++l) bc = __fmaf_rn(kp.B[c * DU32 + l], uk[l], bc);
    y[c] = __fmaf_rn(de, __fadd_rn(f[c], bc), y[c]);
  }
}

// Sorted jump-time fractions of step k (n jumps): regenerated from word 0 of each slot.
__device__ __forceinline__ void regen_jump_times(const KP32 &kp, int k, uint32_t m, int n, float *th) {
#pragma unroll 1
  for (int i = 0; i < n; ++i)
    th[i] = Ar<float>::u01(philox10((uint32_t)k, m, (1u << 24) | ((uint32_t)(i + 1) << 16), kp.epoch, kp.key0,
                                    kp.key1).x);
#pragma unroll 1
  for (int i = 1; i < n; ++i) {
    const float cur = th[i];
    int j = i - 1;
    while (j >= 0 && th[j] > cur) {
      th[j + 1] = th[j];
      --j;
    }
    th[j + 1] = cur;
  }
}

// One-jump steps of a warp (linear drift, d = 32), done by the whole warp.  The step of
// a lane with one jump at fraction th (word 0 of jump slot 0): sub-step 0 of length
// d0 = dt th from X_k with the step's main-stream normals (words 1..32, pair p of
// components (2p, 2p + 1) from words (2p + 1, 2p + 2)) scaled by sigma_c sqrt(d0) and the
// drift f = A X_k + B u_k; the jump Y_1 = Y + jump_scale xi (sizes xi from slot-0 words
// 1..32: normal pairs, or 2 u - 1 per word for the uniform law); sub-step 1 of length
// d1 = dt (1 - th) from Y_1 with the post-jump normals (slot-0 words 33..64) and the drift
// A Y_1 + B u_k.  For each such lane the 32 lanes draw its Philox blocks (the 9 of its
// main stream and the 17 of its slot) in one round and its 48 Box-Muller pairs in two,
// and then carry one component each through the step's arithmetic (A Y_1 in k order from
// zero, as cc_matvec); every component gets the operations of the one-lane routine in the
// same order, so the same bits.  A lane alone drew 27 blocks and 48 pairs and did all 32
// components while its warp (and, with the tensor cores, its CTA at the next step's
// barrier) waited; here it only hands over X_k and A X_k and takes X_{k+1} and Y_1 back.
// ws: the warp's 32 x TPB floats of vbuf, free at this point of the step (rows: 0-1 main
// words, 2-4 slot words, 5 main normals, 6 jump sizes, 7 post-jump normals, 8 Y_1, 9 X,
// 10 A X_k).  Called by every lane of the warp; returns th in the jump lanes.
__device__ __forceinline__ float coop_one_jumps(const KP32 &kp, const float *at, float *ws, int k, uint32_t m,
                                                const float *__restrict__ u, unsigned om, float (&x)[32],
                                                const float (&f)[32], float (&y1)[32]) {
  const int lane = threadIdx.x & 31;
  uint32_t *wu = reinterpret_cast<uint32_t *>(ws);
  auto mword = [&](int w) -> uint32_t & { return wu[(w >> 5) * TPB + (w & 31)]; };
  auto sword = [&](int w) -> uint32_t & { return wu[(2 + (w >> 5)) * TPB + (w & 31)]; };
  float *zm = ws + 5 * TPB, *zs = ws + 6 * TPB, *zp = ws + 7 * TPB, *yv = ws + 8 * TPB, *xv = ws + 9 * TPB,
        *fv = ws + 10 * TPB;
  const uint32_t tag = (1u << 24) | (1u << 16);   // jump slot 0
  const bool sizes_normal = kp.jump_law != JD_JUMP_UNIFORM;
  float th_out = 0.f;
  while (om) {
    const int j = __ffs(om) - 1;
    om &= om - 1;
    const uint32_t mj = __shfl_sync(0xffffffffu, m, j);
    if (lane < 26) {   // lanes 0..8: main blocks 0..8; lanes 9..25: slot blocks 0..16
      const bool slot = lane >= 9;
      const uint32_t b = slot ? (uint32_t)(lane - 9) : (uint32_t)lane;
      const uint4 o = philox10((uint32_t)k, mj, slot ? (tag | b) : b, kp.epoch, kp.key0, kp.key1);
      const int w = 4 * (int)b;
      if (slot) {
        sword(w) = o.x;
        sword(w + 1) = o.y;
        sword(w + 2) = o.z;
        sword(w + 3) = o.w;
      } else {
        mword(w) = o.x;
        mword(w + 1) = o.y;
        mword(w + 2) = o.z;
        mword(w + 3) = o.w;
      }
    }
    if (lane == j) {   // X_k and A X_k of the jump lane
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        xv[c] = x[c];
        fv[c] = f[c];
      }
    }
    __syncwarp();
    {   // pair p of components (2p, 2p + 1) takes words (2p + 1, 2p + 2) of its set
      float z0, z1;
      if (lane < 16) {
        normal_pair<float>(mword(2 * lane + 1), mword(2 * lane + 2), z0, z1);
        zm[2 * lane] = z0;
        zm[2 * lane + 1] = z1;
        normal_pair<float>(sword(2 * lane + 33), sword(2 * lane + 34), z0, z1);
        zp[2 * lane] = z0;
        zp[2 * lane + 1] = z1;
      } else if (sizes_normal) {
        const int q = lane - 16;
        normal_pair<float>(sword(2 * q + 1), sword(2 * q + 2), z0, z1);
        zs[2 * q] = z0;
        zs[2 * q + 1] = z1;
      }
    }
    __syncwarp();
    // component c = lane of the jump lane's step
    const int c = lane;
    const float th = Ar<float>::u01(sword(0));
    const float d0 = __fmul_rn(kp.dt, th), d1 = __fmul_rn(kp.dt, __fsub_rn(1.f, th));
    float bc = 0.f;
#pragma unroll
    for (int l = 0; l < DU32; ++l) bc = __fmaf_rn(kp.B[c * DU32 + l], __ldg(u + (size_t)k * DU32 + l), bc);
    float xc = __fmaf_rn(__fmul_rn(kp.sigma[c], __fsqrt_rn(d0)), zm[c], xv[c]);
    xc = __fmaf_rn(d0, __fadd_rn(fv[c], bc), xc);
    if (sizes_normal)
      xc = __fadd_rn(xc, __fmul_rn(kp.jump_scale, zs[c]));
    else
      xc = __fadd_rn(xc, __fmul_rn(kp.jump_scale, __fsub_rn(__fmul_rn(2.f, Ar<float>::u01(sword(1 + c))), 1.f)));
    yv[c] = xc;
    __syncwarp();
    float acc = 0.f;   // (A Y_1)_c
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) acc = __fmaf_rn(at[kk * 32 + c], yv[kk], acc);
    xc = __fmaf_rn(__fmul_rn(kp.sigma[c], __fsqrt_rn(d1)), zp[c], xc);
    xv[c] = __fmaf_rn(d1, __fadd_rn(acc, bc), xc);
    __syncwarp();
    if (lane == j) {
#pragma unroll
      for (int cc = 0; cc < 32; ++cc) {
        x[cc] = xv[cc];
        y1[cc] = yv[cc];
      }
      th_out = th;
    }
    __syncwarp();   // the scratch is the next jump lane's
  }
  return th_out;
}

// bu[k][c] = sum_l B[c][l] u_k[l] (FP32, multiply-adds in the order l = 0..3 from zero):
// the control's drift term is the same for every path, so it is formed once per step.
__global__ void bu32_kernel(const KP32 *__restrict__ kpg, const float *__restrict__ u, float *__restrict__ bu,
                            int Nt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nt * 32) return;
  const int k = i >> 5, c = i & 31;
  float bc = 0.f;
#pragma unroll
  for (int l = 0; l < DU32; ++l) bc = __fmaf_rn(kpg->B[c * DU32 + l], u[(size_t)k * DU32 + l], bc);
  bu[i] = bc;
}

template <int TC>
__global__ void __launch_bounds__(TPB, 4)
fwd32_kernel(const KP32 *__restrict__ kpg, const float *__restrict__ u, const float *__restrict__ bu,
             const float *__restrict__ xd,
             double *__restrict__ partC, float *__restrict__ traj, uint32_t *__restrict__ flags,
             float *__restrict__ pcost, JLog<float, D32> jl, int *__restrict__ jcnt, int *status,
             int64_t mloc, const __grid_constant__ RoundKeys rk) {
  constexpr bool SPLIT = TC == 2;
  __shared__ __align__(1024) TcShared sh;
  __shared__ __align__(16) CcShared cs;
  __shared__ __align__(16) float vbuf[32 * TPB];   // product staging (CUDA cores, jump steps)
  __shared__ Pair<float> red[TPB / 32];
  stage_params(cs, kpg);
  const KP32 &kp = cs.kp;
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
      cc_matvec(cs.at, vbuf + threadIdx.x, x, f);
    }
    bool jump;
    const uint32_t w0 = main_noise_or_jump(kp, rk, k, m, x, vbuf + threadIdx.x, jump);   // x += noise unless jump
    if (TC) tc_collect(sh, (uint32_t)(k & 1), f, status);
    const bool one = jump && kp.npair == 16 && (unsigned long long)w0 < kp.thr[1];
    if (!jump) {
      const float4 *b4 = reinterpret_cast<const float4 *>(bu + (size_t)k * 32);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 bc = __ldg(b4 + q);
        const float2 s01 = __fadd2_rn(make_float2(f[4 * q], f[4 * q + 1]), make_float2(bc.x, bc.y));
        const float2 s23 = __fadd2_rn(make_float2(f[4 * q + 2], f[4 * q + 3]), make_float2(bc.z, bc.w));
        Pr<float>::fma(kp.dt, kp.dt, s01.x, s01.y, x[4 * q], x[4 * q + 1]);
        Pr<float>::fma(kp.dt, kp.dt, s23.x, s23.y, x[4 * q + 2], x[4 * q + 3]);
      }
    }
    const unsigned om = __ballot_sync(0xffffffffu, one);   // every lane of the warp is in the loop
    if (__builtin_expect(om != 0u, 0)) {
      float y1[32];
      const float th = coop_one_jumps(kp, cs.at, vbuf + (threadIdx.x & ~31u), k, m, u, om, x, f, y1);
      if (one) {
        fw |= 1u << (k & 31);
        if (lw.fits(1)) lw.put(k, 0, th, y1);
      }
    }
    if (jump && !one) {
      // two or more jumps (rare): the generic routine on the CUDA cores (x is X_k)
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
          lw.put(k, i, S.th[i], y);
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

// Adjoint of a step with jumps (linear drift), out of line: sub-steps n..0 with the
// Jacobian A; sub-step n uses this step's A^T lambda (t), earlier ones the CUDA cores.
__device__ __noinline__ void adj32_jump_substeps(const KP32 &kp, float *vcol, int k, uint32_t m,
                                                 LogReader<float, D32> *lr, float *muio, const float *tin,
                                                 float *gout) {
  float mu[32], t[32], g[DU32], th[NMAX];
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    mu[c] = muio[c];
    t[c] = tin[c];
  }
#pragma unroll
  for (int l = 0; l < DU32; ++l) g[l] = 0.f;
  int n = 0;
  if (lr->has(k)) {
    float tmp[32];
    while (lr->has(k) && n < NMAX) {
      lr->pop(th[n], tmp);
      ++n;
    }
    for (int i = 0; i < n / 2; ++i) {   // popped latest first: reverse into time order
      const float a = th[i];
      th[i] = th[n - 1 - i];
      th[n - 1 - i] = a;
    }
  } else {
    const uint4 o0 = philox10((uint32_t)k, m, 0u, kp.epoch, kp.key0, kp.key1);
    for (int i = 0; i < NMAX; ++i) n += ((unsigned long long)o0.x >= kp.thr[i]) ? 1 : 0;
    regen_jump_times(kp, k, m, n, th);
  }
  float thn = 1.f;
  for (int i = n; i >= 0; --i) {
    const float the = i > 0 ? th[i - 1] : 0.f;
    const float de = i > 0 ? __fmul_rn(kp.dt, __fsub_rn(thn, the)) : __fmul_rn(kp.dt, thn);
    control_sensitivity(kp, mu, de, g);
    if (i < n) cc_matvec(kp.A, vcol, mu, t);
#pragma unroll
    for (int c = 0; c < 32; ++c) mu[c] = __fmaf_rn(de, t[c], mu[c]);
    thn = the;
  }
#pragma unroll
  for (int c = 0; c < 32; ++c) muio[c] = mu[c];
#pragma unroll
  for (int l = 0; l < DU32; ++l) gout[l] = g[l];
}

// mu <- mu + de (A^T mu) for every lane of om, the product formed by the whole warp: the
// lane's costate goes to the warp's scratch (row 0 of ws, its 32 x TPB floats of vbuf)
// and lane c forms component c in cc_matvec's order (k from 0, from zero), into row 1.
__device__ __forceinline__ void coop_adj_product(const float *A, float *ws, unsigned om, float de, float (&mu)[32]) {
  const int lane = threadIdx.x & 31;
  float *mv = ws, *tv = ws + TPB;
  while (om) {
    const int j = __ffs(om) - 1;
    om &= om - 1;
    if (lane == j) {
#pragma unroll
      for (int c = 0; c < 32; ++c) mv[c] = mu[c];
    }
    __syncwarp();
    float acc = 0.f;
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) acc = __fmaf_rn(A[kk * 32 + lane], mv[kk], acc);
    tv[lane] = acc;
    __syncwarp();
    if (lane == j) {
#pragma unroll
      for (int c = 0; c < 32; ++c) mu[c] = __fmaf_rn(de, tv[c], mu[c]);
    }
    __syncwarp();   // the scratch is the next lane's
  }
}

template <int TC>
__global__ void __launch_bounds__(TPB, 4)
adj32_kernel(const KP32 *__restrict__ kpg, const float *__restrict__ u, const float *__restrict__ xd,
             const float *__restrict__ traj, const uint32_t *__restrict__ flags, JLog<float, D32> jl,
             const int *__restrict__ jcnt, double *__restrict__ partG, float *__restrict__ lam_out,
             int *status, int64_t mloc) {
  constexpr bool SPLIT = TC == 2;
  __shared__ __align__(1024) TcShared sh;
  __shared__ __align__(16) CcShared cs;
  __shared__ __align__(16) float vbuf[32 * TPB];   // product staging (CUDA cores, jump sub-steps)
  stage_params(cs, kpg);
  const KP32 &kp = cs.kp;
  const int64_t npart = kp.npart;
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
    if (k >= 2) {   // the next step's stored state, into L2 ahead of its use
#pragma unroll
      for (int c4 = 0; c4 < 8; ++c4)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(traj + (((size_t)(k - 1) * 8 + c4) * mloc + lmc) * 4));
    }
    float t[32];
    if (TC)
      tc_collect(sh, (uint32_t)((Nt - 1 - k) & 1), t, status);
    else
      cc_matvec(cs.kp.A, vbuf + threadIdx.x, mu, t);
    float g[DU32];
#pragma unroll
    for (int l = 0; l < DU32; ++l) g[l] = 0.f;
    if (!jumped) {
      control_sensitivity(kp, mu, kp.dt, g);
#pragma unroll
      for (int c = 0; c < 32; c += 2) Pr<float>::fma(kp.dt, kp.dt, t[c], t[c + 1], mu[c], mu[c + 1]);
    }
    // CUDA cores: a step with one jump at fraction th takes sub-step 1 (length dt (1 - th))
    // with this step's product, then sub-step 0 (length dt th) with A^T of the updated
    // costate, formed by the whole warp one component per lane (cc_matvec's order: the same
    // bits); a step with more jumps, and every jump step with the tensor cores, takes the
    // one-lane routine (measured: the warp-wide form there slowed the jump-free steps more,
    // 5.8 -> 6.9 ms per sweep, than it saved on the jump steps)
    bool one = false;
    float de0 = 0.f;
    if (jumped) {
      const uint32_t w0 = TC == 0 ? philox10((uint32_t)k, m, 0u, kp.epoch, kp.key0, kp.key1).x : 0xffffffffu;
      one = TC == 0 && (unsigned long long)w0 < kp.thr[1];
      if (one) {
        float th;
        if (lr.has(k)) {
          float ylog[32];
          lr.pop(th, ylog);
        } else {
          th = Ar<float>::u01(
              philox10((uint32_t)k, m, (1u << 24) | (1u << 16), kp.epoch, kp.key0, kp.key1).x);
        }
        const float de1 = __fmul_rn(kp.dt, __fsub_rn(1.f, th));
        control_sensitivity(kp, mu, de1, g);
#pragma unroll
        for (int c = 0; c < 32; ++c) mu[c] = __fmaf_rn(de1, t[c], mu[c]);
        de0 = __fmul_rn(kp.dt, th);
        control_sensitivity(kp, mu, de0, g);
      } else {
        float ml[32], tl[32], gl[DU32];
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          ml[c] = mu[c];
          tl[c] = t[c];
        }
        adj32_jump_substeps(kp, vbuf + threadIdx.x, k, m, &lr, ml, tl, gl);
#pragma unroll
        for (int c = 0; c < 32; ++c) mu[c] = ml[c];
#pragma unroll
        for (int l = 0; l < DU32; ++l) g[l] = gl[l];
      }
    }
    if constexpr (TC == 0) {
      const unsigned om = __ballot_sync(0xffffffffu, one);   // every lane of the warp is in the loop
      if (__builtin_expect(om != 0u, 0)) coop_adj_product(kp.A, vbuf + (threadIdx.x & ~31u), om, de0, mu);
    }
    if (k >= 1) {
      // cost gradient dt q (X_k - xd_k), the stored state streamed 4 components at a time
#pragma unroll
      for (int c4 = 0; c4 < 8; ++c4) {
        float v[4];
        Vec4<float>::load(traj + (((size_t)k * 8 + c4) * mloc + lmc) * 4, v);
#pragma unroll
        for (int q = 0; q < 4; q += 2) {   // paired: the rounding of __fsub_rn / __fmaf_rn per component
          const int c = 4 * c4 + q;
          float e0, e1;
          Pr<float>::sub(v[q], v[q + 1], __ldg(xd + (size_t)k * D32 + c), __ldg(xd + (size_t)k * D32 + c + 1), e0, e1);
          Pr<float>::fma(kp.qdt[c], kp.qdt[c + 1], e0, e1, mu[c], mu[c + 1]);
        }
      }
    }
    if (lam_out && active)
#pragma unroll
      for (int c = 0; c < 32; ++c) lam_out[((size_t)k * D32 + c) * mloc + lm] = mu[c];
    // per-step, per-warp compensated sums of the four control sensitivities, transposed:
    // at offset 16 a lane keeps two components and sends the other two, at offset 8 one,
    // then one pair per lane through offsets 4, 2, 1 (12 shuffles and 6 TwoSums instead of
    // 40 and 20 for four separate butterflies); lane 8 c then holds component c's sum
    static_assert(DU32 == 4, "the transposed reduction takes four components");
    {
      Pair<float> v[4];
#pragma unroll
      for (int l = 0; l < 4; ++l) v[l] = Pair<float>{active ? g[l] : 0.f, 0.f};
      const bool up16 = (lane & 16) != 0, up8 = (lane & 8) != 0;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const Pair<float> send = up16 ? v[i] : v[i + 2];
        const Pair<float> keep = up16 ? v[i + 2] : v[i];
        v[i] = padd(keep, shfl_xor(send, 16));
      }
      {
        const Pair<float> send = up8 ? v[0] : v[1];
        const Pair<float> keep = up8 ? v[1] : v[0];
        v[0] = padd(keep, shfl_xor(send, 8));
      }
#pragma unroll
      for (int o = 4; o >= 1; o >>= 1) v[0] = padd(v[0], shfl_xor(v[0], o));
      if ((lane & 7) == 0)
        partG[((int64_t)k * DU32 + (lane >> 3)) * npart + wid] = (double)v[0].s + (double)v[0].e;
    }
  }
  if (TC) tc_teardown(sh);
}

}  // namespace jd
