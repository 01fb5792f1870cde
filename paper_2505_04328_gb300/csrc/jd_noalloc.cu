// jd_noalloc.cu -- J(u) for callers that cannot allocate device memory.
//
// Some callers must not allocate once they are running: a real-time control loop
// (a cudaMalloc can take milliseconds and synchronizes the device), or a host
// application whose memory pool has reserved the whole GPU and forbids foreign
// allocations.  jd_cost_noalloc serves them: it evaluates the same forward cost
// kernel as jd_cost, but its scratch (the padded control and target in kernel
// precision and the per-block cost partials) lives in one fixed file-scope device
// array, so the call allocates nothing, on the device or on the host.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "jd_kernels.cuh"

namespace jd {

// Scratch shared by every jd_cost_noalloc call on a device.  Every GPU that loads
// this library holds it until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)4 << 20;   // 4 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device addresses of g_noalloc_scratch, taken once per device with that device current.
constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_ptr[kNoAllocMaxDevices];
static size_t g_noalloc_stack[kNoAllocMaxDevices][4];   // local bytes per thread of each cost kernel

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Target (FP64, unpadded) -> kernel precision padded to D; control (FP64, Nt*du) ->
// kernel precision, one column.
template <typename R>
__global__ void noalloc_prep_kernel(const double *__restrict__ xd64, int Nt, int d, int D,
                                    R *__restrict__ xdk, const double *__restrict__ u, R *__restrict__ uk) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (int64_t)(Nt + 1) * D) {
    const int64_t k = i / D;
    const int c = (int)(i % D);
    xdk[i] = c < d ? (R)xd64[k * d + c] : R(0);
  }
  if (i < Nt) uk[i] = (R)u[i];
}

// J = (1/M) sum_b partC[b] + (nu dt / 2) sum_k u_k^2, fixed summation order.
__global__ void noalloc_finalize_kernel(const double *__restrict__ partC, int64_t nblk,
                                        const double *__restrict__ u, int n, double half_nu_dt,
                                        double invM, double *__restrict__ J) {
  __shared__ double sm[2][8];
  double a = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < nblk; i += blockDim.x) a += partC[i];
  for (int i = threadIdx.x; i < n; i += blockDim.x) b += u[i] * u[i];
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sm[0][w] = a;
    sm[1][w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      sa += sm[0][i];
      sb += sm[1][i];
    }
    *J = sa * invM + half_nu_dt * sb;
  }
}

// Kernel parameters straight from the descriptor (no problem object, no allocation).
template <typename R, int D, int DU>
static void noalloc_kparams(const jd_problem_desc &q, KParams<R, D, DU> &kp) {
  const int d = q.d;
  const double dt = q.T / (double)q.Nt, sqdt = std::sqrt(dt);
  for (int i = 0; i < D * D; ++i) kp.A[i] = kp.C[i] = kp.dA[i] = R(0);
  for (int i = 0; i < D * DU; ++i) kp.B[i] = R(0);
  for (int i = 0; i < d; ++i) {
    for (int j = 0; j < d; ++j) {
      kp.A[i * D + j] = (R)q.A[i * d + j];
      if (q.drift == JD_DRIFT_CUBIC) kp.C[i * D + j] = (R)q.C[i * d + j];
    }
    kp.B[i * DU] = (R)q.B[i];
  }
  for (int c = 0; c < D; ++c) {
    const bool in = c < d;
    kp.sigma[c] = in ? (R)q.sigma[c] : R(0);
    kp.sig_sqdt[c] = in ? (R)(q.sigma[c] * sqdt) : R(0);
    kp.qdt[c] = in ? (R)(q.q[c] * dt) : R(0);
    kp.hqdt[c] = in ? (R)(0.5 * q.q[c] * dt) : R(0);
    kp.x0[c] = in ? (R)q.x0[c] : R(0);
    kp.jgain[c] = R(1);   // the additive laws only (a Keilson-Storer problem is rejected)
    kp.jscl[c] = (R)q.jump_scale;
  }
  kp.dt = (R)dt;
  kp.sqdt = (R)sqdt;
  kp.jump_scale = (R)q.jump_scale;
  kp.kvel = 0;
  poisson_thresholds(q.lambda * dt, kp.thr);
  set_philox_key(kp, q.seed);
  kp.epoch = q.epoch;
  kp.d = d;
  kp.npair = (d + 1) / 2;
  kp.Nt = q.Nt;
  kp.cubic = q.drift == JD_DRIFT_CUBIC;
  kp.jump_law = (int)q.jump_law;
  kp.jumps_on = q.jump_law != JD_JUMP_NONE && q.lambda > 0.0;
  kp.has_dA = 0;
  kp.S = seg_len<D>();
  kp.nblk = (int)ceil_div(q.M, TPB);
  kp.m_begin = q.m_offset;   // global index of the first path
  kp.npart = kp.nblk * (int64_t)(TPB / 32);
}

template <typename R, int D>
static jd_status noalloc_run(const jd_problem_desc &q, unsigned char *scratch, const double *u,
                             double *J) {
  cudaStream_t s = (cudaStream_t)q.cuda_stream;
  const int Nt = q.Nt;
  const int64_t M = q.M, nblk = ceil_div(M, TPB);
  unsigned char *p = scratch;
  double *xd64 = reinterpret_cast<double *>(p);
  p += align256((size_t)(Nt + 1) * q.d * sizeof(double));
  R *xdk = reinterpret_cast<R *>(p);
  p += align256((size_t)(Nt + 1) * D * sizeof(R));
  R *uk = reinterpret_cast<R *>(p);
  p += align256((size_t)Nt * sizeof(R));
  double *partC = reinterpret_cast<double *>(p);
  // every scratch entry that is read is written earlier in the same call, so
  // nothing has to be cleared
  if (cudaMemcpyAsync(xd64, q.xd, (size_t)(Nt + 1) * q.d * sizeof(double), cudaMemcpyHostToDevice, s) !=
      cudaSuccess)
    return JD_ERR_CUDA;
  const int64_t nprep = (int64_t)(Nt + 1) * D;
  noalloc_prep_kernel<R><<<(unsigned)ceil_div(nprep, 256), 256, 0, s>>>(xd64, Nt, q.d, D, xdk, u, uk);
  KParams<R, D, 1> kp;
  noalloc_kparams<R, D, 1>(q, kp);
  const JLog<R, D> nolog{nullptr, nullptr, M, 0};
  fwd_kernel<R, D, 1, FWD_COST><<<(unsigned)nblk, TPB, 0, s>>>(kp, uk, xdk, partC, nullptr, nullptr, nullptr,
                                                               nullptr, nolog, nullptr, M, PairOut<R, D>{});
  noalloc_finalize_kernel<<<1, 256, 0, s>>>(partC, nblk, u, Nt, 0.5 * q.nu * (q.T / Nt), 1.0 / (double)M, J);
  count_launch(3);
  return cudaGetLastError() == cudaSuccess ? JD_OK : JD_ERR_CUDA;
}

}  // namespace jd

using namespace jd;

extern "C" jd_status jd_cost_noalloc(const jd_problem_desc *desc, const double *u, double *J) {
  if (!desc || !u || !J) return JD_ERR_INVALID_ARG;
  const jd_problem_desc &q = *desc;
  if (q.d < 1 || q.du < 1 || q.Nt < 1 || q.M < 1 || q.M > 0xFFFFFFFFll || !(q.T > 0.0) ||
      !std::isfinite(q.T) || !q.A || !q.B || !q.sigma || !q.x0 || !q.q || !q.xd ||
      (q.drift == JD_DRIFT_CUBIC && !q.C) || q.drift < JD_DRIFT_LINEAR || q.drift > JD_DRIFT_CUBIC ||
      q.jump_law < JD_JUMP_NONE || q.jump_law > JD_JUMP_UNIFORM || !(q.lambda >= 0.0) ||
      !std::isfinite(q.lambda) || !(q.jump_scale >= 0.0) || !std::isfinite(q.jump_scale) ||
      !std::isfinite(q.nu) || (q.prec != JD_FP32 && q.prec != JD_FP64) || q.m_offset < 0 ||
      q.m_offset + q.M > 0x100000000ll)
    return JD_ERR_INVALID_ARG;
  if (q.d > 2 || q.du != 1 || q.use_tensor_cores) return JD_ERR_UNSUPPORTED;
  const int D = q.d;
  const size_t es = q.prec == JD_FP64 ? 8 : 4;
  const size_t need = align256((size_t)(q.Nt + 1) * q.d * 8) + align256((size_t)(q.Nt + 1) * D * es) +
                      align256((size_t)q.Nt * es) + align256((size_t)ceil_div(q.M, TPB) * 8);
  if (need > kNoAllocScratchBytes) return JD_ERR_OOM;   // beyond the fixed scratch

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return JD_ERR_CUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return JD_ERR_UNSUPPORTED;
  const int kid = (q.prec == JD_FP64 ? 2 : 0) + (D - 1);   // which cost kernel runs
  unsigned char *scratch = nullptr;
  size_t need_stack = 0;
  {
    // first call on a device: take the device address of the scratch array with this
    // device current (the host-side symbol is not a device address), and the per-thread
    // stack each of the four cost kernels needs
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void *ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return JD_ERR_CUDA;
      const void *ks[4] = {(const void *)fwd_kernel<float, 1, 1, FWD_COST>,
                           (const void *)fwd_kernel<float, 2, 1, FWD_COST>,
                           (const void *)fwd_kernel<double, 1, 1, FWD_COST>,
                           (const void *)fwd_kernel<double, 2, 1, FWD_COST>};
      for (int i = 0; i < 4; ++i) {
        cudaFuncAttributes a;
        if (cudaFuncGetAttributes(&a, ks[i]) != cudaSuccess) return JD_ERR_CUDA;
        g_noalloc_stack[dev][i] = a.localSizeBytes;
      }
      g_noalloc_ptr[dev] = static_cast<unsigned char *>(ptr);
    }
    scratch = g_noalloc_ptr[dev];
    need_stack = g_noalloc_stack[dev][kid];
  }
  // The context's per-thread stack must hold the kernel's local frame; refuse rather
  // than raise the limit (raising it makes the driver allocate).
  size_t stack = 0;
  if (cudaDeviceGetLimit(&stack, cudaLimitStackSize) != cudaSuccess || stack < need_stack)
    return JD_ERR_UNSUPPORTED;
  if (q.prec == JD_FP64) return D == 1 ? noalloc_run<double, 1>(q, scratch, u, J) : noalloc_run<double, 2>(q, scratch, u, J);
  return D == 1 ? noalloc_run<float, 1>(q, scratch, u, J) : noalloc_run<float, 2>(q, scratch, u, J);
}
