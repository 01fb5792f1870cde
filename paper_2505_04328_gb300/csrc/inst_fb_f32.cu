// Feedback-control kernels, FP32 path arithmetic (FP64 reductions), padded 4x4, 10x10
// and 16x16 weights per step; the FP64 finalize of both precisions.
#include "jd_feedback.cuh"

namespace jd {

extern const FbOps fb_ops_f32[3] = {fb_make_ops<float, 4, 4>(), fb_make_ops<float, 10, 10>(),
                                    fb_make_ops<float, 16, 16>()};

__global__ void fb_finalize_kernel(const double *__restrict__ partC, const double *__restrict__ partG,
                                   int64_t nblk, int64_t ngroup, int Nt, int nx, int nv, int NX, int NV,
                                   int64_t M, double *__restrict__ J, double *__restrict__ grad) {
  const int64_t n = (int64_t)Nt * nx * nv, ncol = (int64_t)Nt * NX * NV;
  const double inv = 1.0 / (double)M;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t / (nx * nv);
    const int r = (int)(t - k * nx * nv), i = r / nv, l = r - i * nv;
    const int64_t src = k * NX * NV + ((i / 2) * NV + l) * 2 + (i & 1);   // pair layout
    double s = 0.0;
#pragma unroll 8
    for (int64_t g = 0; g < ngroup; ++g) s += partG[g * ncol + src];
    grad[t] = s * inv;
  }
  if (J && blockIdx.x == 0) {
    // J: block 0's threads take partC[t], partC[t + 128], ... then a fixed tree
    __shared__ double red[128];
    double s = 0.0;
    for (int64_t b = threadIdx.x; b < nblk; b += blockDim.x) s += partC[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = 64; h >= 1; h >>= 1) {
      if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) *J = red[0] * inv;
  }
}

// |g|^2_{L2} = dt sum_t (grad_t / dt)^2 in one block, fixed order (strided sums, then a
// tree); and the trial point mu_t = mu - zeta (grad / dt) with the oracle's rounding.
__global__ void fb_norm_kernel(const double *__restrict__ grad, int64_t n, double dt, double *__restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
    const double g = __ddiv_rn(grad[t], dt);
    s = __dadd_rn(s, __dmul_rn(dt, __dmul_rn(g, g)));
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h >= 1; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void fb_trial_kernel(const double *__restrict__ mu, const double *__restrict__ grad, int64_t n,
                                double zeta, double dt, double *__restrict__ mt) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    mt[t] = __dsub_rn(mu[t], __dmul_rn(zeta, __ddiv_rn(grad[t], dt)));
}

cudaError_t fb_norm(const double *grad, int64_t n, double dt, double *out, cudaStream_t s) {
  fb_norm_kernel<<<1, 256, 0, s>>>(grad, n, dt, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t fb_trial(const double *mu, const double *grad, int64_t n, double zeta, double dt, double *mt,
                     cudaStream_t s) {
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 1024));
  fb_trial_kernel<<<grid, 256, 0, s>>>(mu, grad, n, zeta, dt, mt);
  count_launch();
  return cudaGetLastError();
}

cudaError_t fb_finalize(const double *partC, const double *partG, int64_t nblk, int64_t ngroup, int Nt, int nx,
                        int nv, int NX, int NV, int64_t M, double *J, double *grad, cudaStream_t s) {
  const int64_t n = grad ? (int64_t)Nt * nx * nv : 0;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 128), 4096));
  fb_finalize_kernel<<<grid, 128, 0, s>>>(partC, grad ? partG : nullptr, nblk, ngroup, grad ? Nt : 0, nx, nv, NX,
                                         NV, M, J, grad);
  count_launch();
  return cudaGetLastError();
}

}  // namespace jd
