// d = 32 linear-drift kernels (FP32 paths; CUDA cores or tcgen05 tensor cores).
#include "jd_tc32.cuh"

namespace jd {

// Coefficients go to the problem's device buffer (stream ordered) for the kernels to stage.
static cudaError_t upload_kp(const jd_problem *p, int64_t m_begin, int64_t mloc, const PathBufs &b,
                             cudaStream_t s, KP32 **dev, RoundKeys *rk = nullptr) {
  if (!p->kp_dev) return cudaErrorInvalidValue;
  thread_local KP32 kp;   // 13 KB: not on the stack, and not allocated per launch
  make_kparams<float, D32, DU32>(p, m_begin, mloc, kp);
  if (b.npart) kp.npart = b.npart;
  if (rk) {
    for (int r = 0; r < 10; ++r) {
      rk->k0[r] = kp.rk0[r];
      rk->k1[r] = kp.rk1[r];
    }
  }
  // pageable source: the copy is staged before cudaMemcpyAsync returns
  const cudaError_t e = cudaMemcpyAsync(p->kp_dev, &kp, sizeof(KP32), cudaMemcpyHostToDevice, s);
  *dev = static_cast<KP32 *>(p->kp_dev);
  return e;
}

static cudaError_t op32_fwd(const jd_problem *p, int mode, int64_t m_begin, int64_t mloc, const void *uk,
                            const PathBufs &b, cudaStream_t s) {
  if (mode == FWD_CKPT) return cudaErrorNotSupported;
  KP32 *kp = nullptr;
  RoundKeys rk;
  const cudaError_t ue = upload_kp(p, m_begin, mloc, b, s, &kp, &rk);
  if (ue != cudaSuccess) return ue;
  const dim3 grid((unsigned)ceil_div(mloc, TPB));
  const float *u = static_cast<const float *>(uk);
  const float *xd = static_cast<const float *>(p->xdk);
  float *traj = mode == FWD_STORE ? static_cast<float *>(b.traj) : nullptr;
  const JLog<float, D32> jl{static_cast<float2 *>(b.log_kt), static_cast<float *>(b.log_y), mloc, b.log_cap};
  float *pc = static_cast<float *>(b.pcost);
  const int Nt = p->desc.Nt;
  bu32_kernel<<<(unsigned)ceil_div((int64_t)Nt * 32, 256), 256, 0, s>>>(kp, u, p->bu_dev, Nt);
  const float *bu = p->bu_dev;
  switch (p->desc.use_tensor_cores) {
    case 1:
      fwd32_kernel<1><<<grid, TPB, 0, s>>>(kp, u, bu, xd, b.partC, traj, b.flags, pc, jl, b.jcnt, b.status, mloc, rk);
      break;
    case 2:
      fwd32_kernel<2><<<grid, TPB, 0, s>>>(kp, u, bu, xd, b.partC, traj, b.flags, pc, jl, b.jcnt, b.status, mloc, rk);
      break;
    default:   // 0, and 3 (tensor cores in the adjoint only)
      fwd32_kernel<0><<<grid, TPB, 0, s>>>(kp, u, bu, xd, b.partC, traj, b.flags, pc, jl, b.jcnt, b.status, mloc, rk);
      break;
  }
  count_launch(2);
  return cudaGetLastError();
}

static cudaError_t op32_adj(const jd_problem *p, int variant, bool theta, int64_t m_begin, int64_t mloc,
                            const void *uk, const PathBufs &b, cudaStream_t s) {
  if (variant != ADJ_STORED_V || theta) return cudaErrorNotSupported;
  KP32 *kp = nullptr;
  const cudaError_t ue = upload_kp(p, m_begin, mloc, b, s, &kp);
  if (ue != cudaSuccess) return ue;
  const dim3 grid((unsigned)ceil_div(mloc, TPB));
  const float *u = static_cast<const float *>(uk);
  const float *xd = static_cast<const float *>(p->xdk);
  const float *traj = static_cast<const float *>(b.traj);
  const JLog<float, D32> jl{static_cast<float2 *>(b.log_kt), static_cast<float *>(b.log_y), mloc, b.log_cap};
  float *lo = static_cast<float *>(b.lam_out);
  switch (p->desc.use_tensor_cores) {
    case 1:
      adj32_kernel<1><<<grid, TPB, 0, s>>>(kp, u, xd, traj, b.flags, jl, b.jcnt, b.partG, lo, b.status, mloc);
      break;
    case 2:
    case 3:   // BF16 x3 in the adjoint after an FP32 CUDA-core forward
      adj32_kernel<2><<<grid, TPB, 0, s>>>(kp, u, xd, traj, b.flags, jl, b.jcnt, b.partG, lo, b.status, mloc);
      break;
    default:
      adj32_kernel<0><<<grid, TPB, 0, s>>>(kp, u, xd, traj, b.flags, jl, b.jcnt, b.partG, lo, b.status, mloc);
      break;
  }
  count_launch();
  return cudaGetLastError();
}

static size_t op32_stack() {
  size_t need = 4 * sizeof(JumpStep<float, D32>) + 2048;   // >= the cumulative frames reported by ptxas
  const void *ks[] = {(const void *)fwd32_kernel<0>, (const void *)fwd32_kernel<1>, (const void *)fwd32_kernel<2>,
                      (const void *)adj32_kernel<0>, (const void *)adj32_kernel<1>, (const void *)adj32_kernel<2>};
  for (const void *k : ks) {
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, k) == cudaSuccess && a.localSizeBytes + 1024 > need) need = a.localSizeBytes + 1024;
  }
  return (need + 255) & ~(size_t)255;
}

extern const PathOps ops_f32_d32_u4 = PathOps{D32, DU32, 8, 4, 1, &op32_stack, &op32_fwd, &op32_adj, nullptr,
                                                    nullptr, nullptr};

}  // namespace jd
