// jd_internal.h -- types shared by the host library and the path kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "jd.h"

namespace jd {

constexpr int NMAX = 16;   // jumps per uniform step are capped at this count
constexpr int TPB = 128;   // threads (one path each) per block of the path kernels
constexpr int BATCH = 8;   // steps per transposed warp reduction

enum FwdMode { FWD_COST = 0, FWD_STORE = 1, FWD_CKPT = 2 };
enum AdjVariant { ADJ_STORED_V = 1, ADJ_RECOMPUTE_V = 2 };

// Kernel parameters: coefficients padded to the compiled dimensions D, DU and passed
// by value, so the hot loop reads them as constant-bank operands.
template <typename R, int D, int DU>
struct KParams {
  R A[D * D], C[D * D], dA[D * D], B[D * DU];
  R sigma[D];      // sigma_c
  R sig_sqdt[D];   // sigma_c * sqrt(dt)
  R qdt[D];        // q_c * dt            (cost gradient)
  R hqdt[D];       // q_c * dt / 2        (cost)
  R x0[D];
  R dt, sqdt, jump_scale;
  unsigned long long thr[NMAX];  // Poisson thresholds floor(2^32 F(n; lambda dt))
  uint32_t key0, key1, epoch;
  int d, npair, Nt, cubic, jump_law, jumps_on, has_dA, S, nblk;
  int64_t m_begin;                // global index of path 0 of this launch
};

// Device buffers of one launch (unused ones are null).
struct PathBufs {
  void *traj = nullptr;        // stored states
  uint32_t *flags = nullptr;   // jump flags, 1 bit per path-step
  void *ckpt = nullptr;        // checkpoints (recompute variant)
  void *pcost = nullptr;       // per-path cost (optional)
  void *log_kt = nullptr;      // jump log: (step, time fraction) per record
  void *log_y = nullptr;       // jump log: post-jump states
  int *jcnt = nullptr;         // jump log: records per path
  int log_cap = 0;             // jump log: records per path capacity
  double *partC = nullptr, *partG = nullptr, *partT = nullptr;
  void *lam_out = nullptr;     // adjoint states (optional)
  int *status = nullptr;       // device status word (bounded waits record timeouts here)
};

// Per-instantiation launch table (one entry per precision x compiled dimension).
struct PathOps {
  int D, DU, S, elem;
  int traj_layout;   // 0: [ceil((Nt+1)/4)][D][M][4]; 1: [Nt+1][D/4][M][4]
  // per-thread stack bytes the kernels of this instantiation may need (the jump path
  // keeps its sub-step states in local memory behind a non-inlined call)
  size_t (*stack_bytes)();
  // forward sweep in mode FWD_COST / FWD_STORE / FWD_CKPT
  cudaError_t (*fwd)(const struct ::jd_problem *p, int mode, int64_t m_begin, int64_t mloc,
                     const void *uk, const PathBufs &b, cudaStream_t s);
  // adjoint sweep: per-step gradient partials [Nt][DU][nblk * TPB/32] (one per warp);
  // theta partials [D+2][nblk]
  cudaError_t (*adj)(const struct ::jd_problem *p, int variant, bool theta, int64_t m_begin,
                     int64_t mloc, const void *uk, const PathBufs &b, cudaStream_t s);
};

const PathOps *path_ops_dims(int prec, int D, int DU);
int compiled_dim(int d);         // smallest compiled D >= d, or 0

void count_launch(int n = 1);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Gradient partials per launch of mloc paths: one per warp of every block.
inline int64_t grad_parts(int64_t mloc) { return ceil_div(mloc, TPB) * (TPB / 32); }

}  // namespace jd

// Host-side problem object (opaque to the ABI user).
struct jd_problem {
  jd_problem_desc desc;              // scalars; array pointers are cleared
  std::vector<double> A, C, B, dA, sigma, x0, q, xd;
  int D = 0, DU = 0;
  const jd::PathOps *ops = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  size_t budget = 0;
  jd_adjoint_mode plan = JD_ADJ_AUTO;
  // device buffers
  void *uk = nullptr;        // kernel-precision padded control, Nt*DU
  void *xdk = nullptr;       // kernel-precision padded target, (Nt+1)*D
  double *u_in = nullptr;    // FP64 control copy, Nt*du
  double *grad_d = nullptr;  // FP64 gradient, Nt*du
  double *scal_d = nullptr;  // FP64 scalars: J, theta grads, optimizer values
  double *partC = nullptr, *partG = nullptr, *partT = nullptr;
  void *traj = nullptr;
  uint32_t *flags = nullptr;
  void *ckpt = nullptr;
  void *log_kt = nullptr, *log_y = nullptr;
  int *jcnt = nullptr;
  int log_cap = 0;
  double *opt_u = nullptr, *opt_ut = nullptr, *opt_g = nullptr;
  int *status_d = nullptr;   // kernel status word (JD_OK or JD_ERR_TIMEOUT)
  void *kp_dev = nullptr;    // coefficient struct of the d = 32 kernels (device copy)
  double *host_pinned = nullptr;  // small pinned staging buffer
  size_t bytes = 0;
  int64_t nblk = 0;
};
