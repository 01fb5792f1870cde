/*
 * jd_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see jd_oracle.h).
 *
 * Written for readability: one path at a time, the paper's order of operations,
 * no blocking, fusion or reordering.  Threads only split the path range; every
 * sum is taken in a fixed order so results do not depend on the thread count.
 */
#include "jd_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, as published by Salmon et al. (SC'11): ten rounds of two     */
/* 32x32->64 multiplies, the key bumped by the Weyl constants between rounds.  */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t key[2], const uint32_t ctr[4], uint32_t out[4]) {
  const uint32_t MUL0 = 0xD2511F53u, MUL1 = 0xCD9E8D57u;
  const uint32_t WEYL0 = 0x9E3779B9u, WEYL1 = 0xBB67AE85u;
  uint32_t k0 = key[0], k1 = key[1];
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += WEYL0;
      k1 += WEYL1;
    }
    uint64_t prod0 = (uint64_t)MUL0 * (uint64_t)x0;
    uint64_t prod1 = (uint64_t)MUL1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

double orc_u01(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Words 0..nwords-1 of one stream: word j is word (j mod 4) of the Philox block
 * with counter (k, m, purpose<<24 | slot<<16 | j/4, epoch). */
static void stream_words(const orc_problem *P, int k, int64_t m, uint32_t purpose, uint32_t slot,
                         int nwords, uint32_t *w) {
  uint32_t key[2] = {(uint32_t)(P->seed & 0xffffffffu), (uint32_t)(P->seed >> 32)};
  for (int j = 0; j < nwords; j += 4) {
    uint32_t ctr[4] = {(uint32_t)k, (uint32_t)m, (purpose << 24) | (slot << 16) | (uint32_t)(j / 4),
                       P->epoch};
    uint32_t blk[4];
    orc_philox4x32_10(key, ctr, blk);
    for (int t = 0; t < 4 && j + t < nwords; ++t) w[j + t] = blk[t];
  }
}

/* Box-Muller: one pair of standard normals from two words. */
static void normal_pair(uint32_t wa, uint32_t wb, double *z0, double *z1) {
  double ua = orc_u01(wa), ub = orc_u01(wb);
  double r = sqrt(-2.0 * log(ua));
  *z0 = r * cos(2.0 * M_PI * ub);
  *z1 = r * sin(2.0 * M_PI * ub);
}

/* d standard normals from words w[0..2*ceil(d/2)-1]. */
static void normals_from_words(int d, const uint32_t *w, double *z) {
  for (int p = 0; 2 * p < d; ++p) {
    double a, b;
    normal_pair(w[2 * p], w[2 * p + 1], &a, &b);
    z[2 * p] = a;
    if (2 * p + 1 < d) z[2 * p + 1] = b;
  }
}

/* Poisson CDF thresholds, pmf accumulated in order p_0 = e^-mu, p_n = p_{n-1} mu / n. */
void orc_poisson_thresholds(double mu, uint64_t thr[ORC_NMAX]) {
  double p = exp(-mu), F = p;
  for (int n = 0; n < ORC_NMAX; ++n) {
    if (n > 0) {
      p = p * mu / (double)n;
      F = F + p;
    }
    double t = floor(F * 4294967296.0);
    if (t > 4294967296.0) t = 4294967296.0;
    if (t < 0.0) t = 0.0;
    thr[n] = (uint64_t)t;
  }
}

int orc_poisson_count(uint32_t w, const uint64_t thr[ORC_NMAX]) {
  /* n = #{n : T_n <= w}, so that P(count <= n) = P(w < T_n) = T_n / 2^32 ~ F(n) */
  int n = 0;
  for (int i = 0; i < ORC_NMAX; ++i)
    if ((uint64_t)w >= thr[i]) n++;
  return n;
}

void orc_normal_pair(uint32_t wa, uint32_t wb, double z[2]) { normal_pair(wa, wb, &z[0], &z[1]); }

static int jumps_enabled(const orc_problem *P) {
  return P->jump_law != ORC_JUMP_NONE && P->lambda > 0.0;
}

/* The draws of uniform step k of path m: Poisson count from main-stream word 0,
 * sub-step-0 normals from main-stream words 1.., and for every jump slot i a time
 * fraction, a jump size and the normals of the sub-step that starts at that jump.
 * Jump times are sorted (stable) and each slot's size and normals travel with its
 * time.  This is the per-step form of Algorithm 5.2's jump-time sampling: given the
 * count, the times of a Poisson process on a step are uniform order statistics. */
int orc_step_draws(const orc_problem *P, int k, int64_t m, orc_draws *D) {
  const int d = P->d, npair = (d + 1) / 2;
  const double dt = P->T / (double)P->Nt;
  uint32_t w[1 + 2 * ((ORC_DMAX + 1) / 2) + 2 * ((ORC_DMAX + 1) / 2) + 4];

  memset(D, 0, sizeof(*D));
  stream_words(P, k, m, 0u, 0u, 1 + 2 * npair, w);
  int n = 0;
  if (jumps_enabled(P)) {
    uint64_t thr[ORC_NMAX];
    orc_poisson_thresholds(P->lambda * dt, thr);
    n = orc_poisson_count(w[0], thr);
  }
  D->n = n;
  normals_from_words(d, w + 1, D->Z[0]);

  /* slots in draw order */
  double theta[ORC_NMAX], xi[ORC_NMAX][ORC_DMAX], zs[ORC_NMAX][ORC_DMAX];
  for (int i = 0; i < n; ++i) {
    stream_words(P, k, m, 1u, (uint32_t)(i + 1), 1 + 4 * npair, w);
    theta[i] = orc_u01(w[0]);
    if (P->jump_law == ORC_JUMP_NORMAL || P->jump_law == ORC_JUMP_KS) {
      normals_from_words(d, w + 1, xi[i]);
    } else {
      for (int c = 0; c < d; ++c) xi[i][c] = 2.0 * orc_u01(w[1 + c]) - 1.0;
    }
    normals_from_words(d, w + 1 + 2 * npair, zs[i]);
  }
  /* stable insertion sort of the slots by time */
  int order[ORC_NMAX];
  for (int i = 0; i < n; ++i) order[i] = i;
  for (int i = 1; i < n; ++i) {
    int cur = order[i], j = i - 1;
    while (j >= 0 && theta[order[j]] > theta[cur]) {
      order[j + 1] = order[j];
      j--;
    }
    order[j + 1] = cur;
  }
  for (int i = 0; i < n; ++i) {
    D->theta[i] = theta[order[i]];
    memcpy(D->xi_hat[i], xi[order[i]], sizeof(double) * d);
    memcpy(D->Z[i + 1], zs[order[i]], sizeof(double) * d);
  }
  /* sub-step lengths between consecutive grid points of the jump-adapted grid */
  if (n == 0) {
    D->delta[0] = dt;
  } else {
    D->delta[0] = dt * D->theta[0];
    for (int i = 1; i < n; ++i) D->delta[i] = dt * (D->theta[i] - D->theta[i - 1]);
    D->delta[n] = dt * (1.0 - D->theta[n - 1]);
  }
  return 0;
}

/* f(y,u) = A y + C y^3 + B u */
static void drift(const orc_problem *P, const double *y, const double *u, double *f) {
  const int d = P->d, du = P->du;
  for (int i = 0; i < d; ++i) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) s += P->A[i * d + j] * y[j];
    if (P->drift == ORC_CUBIC)
      for (int j = 0; j < d; ++j) s += P->C[i * d + j] * y[j] * y[j] * y[j];
    for (int l = 0; l < du; ++l) s += P->B[i * du + l] * u[l];
    f[i] = s;
  }
}

/* out = J_f(y)^T v,  J_f = A + 3 C diag(y^2) */
static void drift_jacobian_T(const orc_problem *P, const double *y, const double *v, double *out) {
  const int d = P->d;
  for (int j = 0; j < d; ++j) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) {
      double Jij = P->A[i * d + j];
      if (P->drift == ORC_CUBIC) Jij += 3.0 * P->C[i * d + j] * y[j] * y[j];
      s += Jij * v[i];
    }
    out[j] = s;
  }
}

/* The jump map c acts on component c of the state: additive jumps move every component,
 * y + s xi (NORMAL, UNIFORM); the Keilson-Storer reset (Sec. 5.3 Eq. jump_law) acts on
 * the velocity half of the state z = (x, v), components c >= d/2: v <- gamma v + s xi,
 * positions unchanged.  jump_gain_of is the diagonal of the map's Jacobian. */
static int jump_acts_on(const orc_problem *P, int c) {
  return P->jump_law != ORC_JUMP_KS || c >= P->d / 2;
}

static double jump_gain_of(const orc_problem *P, int c) {
  return (P->jump_law == ORC_JUMP_KS && c >= P->d / 2) ? P->jump_gain : 1.0;
}

/* Sub-step start states of step k (Algorithm 5.1): Y[0] = X_k; Euler sub-step of
 * length delta_i with the drift at its left end; the jump of slot i+1 is applied after
 * sub-step i (c(z) = z + xi, or the velocity reset). Y[n+1] = X_{k+1}. */
static void integrate_step(const orc_problem *P, const orc_draws *D, const double *xk,
                           const double *uk, double (*Y)[ORC_DMAX]) {
  const int d = P->d;
  double f[ORC_DMAX];
  memcpy(Y[0], xk, sizeof(double) * d);
  for (int i = 0; i <= D->n; ++i) {
    drift(P, Y[i], uk, f);
    double sq = sqrt(D->delta[i]);
    for (int c = 0; c < d; ++c) {
      Y[i + 1][c] = Y[i][c] + D->delta[i] * f[c] + P->sigma[c] * sq * D->Z[i][c];
      if (i < D->n && jump_acts_on(P, c))
        Y[i + 1][c] = jump_gain_of(P, c) * Y[i + 1][c] + P->jump_scale * D->xi_hat[i][c];
    }
  }
}

static double running_cost(const orc_problem *P, const double *x, int k) {
  double s = 0.0;
  for (int i = 0; i < P->d; ++i) {
    double e = x[i] - P->xd[k * P->d + i];
    s += P->q[i] * e * e;
  }
  return 0.5 * s;
}

static int valid(const orc_problem *P) {
  if (!P || P->d < 1 || P->d > ORC_DMAX || P->du < 1 || P->du > ORC_DUMAX || P->Nt < 1 ||
      P->M < 1 || !(P->T > 0.0))
    return 0;
  if (!P->A || !P->B || !P->sigma || !P->x0 || !P->q || !P->xd) return 0;
  if (P->drift == ORC_CUBIC && !P->C) return 0;
  if (P->jump_law < 0 || P->jump_law > 3) return 0;
  return 1;
}

int orc_path(const orc_problem *P, const double *u, int64_t m, double *X, double *lam, double *G,
             double *cost, double *gtheta, int *njumps) {
  if (!valid(P) || !u || m < 0 || m >= P->M) return 1;
  const int d = P->d, du = P->du, Nt = P->Nt;
  const double dt = P->T / (double)Nt;
  double *Xs = X ? X : (double *)malloc(sizeof(double) * (size_t)(Nt + 1) * d);
  orc_draws *D = (orc_draws *)malloc(sizeof(orc_draws));
  double (*Y)[ORC_DMAX] = (double (*)[ORC_DMAX])malloc(sizeof(double) * ORC_DMAX * (ORC_NMAX + 2));
  if (!Xs || !D || !Y) return 2;

  /* forward sweep */
  memcpy(Xs, P->x0, sizeof(double) * d);
  double c_m = 0.0;
  for (int k = 0; k < Nt; ++k) {
    orc_step_draws(P, k, m, D);
    if (njumps) njumps[k] = D->n;
    integrate_step(P, D, Xs + (size_t)k * d, u + (size_t)k * du, Y);
    memcpy(Xs + (size_t)(k + 1) * d, Y[D->n + 1], sizeof(double) * d);
    c_m += dt * running_cost(P, Xs + (size_t)(k + 1) * d, k + 1);
  }
  if (cost) *cost = c_m;

  /* adjoint sweep: mu is the derivative of the path cost with respect to the
   * current state, carried backwards through every sub-step */
  if (G || lam || gtheta) {
    double mu[ORC_DMAX], jt[ORC_DMAX];
    if (gtheta) memset(gtheta, 0, sizeof(double) * (d + 2));
    for (int i = 0; i < d; ++i)
      mu[i] = dt * P->q[i] * (Xs[(size_t)Nt * d + i] - P->xd[(size_t)Nt * d + i]);
    if (lam) memcpy(lam + (size_t)Nt * d, mu, sizeof(double) * d);
    for (int k = Nt - 1; k >= 0; --k) {
      orc_step_draws(P, k, m, D);
      integrate_step(P, D, Xs + (size_t)k * d, u + (size_t)k * du, Y);
      double g[ORC_DUMAX];
      memset(g, 0, sizeof(g));
      for (int i = D->n; i >= 0; --i) {
        /* mu = derivative w.r.t. Y[i+1], the state after the jump that follows sub-step
         * i; the jump's Jacobian (identity for additive jumps, gamma on the velocities
         * for the reset) turns it into the derivative w.r.t. the pre-jump state */
        if (i < D->n) {
          if (gtheta)
            for (int c = 0; c < d; ++c)
              if (jump_acts_on(P, c)) gtheta[d + 1] += mu[c] * D->xi_hat[i][c];
          for (int c = 0; c < d; ++c) mu[c] *= jump_gain_of(P, c);
        }
        for (int l = 0; l < du; ++l) {
          double s = 0.0;
          for (int c = 0; c < d; ++c) s += P->B[c * du + l] * mu[c];
          g[l] += D->delta[i] * s;
        }
        if (gtheta) {
          double sq = sqrt(D->delta[i]);
          for (int c = 0; c < d; ++c) gtheta[1 + c] += mu[c] * sq * D->Z[i][c];
          if (P->dA) {
            double s = 0.0;
            for (int r = 0; r < d; ++r)
              for (int c = 0; c < d; ++c) s += mu[r] * P->dA[r * d + c] * Y[i][c];
            gtheta[0] += D->delta[i] * s;
          }
        }
        drift_jacobian_T(P, Y[i], mu, jt);
        for (int c = 0; c < d; ++c) mu[c] = mu[c] + D->delta[i] * jt[c];
      }
      if (G) memcpy(G + (size_t)k * du, g, sizeof(double) * du);
      if (k >= 1)
        for (int c = 0; c < d; ++c)
          mu[c] += dt * P->q[c] * (Xs[(size_t)k * d + c] - P->xd[(size_t)k * d + c]);
      if (lam) memcpy(lam + (size_t)k * d, mu, sizeof(double) * d);
    }
  }
  if (!X) free(Xs);
  free(D);
  free(Y);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Sums over paths: fixed chunks of ORC_CHUNK paths, summed in path order;      */
/* chunk sums are then added in chunk order.  Threads only pick chunks.        */
/* ------------------------------------------------------------------------- */
#define ORC_CHUNK 256

typedef struct {
  const orc_problem *P;
  const double *u;
  int want_grad, want_theta;
  int64_t nchunks;
  double *chunk_cost;   /* nchunks */
  double *chunk_grad;   /* nchunks * Nt * du */
  double *chunk_theta;  /* nchunks * (d+2) */
  int64_t next;
  pthread_mutex_t lock;
  int err;
} sweep_job;

static void *sweep_worker(void *arg) {
  sweep_job *J = (sweep_job *)arg;
  const orc_problem *P = J->P;
  const int Nt = P->Nt, du = P->du, d = P->d;
  double *G = (double *)malloc(sizeof(double) * (size_t)Nt * du);
  double gth[ORC_DMAX + 2];
  for (;;) {
    pthread_mutex_lock(&J->lock);
    int64_t c = J->next++;
    pthread_mutex_unlock(&J->lock);
    if (c >= J->nchunks) break;
    double cs = 0.0;
    double *cg = J->want_grad ? J->chunk_grad + (size_t)c * Nt * du : NULL;
    double *ct = J->want_theta ? J->chunk_theta + (size_t)c * (d + 2) : NULL;
    if (cg) memset(cg, 0, sizeof(double) * (size_t)Nt * du);
    if (ct) memset(ct, 0, sizeof(double) * (d + 2));
    int64_t m_end = (c + 1) * ORC_CHUNK < P->M ? (c + 1) * ORC_CHUNK : P->M;
    for (int64_t m = c * ORC_CHUNK; m < m_end; ++m) {
      double cm = 0.0;
      int rc = orc_path(P, J->u, m, NULL, NULL, cg ? G : NULL, &cm, ct ? gth : NULL, NULL);
      if (rc) J->err = rc;
      cs += cm;
      if (cg)
        for (size_t t = 0; t < (size_t)Nt * du; ++t) cg[t] += G[t];
      if (ct)
        for (int t = 0; t < d + 2; ++t) ct[t] += gth[t];
    }
    J->chunk_cost[c] = cs;
  }
  free(G);
  return NULL;
}

static int sweep(const orc_problem *P, const double *u, int nthreads, int want_grad, int want_theta,
                 double *J, double *grad, double *gtheta) {
  if (!valid(P) || !u) return 1;
  const int Nt = P->Nt, du = P->du, d = P->d;
  const double dt = P->T / (double)Nt;
  sweep_job job;
  memset(&job, 0, sizeof(job));
  job.P = P;
  job.u = u;
  job.want_grad = want_grad;
  job.want_theta = want_theta;
  job.nchunks = (P->M + ORC_CHUNK - 1) / ORC_CHUNK;
  job.chunk_cost = (double *)calloc((size_t)job.nchunks, sizeof(double));
  if (want_grad) job.chunk_grad = (double *)calloc((size_t)job.nchunks * Nt * du, sizeof(double));
  if (want_theta) job.chunk_theta = (double *)calloc((size_t)job.nchunks * (d + 2), sizeof(double));
  pthread_mutex_init(&job.lock, NULL);
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, sweep_worker, &job);
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  pthread_mutex_destroy(&job.lock);

  /* J = (1/M) sum_m c_m + (nu/2) dt sum_k |u_k|^2 */
  double csum = 0.0;
  for (int64_t c = 0; c < job.nchunks; ++c) csum += job.chunk_cost[c];
  double usq = 0.0;
  for (size_t t = 0; t < (size_t)Nt * du; ++t) usq += u[t] * u[t];
  if (J) *J = csum / (double)P->M + 0.5 * P->nu * dt * usq;

  /* dJ/du_k = nu dt u_k + (1/M) sum_m G_k^m */
  if (want_grad && grad) {
    for (size_t t = 0; t < (size_t)Nt * du; ++t) {
      double s = 0.0;
      for (int64_t c = 0; c < job.nchunks; ++c) s += job.chunk_grad[(size_t)c * Nt * du + t];
      grad[t] = P->nu * dt * u[t] + s / (double)P->M;
    }
  }
  if (want_theta && gtheta) {
    for (int t = 0; t < d + 2; ++t) {
      double s = 0.0;
      for (int64_t c = 0; c < job.nchunks; ++c) s += job.chunk_theta[(size_t)c * (d + 2) + t];
      gtheta[t] = s / (double)P->M;
    }
  }
  int err = job.err;
  free(job.chunk_cost);
  free(job.chunk_grad);
  free(job.chunk_theta);
  return err;
}

int orc_cost(const orc_problem *P, const double *u, int nthreads, double *J) {
  return sweep(P, u, nthreads, 0, 0, J, NULL, NULL);
}

int orc_gradient(const orc_problem *P, const double *u, int nthreads, double *J, double *grad,
                 double *gtheta) {
  return sweep(P, u, nthreads, 1, gtheta != NULL, J, grad, gtheta);
}

/* ------------------------------------------------------------------------- */
/* Projected gradient descent with the Armijo rule (Algorithm 5.4).            */
/* g = (dJ/du)/dt is the L2 representative of the gradient; the trial point is  */
/* u+ = clip(u - zeta g); accept when J(u+) <= J(u) + c <g, u+ - u>_{L2}, which  */
/* without active bounds is J(u) - c zeta |g|^2_{L2} (eq:Stochastic_Armijo).     */
/* ------------------------------------------------------------------------- */
static double clip(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

int orc_optimize(const orc_problem *P, double *u, const orc_opt_params *o, int nthreads,
                 orc_opt_result *r, double *J_hist) {
  if (!valid(P) || !u || !o || !r) return 1;
  const size_t n = (size_t)P->Nt * P->du;
  const double dt = P->T / (double)P->Nt;
  double *grad = (double *)malloc(sizeof(double) * n);
  double *g = (double *)malloc(sizeof(double) * n);
  double *ut = (double *)malloc(sizeof(double) * n);
  memset(r, 0, sizeof(*r));
  double J = 0.0, pg0 = -1.0, zeta = o->zeta0 > 0 ? o->zeta0 : 1.0;
  double zeta_max = o->zeta_max > 0 ? o->zeta_max : 1e3;
  int status = 0, it = 0;
  /* Algorithm 5.4: while not converged and n < n_max: gradient at u^n, Armijo step
   * size, update, step-norm test.  The projected-gradient test (relative to the first
   * iterate) is checked when the gradient is available, at the top of the loop. */
  orc_problem Pn = *P;   /* the sample of iteration it: epoch P->epoch + it when resampling */
  for (it = 0; it < o->max_iter; ++it) {
    if (o->resample) Pn.epoch = P->epoch + (uint32_t)it;
    int rc = orc_gradient(&Pn, u, nthreads, &J, grad, NULL);
    r->evals++;
    if (rc) { status = 1; break; }
    if (J_hist) J_hist[it] = J;
    /* projected-gradient norm |P(u - g) - u|_{L2} */
    double pg = 0.0;
    for (size_t t = 0; t < n; ++t) {
      g[t] = grad[t] / dt;
      double e = clip(u[t] - g[t], P->u_min, P->u_max) - u[t];
      pg += dt * e * e;
    }
    pg = sqrt(pg);
    if (pg0 < 0.0) pg0 = pg;
    r->rel_grad_norm = pg0 > 0.0 ? pg / pg0 : 0.0;
    if (r->rel_grad_norm <= o->tol_rel_grad) break;

    /* Armijo backtracking on the projected path */
    if (it > 0) zeta = fmin(2.0 * zeta, zeta_max);
    int accepted = 0;
    double Jt = 0.0, step2 = 0.0;
    for (int b = 0; b <= o->max_backtracks; ++b) {
      double dot = 0.0;
      for (size_t t = 0; t < n; ++t) {
        ut[t] = clip(u[t] - zeta * g[t], P->u_min, P->u_max);
        dot += dt * g[t] * (ut[t] - u[t]);
      }
      rc = orc_cost(&Pn, ut, nthreads, &Jt);
      r->evals++;
      if (rc) { status = 1; break; }
      if (Jt <= J + o->armijo_c * dot) { accepted = 1; break; }
      zeta *= 0.5;
    }
    if (status) break;
    if (!accepted) { status = 5; break; }
    step2 = 0.0;
    for (size_t t = 0; t < n; ++t) {
      step2 += dt * (ut[t] - u[t]) * (ut[t] - u[t]);
      u[t] = ut[t];
    }
    J = Jt;
    if (J_hist) J_hist[it + 1] = J;
    if (sqrt(step2) < o->tol_step) {
      it++;
      break;
    }
  }
  r->iters = it;
  r->J = J;
  r->zeta = zeta;
  r->status = status;
  free(grad);
  free(g);
  free(ut);
  return status;
}

/* ------------------------------------------------------------------------- */
/* Feedback control u(z, t) = mu(t)^T phi(z) (Sec. 2 eq:control_structure) on  */
/* the phase space z = (x, v) of Sec. 5: L = nx nv products of bump functions  */
/* (Sec. 5.2 eq:Gaussian_RBF) centred on the cell centres of Sec. 5.1.         */
/* ------------------------------------------------------------------------- */

/* phi(x, x_c, eps) with r = x - x_c: exp(-1 / (1 - (eps r)^2)) for |r| < 1/eps, else 0 */
double orc_bump(double r, double eps) {
  double s = (eps * r) * (eps * r);
  if (!(s < 1.0)) return 0.0;
  return exp(-1.0 / (1.0 - s));
}

/* d phi / d x = phi * (-2 eps^2 r) / (1 - (eps r)^2)^2 (zero outside the support) */
double orc_bump_dr(double r, double eps) {
  double s = (eps * r) * (eps * r);
  if (!(s < 1.0)) return 0.0;
  double e = 1.0 / (1.0 - s);
  return exp(-e) * (-2.0 * eps * eps * r) * e * e;
}

/* cell centres x^i = (i - 1/2) dx - x_max, i = 1..n (0-based here: i + 1/2) */
static double centre(int i, int n, double half_width) {
  return ((double)i + 0.5) * (2.0 * half_width / (double)n) - half_width;
}

/* u = sum_{i,l} mu[i nv + l] phi(x - x^i) phi(v - v^l) at z = (x, v); du (nullable)
 * receives (u_x, u_v), phi (nullable, L) the shape-function values. */
double orc_fb_control(const orc_feedback *F, const double *mu_k, const double *z, double *du,
                      double *phi) {
  double px[ORC_FBMAX], dpx[ORC_FBMAX], pv[ORC_FBMAX], dpv[ORC_FBMAX];
  for (int i = 0; i < F->nx; ++i) {
    double r = z[0] - centre(i, F->nx, F->x_max);
    px[i] = orc_bump(r, F->eps);
    dpx[i] = orc_bump_dr(r, F->eps);
  }
  for (int l = 0; l < F->nv; ++l) {
    double r = z[1] - centre(l, F->nv, F->v_max);
    pv[l] = orc_bump(r, F->eps);
    dpv[l] = orc_bump_dr(r, F->eps);
  }
  double u = 0.0, ux = 0.0, uv = 0.0;
  for (int i = 0; i < F->nx; ++i)
    for (int l = 0; l < F->nv; ++l) {
      double m = mu_k[i * F->nv + l];
      u += m * px[i] * pv[l];
      ux += m * dpx[i] * pv[l];
      uv += m * px[i] * dpv[l];
      if (phi) phi[i * F->nv + l] = px[i] * pv[l];
    }
  if (du) {
    du[0] = ux;
    du[1] = uv;
  }
  return u;
}

/* Tracking term l(z, t_k) and its gradient (nullable): quadratic 1/2 sum q_c e_c^2, or
 * the Gaussian of Sec. 6 eq:tracking_cost, -exp(-sum q_c e_c^2 / (2 sigma_J^2)),
 * e = z - z_d(t_k). */
static double fb_track(const orc_problem *P, const orc_feedback *F, const double *z, int k,
                       double *grad) {
  double Q = 0.0, e[ORC_DMAX];
  for (int c = 0; c < P->d; ++c) {
    e[c] = z[c] - P->xd[k * P->d + c];
    Q += P->q[c] * e[c] * e[c];
  }
  if (F->track == ORC_TRACK_GAUSS) {
    double s2 = F->sigma_J * F->sigma_J, E = exp(-Q / (2.0 * s2));
    if (grad)
      for (int c = 0; c < P->d; ++c) grad[c] = E * P->q[c] * e[c] / s2;
    return -E;
  }
  if (F->track == ORC_TRACK_ELLIPSE) {
    /* -exp(-(x^2/ax^2 + v^2/av^2 - 1)^2 / (2 sigma_J^2)) (Sec. 6.4 Eq. phonon_functional_tracking) */
    double s2 = F->sigma_J * F->sigma_J;
    double Ee = z[0] * z[0] / (F->ax * F->ax) + z[1] * z[1] / (F->av * F->av) - 1.0;
    double E = exp(-Ee * Ee / (2.0 * s2));
    if (grad) {
      grad[0] = E * (Ee / s2) * (2.0 * z[0] / (F->ax * F->ax));
      grad[1] = E * (Ee / s2) * (2.0 * z[1] / (F->av * F->av));
    }
    return -E;
  }
  if (grad)
    for (int c = 0; c < P->d; ++c) grad[c] = P->q[c] * e[c];
  return 0.5 * Q;
}

static int fb_valid(const orc_problem *P, const orc_feedback *F) {
  return valid(P) && F && P->d == 2 && P->du == 1 && F->nx >= 1 && F->nx <= ORC_FBMAX &&
         F->nv >= 1 && F->nv <= ORC_FBMAX && F->x_max > 0.0 && F->v_max > 0.0 && F->eps > 0.0 &&
         (F->track == ORC_TRACK_QUAD || ((F->track == ORC_TRACK_GAUSS || F->track == ORC_TRACK_ELLIPSE) &&
                                          F->sigma_J > 0.0)) &&
         (F->track != ORC_TRACK_ELLIPSE || (F->ax > 0.0 && F->av > 0.0)) &&
         (F->adjoint == ORC_FB_EXACT || (F->adjoint == ORC_FB_SURROGATE && F->sur_rate >= 0.0));
}

/* Surrogate state of step k (Sec. 6.5): z_d(t_k) plus a normal pair scaled by the
 * standard deviation sqrt(rate t_k) of a variance that grows linearly in time. */
void orc_fb_surrogate_state(const orc_problem *P, const orc_feedback *F, int k, int64_t m, double zs[2]) {
  uint32_t w[2];
  double xi[2];
  stream_words(P, k, m, 2u, 0u, 2, w);
  normal_pair(w[0], w[1], &xi[0], &xi[1]);
  const double sd = sqrt(F->sur_rate * (P->T / (double)P->Nt) * (double)k);
  for (int c = 0; c < 2; ++c) zs[c] = P->xd[k * 2 + c] + sd * xi[c];
}

/* Sub-steps of step k under feedback (Algorithm 5.1, the control evaluated at the
 * left end of every sub-step); returns sum_i (alpha/2) delta_i u(Y_i)^2. */
static double integrate_step_fb(const orc_problem *P, const orc_feedback *F, const orc_draws *D,
                                const double *xk, const double *mu_k, double cin, double (*Y)[ORC_DMAX]) {
  double f[ORC_DMAX], ucost = 0.0;
  memcpy(Y[0], xk, sizeof(double) * 2);
  for (int i = 0; i <= D->n; ++i) {
    double u = orc_fb_control(F, mu_k, Y[i], NULL, NULL);
    ucost += 0.5 * P->nu * D->delta[i] * u * u;
    drift(P, Y[i], &u, f);
    f[1] += cin;   /* coupled particles: the neighbours' force, fixed over the step */
    double sq = sqrt(D->delta[i]);
    for (int c = 0; c < 2; ++c) {
      Y[i + 1][c] = Y[i][c] + D->delta[i] * f[c] + P->sigma[c] * sq * D->Z[i][c];
      if (i < D->n && jump_acts_on(P, c))
        Y[i + 1][c] = jump_gain_of(P, c) * Y[i + 1][c] + P->jump_scale * D->xi_hat[i][c];
    }
  }
  return ucost;
}

int orc_fb_path(const orc_problem *P, const orc_feedback *F, const double *mu, int64_t m,
                double *X, double *lam, double *G, double *cost, int *njumps) {
  if (!fb_valid(P, F) || !mu || m < 0 || m >= P->M) return 1;
  const int Nt = P->Nt, L = F->nx * F->nv;
  const double dt = P->T / (double)Nt;
  double *Xs = X ? X : (double *)malloc(sizeof(double) * (size_t)(Nt + 1) * 2);
  orc_draws *D = (orc_draws *)malloc(sizeof(orc_draws));
  double (*Y)[ORC_DMAX] = (double (*)[ORC_DMAX])malloc(sizeof(double) * ORC_DMAX * (ORC_NMAX + 2));
  double *phi = (double *)malloc(sizeof(double) * L);
  if (!Xs || !D || !Y || !phi) return 2;

  if (F->adjoint == ORC_FB_SURROGATE && (G || lam)) {
    /* Sec. 6.5: the costates run backwards along the surrogate states zs_k, never the
     * forward's; per step one Euler step of the adjoint at zs_k, the jumps of the path's
     * own step k entering through the Jacobian of the jump map (gamma^n on the reset
     * velocities).  bhat_k = B^T r after the jumps of step k then drives the gradient of
     * the forward sweep: dcost/dmu_k += delta_i phi(Y_i) (alpha u(Y_i) + bhat_k). */
    double *bhat = (double *)malloc(sizeof(double) * Nt);
    double r[2], zs[2], jt[ORC_DMAX], gr[ORC_DMAX], du[2];
    orc_fb_surrogate_state(P, F, Nt, m, zs);
    fb_track(P, F, zs, Nt, gr);
    for (int c = 0; c < 2; ++c) r[c] = dt * gr[c];
    if (lam) memcpy(lam + (size_t)Nt * 2, r, sizeof(r));
    for (int k = Nt - 1; k >= 0; --k) {
      orc_step_draws(P, k, m, D);
      for (int i = 0; i < D->n; ++i)
        for (int c = 0; c < 2; ++c) r[c] *= jump_gain_of(P, c);
      bhat[k] = P->B[0] * r[0] + P->B[1] * r[1];
      orc_fb_surrogate_state(P, F, k, m, zs);
      double u = orc_fb_control(F, mu + (size_t)k * L, zs, du, NULL);
      double w = P->nu * u + bhat[k];
      drift_jacobian_T(P, zs, r, jt);
      for (int c = 0; c < 2; ++c) r[c] = r[c] + dt * (jt[c] + w * du[c]);
      if (k >= 1) {
        fb_track(P, F, zs, k, gr);
        for (int c = 0; c < 2; ++c) r[c] += dt * gr[c];
      }
      if (lam) memcpy(lam + (size_t)k * 2, r, sizeof(r));
    }
    memcpy(Xs, P->x0, sizeof(double) * 2);
    double c_m = 0.0;
    for (int k = 0; k < Nt; ++k) {
      orc_step_draws(P, k, m, D);
      if (njumps) njumps[k] = D->n;
      c_m += integrate_step_fb(P, F, D, Xs + (size_t)k * 2, mu + (size_t)k * L, 0.0, Y);
      if (G) {
        memset(G + (size_t)k * L, 0, sizeof(double) * L);
        for (int i = 0; i <= D->n; ++i) {
          double u = orc_fb_control(F, mu + (size_t)k * L, Y[i], NULL, phi);
          double w = P->nu * u + bhat[k];
          for (int l = 0; l < L; ++l) G[(size_t)k * L + l] += D->delta[i] * phi[l] * w;
        }
      }
      memcpy(Xs + (size_t)(k + 1) * 2, Y[D->n + 1], sizeof(double) * 2);
      c_m += dt * fb_track(P, F, Xs + (size_t)(k + 1) * 2, k + 1, NULL);
    }
    if (cost) *cost = c_m;
    free(bhat);
    if (!X) free(Xs);
    free(D);
    free(Y);
    free(phi);
    return 0;
  }

  /* forward sweep; the cost is sum_k [dt l(X_{k+1}) + sum_i (alpha/2) delta_i u(Y_i)^2] */
  memcpy(Xs, P->x0, sizeof(double) * 2);
  double c_m = 0.0;
  for (int k = 0; k < Nt; ++k) {
    orc_step_draws(P, k, m, D);
    if (njumps) njumps[k] = D->n;
    c_m += integrate_step_fb(P, F, D, Xs + (size_t)k * 2, mu + (size_t)k * L, 0.0, Y);
    memcpy(Xs + (size_t)(k + 1) * 2, Y[D->n + 1], sizeof(double) * 2);
    c_m += dt * fb_track(P, F, Xs + (size_t)(k + 1) * 2, k + 1, NULL);
  }
  if (cost) *cost = c_m;

  /* adjoint sweep: a = derivative of the path cost w.r.t. the current state.  Across
   * sub-step i (Y_i -> Y_{i+1}) with w = alpha u(Y_i) + B^T a:
   *   dcost/dmu_k,l += delta_i phi_l(Y_i) w,
   *   a <- a + delta_i [ (A + 3 C diag(Y_i^2))^T a + w grad u(Y_i) ]
   * (Sec. 5.5 eq:adjoint_eq_approximation with grad_z j^h = grad l + alpha u grad u). */
  if (G || lam) {
    double a[2], jt[ORC_DMAX], gr[ORC_DMAX], du[2];
    fb_track(P, F, Xs + (size_t)Nt * 2, Nt, gr);
    for (int c = 0; c < 2; ++c) a[c] = dt * gr[c];
    if (lam) memcpy(lam + (size_t)Nt * 2, a, sizeof(a));
    for (int k = Nt - 1; k >= 0; --k) {
      const double *mu_k = mu + (size_t)k * L;
      orc_step_draws(P, k, m, D);
      integrate_step_fb(P, F, D, Xs + (size_t)k * 2, mu_k, 0.0, Y);
      if (G) memset(G + (size_t)k * L, 0, sizeof(double) * L);
      for (int i = D->n; i >= 0; --i) {
        if (i < D->n)
          for (int c = 0; c < 2; ++c) a[c] *= jump_gain_of(P, c);
        double u = orc_fb_control(F, mu_k, Y[i], du, phi);
        double w = P->nu * u + P->B[0] * a[0] + P->B[1] * a[1];
        if (G)
          for (int l = 0; l < L; ++l) G[(size_t)k * L + l] += D->delta[i] * phi[l] * w;
        drift_jacobian_T(P, Y[i], a, jt);
        for (int c = 0; c < 2; ++c) a[c] = a[c] + D->delta[i] * (jt[c] + w * du[c]);
      }
      if (k >= 1) {
        fb_track(P, F, Xs + (size_t)k * 2, k, gr);
        for (int c = 0; c < 2; ++c) a[c] += dt * gr[c];
      }
      if (lam) memcpy(lam + (size_t)k * 2, a, sizeof(a));
    }
  }
  if (!X) free(Xs);
  free(D);
  free(Y);
  free(phi);
  return 0;
}

/* Sums over paths under feedback, in the same fixed chunk order as sweep():
 * J = (1/M) sum_m c_m (the control cost is inside c_m), dJ/dmu = (1/M) sum_m G_m. */
typedef struct {
  const orc_problem *P;
  const orc_feedback *F;
  const double *mu;
  int want_grad;
  int64_t nchunks;
  double *chunk_cost, *chunk_grad;
  int64_t next;
  pthread_mutex_t lock;
  int err;
} fb_job;

static void *fb_worker(void *arg) {
  fb_job *J = (fb_job *)arg;
  const orc_problem *P = J->P;
  const size_t n = (size_t)P->Nt * J->F->nx * J->F->nv;
  double *G = J->want_grad ? (double *)malloc(sizeof(double) * n) : NULL;
  for (;;) {
    pthread_mutex_lock(&J->lock);
    int64_t c = J->next++;
    pthread_mutex_unlock(&J->lock);
    if (c >= J->nchunks) break;
    double cs = 0.0;
    double *cg = J->want_grad ? J->chunk_grad + (size_t)c * n : NULL;
    if (cg) memset(cg, 0, sizeof(double) * n);
    int64_t m_end = (c + 1) * ORC_CHUNK < P->M ? (c + 1) * ORC_CHUNK : P->M;
    for (int64_t m = c * ORC_CHUNK; m < m_end; ++m) {
      double cm = 0.0;
      int rc = orc_fb_path(P, J->F, J->mu, m, NULL, NULL, G, &cm, NULL);
      if (rc) J->err = rc;
      cs += cm;
      if (cg)
        for (size_t t = 0; t < n; ++t) cg[t] += G[t];
    }
    J->chunk_cost[c] = cs;
  }
  free(G);
  return NULL;
}

static int fb_sweep(const orc_problem *P, const orc_feedback *F, const double *mu, int nthreads,
                    double *J, double *grad) {
  if (F && F->particles > 0) return orc_fb_coupled_gradient(P, F, mu, nthreads, J, grad);   /* Sec. 6.4 */
  if (!fb_valid(P, F) || !mu) return 1;
  const size_t n = (size_t)P->Nt * F->nx * F->nv;
  fb_job job;
  memset(&job, 0, sizeof(job));
  job.P = P;
  job.F = F;
  job.mu = mu;
  job.want_grad = grad != NULL;
  job.nchunks = (P->M + ORC_CHUNK - 1) / ORC_CHUNK;
  job.chunk_cost = (double *)calloc((size_t)job.nchunks, sizeof(double));
  if (grad) job.chunk_grad = (double *)calloc((size_t)job.nchunks * n, sizeof(double));
  pthread_mutex_init(&job.lock, NULL);
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, fb_worker, &job);
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  pthread_mutex_destroy(&job.lock);
  double csum = 0.0;
  for (int64_t c = 0; c < job.nchunks; ++c) csum += job.chunk_cost[c];
  if (J) *J = csum / (double)P->M;
  if (grad)
    for (size_t t = 0; t < n; ++t) {
      double s = 0.0;
      for (int64_t c = 0; c < job.nchunks; ++c) s += job.chunk_grad[(size_t)c * n + t];
      grad[t] = s / (double)P->M;
    }
  int err = job.err;
  free(job.chunk_cost);
  free(job.chunk_grad);
  return err;
}

int orc_fb_cost(const orc_problem *P, const orc_feedback *F, const double *mu, int nthreads,
                double *J) {
  return fb_sweep(P, F, mu, nthreads, J, NULL);
}

int orc_fb_gradient(const orc_problem *P, const orc_feedback *F, const double *mu, int nthreads,
                    double *J, double *grad) {
  return fb_sweep(P, F, mu, nthreads, J, grad);
}

/* Gradient descent with the Armijo rule on the feedback weights (Algorithm 5.4 with
 * eq:Stochastic_Armijo; mu is unconstrained).  g = (dJ/dmu)/dt is the L2 representative;
 * the trial point is mu+ = mu - zeta g, accepted when J(mu+) <= J(mu) - c zeta |g|_{L2}^2.
 * Same schedule of zeta and the same stopping tests as orc_optimize. */
int orc_fb_optimize(const orc_problem *P, const orc_feedback *F, double *mu, const orc_opt_params *o,
                    int nthreads, orc_opt_result *r, double *J_hist) {
  if (!fb_valid(P, F) || !mu || !o || !r) return 1;
  const size_t n = (size_t)P->Nt * F->nx * F->nv;
  const double dt = P->T / (double)P->Nt;
  double *grad = (double *)malloc(sizeof(double) * n);
  double *mt = (double *)malloc(sizeof(double) * n);
  memset(r, 0, sizeof(*r));
  double J = 0.0, pg0 = -1.0, zeta = o->zeta0 > 0 ? o->zeta0 : 1.0;
  double zeta_max = o->zeta_max > 0 ? o->zeta_max : 1e3;
  int status = 0, it = 0;
  orc_problem Pn = *P;   /* the sample of iteration it: epoch P->epoch + it when resampling */
  for (it = 0; it < o->max_iter; ++it) {
    if (o->resample) Pn.epoch = P->epoch + (uint32_t)it;
    int rc = orc_fb_gradient(&Pn, F, mu, nthreads, &J, grad);
    r->evals++;
    if (rc) { status = 1; break; }
    if (J_hist) J_hist[it] = J;
    double g2 = 0.0;   /* |g|_{L2}^2 = dt sum (grad/dt)^2 */
    for (size_t t = 0; t < n; ++t) g2 += dt * (grad[t] / dt) * (grad[t] / dt);
    double pg = sqrt(g2);
    if (pg0 < 0.0) pg0 = pg;
    r->rel_grad_norm = pg0 > 0.0 ? pg / pg0 : 0.0;
    if (r->rel_grad_norm <= o->tol_rel_grad) break;
    if (it > 0) zeta = fmin(2.0 * zeta, zeta_max);
    int accepted = 0;
    double Jt = 0.0;
    for (int b = 0; b <= o->max_backtracks; ++b) {
      for (size_t t = 0; t < n; ++t) mt[t] = mu[t] - zeta * (grad[t] / dt);
      rc = orc_fb_cost(&Pn, F, mt, nthreads, &Jt);
      r->evals++;
      if (rc) { status = 1; break; }
      if (Jt <= J - o->armijo_c * zeta * g2) { accepted = 1; break; }
      zeta *= 0.5;
    }
    if (status) break;
    if (!accepted) { status = 5; break; }
    double step2 = 0.0;
    for (size_t t = 0; t < n; ++t) {
      step2 += dt * (mt[t] - mu[t]) * (mt[t] - mu[t]);
      mu[t] = mt[t];
    }
    J = Jt;
    if (J_hist) J_hist[it + 1] = J;
    if (sqrt(step2) < o->tol_step) {
      it++;
      break;
    }
  }
  r->iters = it;
  r->J = J;
  r->zeta = zeta;
  r->status = status;
  free(grad);
  free(mt);
  return status;
}

/* ------------------------------------------------------------------------- */
/* Interacting particles (Sec. 6.4)                                           */
/* ------------------------------------------------------------------------- */
/* Path indices of a ring: particle i of realization r has path index S r + i, S the
 * ring's lane count: 32 for N <= 32, the next power of two for N <= 256, then the next
 * multiple of 256 (S >= N; indices S r + N .. S r + S - 1 are not used). */
int orc_ring_lanes(int N) {
  if (N <= 32) return 32;
  if (N <= 256) {
    int s = 64;
    while (s < N) s *= 2;
    return s;
  }
  return 256 * ((N + 255) / 256);
}

static int coupled_valid(const orc_problem *P, const orc_feedback *F) {
  return fb_valid(P, F) && F->particles >= 3 && F->particles <= ORC_RING_MAX && F->ax > 0.0 && F->av > 0.0 &&
         F->adjoint == ORC_FB_EXACT;
}

int orc_fb_coupled(const orc_problem *P0, const orc_feedback *F, const double *mu, int64_t r, double *X,
                   double *lam, double *G, double *cost) {
  const int N = F->particles, S = orc_ring_lanes(N), Nt = P0->Nt, L = F->nx * F->nv;
  if (!coupled_valid(P0, F) || !mu || r < 0 || (int64_t)S * r >= P0->M) return 1;
  const double dt = P0->T / (double)Nt, om = F->omega;
  /* the particle's own share of the coupling, -2 omega x_i, joins its drift matrix */
  orc_problem P = *P0;
  double A2[4] = {P0->A[0], P0->A[1], P0->A[2] - 2.0 * om, P0->A[3]};
  P.A = A2;
  double *Xs = X ? X : (double *)malloc(sizeof(double) * (size_t)(Nt + 1) * N * 2);
  orc_draws *D = (orc_draws *)malloc(sizeof(orc_draws));
  double (*Y)[ORC_DMAX] = (double (*)[ORC_DMAX])malloc(sizeof(double) * ORC_DMAX * (ORC_NMAX + 2));
  double *phi = (double *)malloc(sizeof(double) * L);
  double *cin = (double *)malloc(sizeof(double) * N), *s = (double *)malloc(sizeof(double) * N);
  if (!Xs || !D || !Y || !phi || !cin || !s) return 2;
  for (int i = 0; i < N; ++i) {
    Xs[2 * i] = F->ax * cos(2.0 * M_PI * i / N);
    Xs[2 * i + 1] = F->av * sin(2.0 * M_PI * i / N);
  }
  double c_r = 0.0;
  for (int k = 0; k < Nt; ++k) {
    const double *Xk = Xs + (size_t)k * N * 2;
    for (int i = 0; i < N; ++i) cin[i] = om * (Xk[2 * ((i + N - 1) % N)] + Xk[2 * ((i + 1) % N)]);
    for (int i = 0; i < N; ++i) {
      orc_step_draws(&P, k, S * r + i, D);
      c_r += integrate_step_fb(&P, F, D, Xk + 2 * i, mu + (size_t)k * L, cin[i], Y);
      memcpy(Xs + ((size_t)(k + 1) * N + i) * 2, Y[D->n + 1], sizeof(double) * 2);
      c_r += dt * fb_track(&P, F, Xs + ((size_t)(k + 1) * N + i) * 2, k + 1, NULL);
    }
  }
  if (cost) *cost = c_r;
  if (G || lam) {
    /* per particle the adjoint of its sub-steps and s_i = sum_j delta_j a_v (the derivative
     * in its neighbour force, fixed over the step); then d/dx_j at t_k gains
     * omega (s_{j-1} + s_{j+1}) */
    double *a = (double *)malloc(sizeof(double) * N * 2);
    double jt[ORC_DMAX], gr[ORC_DMAX], du[2];
    for (int i = 0; i < N; ++i) {
      fb_track(&P, F, Xs + ((size_t)Nt * N + i) * 2, Nt, gr);
      a[2 * i] = dt * gr[0];
      a[2 * i + 1] = dt * gr[1];
    }
    if (lam) memcpy(lam + (size_t)Nt * N * 2, a, sizeof(double) * N * 2);
    for (int k = Nt - 1; k >= 0; --k) {
      const double *Xk = Xs + (size_t)k * N * 2, *mu_k = mu + (size_t)k * L;
      if (G) memset(G + (size_t)k * L, 0, sizeof(double) * L);
      for (int i = 0; i < N; ++i) cin[i] = om * (Xk[2 * ((i + N - 1) % N)] + Xk[2 * ((i + 1) % N)]);
      for (int i = 0; i < N; ++i) {
        double *ai = a + 2 * i;
        orc_step_draws(&P, k, S * r + i, D);
        integrate_step_fb(&P, F, D, Xk + 2 * i, mu_k, cin[i], Y);
        s[i] = 0.0;
        for (int j = D->n; j >= 0; --j) {
          if (j < D->n)
            for (int c = 0; c < 2; ++c) ai[c] *= jump_gain_of(&P, c);
          double u = orc_fb_control(F, mu_k, Y[j], du, phi);
          double w = P.nu * u + P.B[0] * ai[0] + P.B[1] * ai[1];
          if (G)
            for (int l = 0; l < L; ++l) G[(size_t)k * L + l] += D->delta[j] * phi[l] * w;
          s[i] += D->delta[j] * ai[1];
          drift_jacobian_T(&P, Y[j], ai, jt);
          for (int c = 0; c < 2; ++c) ai[c] = ai[c] + D->delta[j] * (jt[c] + w * du[c]);
        }
      }
      for (int i = 0; i < N; ++i) a[2 * i] += om * (s[(i + N - 1) % N] + s[(i + 1) % N]);
      if (k >= 1)
        for (int i = 0; i < N; ++i) {
          fb_track(&P, F, Xk + 2 * i, k, gr);
          a[2 * i] += dt * gr[0];
          a[2 * i + 1] += dt * gr[1];
        }
      if (lam) memcpy(lam + (size_t)k * N * 2, a, sizeof(double) * N * 2);
    }
    free(a);
  }
  if (!X) free(Xs);
  free(D);
  free(Y);
  free(phi);
  free(cin);
  free(s);
  return 0;
}

int orc_fb_coupled_gradient(const orc_problem *P, const orc_feedback *F, const double *mu, int nthreads,
                            double *J, double *grad) {
  (void)nthreads;
  const int S = coupled_valid(P, F) ? orc_ring_lanes(F->particles) : 32;
  if (!coupled_valid(P, F) || !mu || P->M % S != 0) return 1;
  const int64_t R = P->M / S;
  const size_t n = (size_t)P->Nt * F->nx * F->nv;
  double *G = grad ? (double *)malloc(sizeof(double) * n) : NULL;
  if (grad) memset(grad, 0, sizeof(double) * n);
  double csum = 0.0;
  int err = 0;
  for (int64_t r = 0; r < R; ++r) {
    double c = 0.0;
    int rc = orc_fb_coupled(P, F, mu, r, NULL, NULL, G, &c);
    if (rc) err = rc;
    csum += c;
    if (grad)
      for (size_t t = 0; t < n; ++t) grad[t] += G[t];
  }
  const double inv = 1.0 / ((double)R * F->particles);
  if (J) *J = csum * inv;
  if (grad)
    for (size_t t = 0; t < n; ++t) grad[t] *= inv;
  free(G);
  return err;
}
