/*
 * jd_oracle.h -- plain FP64 CPU oracle for the discretize-then-optimize method of
 * "Adjoint-based optimal control of jump-diffusion processes" (arXiv 2505.04328).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code, header,
 * table or constant generator with the CUDA path; it implements the same
 * counter-based random streams independently, from the published Philox4x32-10
 * definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3", SC'11).
 *
 * What is computed (paper section / equation in brackets):
 *   - controlled SDE dX = f(X,u) dt + sigma dB + dY with additive compound-Poisson
 *     jumps [Sec. 1 eq:SDE_general; Sec. 2 eq:compact_forward], drift
 *     f(x,u) = A x + C (x*x*x) + B u [Sec. 5.4 eq:coefficients, H <-> A, h <-> C x^3];
 *   - jump-adapted Euler-Maruyama grid: per uniform step the jump times split the
 *     step into sub-steps [Sec. 3 eq:Deterministic_timestep and the grid union that
 *     follows it; Algorithm 5.1; Algorithm 5.2];
 *   - discrete cost  J(u) = (1/M) sum_m sum_{k=1..Nt} dt l(X_k^m, t_k)
 *                        + (nu/2) dt sum_{k=0..Nt-1} |u_k|^2,
 *     l(x,t) = 1/2 sum_i q_i (x_i - xd_i(t))^2   [Sec. 3 eq:discrete_functional];
 *   - the exact discrete adjoint and the reduced gradient [Sec. 4 eq:AdjointModel,
 *     eq:definition_Gradient; Sec. 5.5 eq:adjoint_eq_approximation];
 *   - projected gradient descent with the Armijo rule [Sec. 5.6 eq:Stochastic_Armijo,
 *     Algorithm 5.4];
 *   - the Keilson-Storer velocity reset as jump map [Sec. 5.3 eq:jump_law];
 *   - feedback control u = mu(t)^T phi(z) with bump shape functions, the Gaussian
 *     tracking cost, and the gradient in mu [Sec. 2 eq:control_structure, Sec. 5.1-5.2,
 *     Sec. 5.5, Sec. 6 eq:tracking_cost] (declarations at the end).
 */
#ifndef JD_ORACLE_H
#define JD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_DMAX 64      /* largest state dimension the oracle accepts */
#define ORC_DUMAX 16     /* largest control dimension */
#define ORC_NMAX 16      /* jumps per uniform step are capped at this count */

enum { ORC_LINEAR = 0, ORC_CUBIC = 1 };
enum { ORC_JUMP_NONE = 0, ORC_JUMP_NORMAL = 1, ORC_JUMP_UNIFORM = 2, ORC_JUMP_KS = 3 };

typedef struct {
  int d, du, Nt;
  int64_t M;
  double T;
  int drift;                 /* ORC_LINEAR or ORC_CUBIC */
  const double *A;           /* d*d row-major */
  const double *C;           /* d*d row-major, used when drift == ORC_CUBIC */
  const double *B;           /* d*du row-major */
  const double *dA;          /* d*d direction for the drift-coefficient gradient, or NULL */
  const double *sigma;       /* d, diagonal additive diffusion */
  double lambda;             /* jump intensity */
  int jump_law;              /* ORC_JUMP_* */
  double jump_scale;         /* std (NORMAL, KS) or half-width (UNIFORM) */
  const double *x0;          /* d */
  const double *q;           /* d, diagonal tracking weights */
  const double *xd;          /* (Nt+1)*d target samples xd(t_k) */
  double nu, u_min, u_max;
  uint64_t seed;
  uint32_t epoch;
  double jump_gain;          /* KS: velocity gain gamma of the reset v <- gamma v + s xi */
} orc_problem;

/* One Philox4x32-10 block: out = Philox(key, ctr). */
void orc_philox4x32_10(const uint32_t key[2], const uint32_t ctr[4], uint32_t out[4]);

/* Uniform in (0,1) from one word: ((w >> 9) + 1/2) * 2^-23. */
double orc_u01(uint32_t w);

/* Poisson-count thresholds T_n = floor(2^32 F(n; mu)), n = 0..ORC_NMAX-1 (values in [0, 2^32]). */
void orc_poisson_thresholds(double mu, uint64_t thr[ORC_NMAX]);

/* Poisson count of one word: n = #{n : T_n <= w}. */
int orc_poisson_count(uint32_t w, const uint64_t thr[ORC_NMAX]);

/* Box-Muller pair from two words: the first word sets the radius
 * sqrt(-2 ln U(wa)), the second the angle 2 pi U(wb); z = (r cos, r sin). */
void orc_normal_pair(uint32_t wa, uint32_t wb, double z[2]);

/* The random draws of one uniform step, in the order the integrator uses them. */
typedef struct {
  int n;                                   /* jumps in this step */
  double theta[ORC_NMAX];                  /* sorted jump-time fractions in (0,1) */
  double delta[ORC_NMAX + 1];              /* sub-step lengths */
  double Z[ORC_NMAX + 1][ORC_DMAX];        /* standard normals per sub-step */
  double xi_hat[ORC_NMAX][ORC_DMAX];       /* unit jump sizes, time order */
} orc_draws;

/* Draws of step k of path m (used by tests to check the jump law and to drive
 * independent re-derivations). */
int orc_step_draws(const orc_problem *P, int k, int64_t m, orc_draws *out);

/* One path: forward sweep, optional adjoint sweep.
 *   X      (Nt+1)*d states on the uniform grid, or NULL
 *   lam    (Nt+1)*d adjoint states lambda_k, or NULL (lambda_0 = derivative w.r.t. X_0)
 *   G      Nt*du per-path control sensitivities sum_i delta_i B^T lambda', or NULL
 *          (NULL also skips the adjoint sweep unless gtheta or lam is given)
 *   cost   per-path running cost sum_k dt l(X_k, t_k), or NULL
 *   gtheta d+2 per-path parameter sensitivities [dA-direction, sigma_0..sigma_{d-1},
 *          jump_scale], or NULL
 *   njumps Nt jump counts, or NULL
 * u is Nt*du.  Returns 0 on success, nonzero on invalid input. */
int orc_path(const orc_problem *P, const double *u, int64_t m, double *X, double *lam,
             double *G, double *cost, double *gtheta, int *njumps);

/* Reduced cost J(u), paths summed in fixed chunks so the result does not depend on
 * nthreads. */
int orc_cost(const orc_problem *P, const double *u, int nthreads, double *J);

/* J(u) and the Euclidean gradient dJ/du_k (Nt*du); gtheta (d+2, nullable) is the
 * gradient with respect to [drift direction dA, sigma_i, jump_scale]. */
int orc_gradient(const orc_problem *P, const double *u, int nthreads, double *J,
                 double *grad, double *gtheta);

typedef struct {
  int max_iter;
  double tol_rel_grad, tol_step, armijo_c, zeta0, zeta_max;
  int max_backtracks;
  int resample;   /* 1: iteration n draws a fresh sample, epoch = P->epoch + n (Sec. 5.6 SGD) */
} orc_opt_params;

typedef struct {
  int iters, evals, status;     /* status 0 ok, 5 = line search failed */
  double J, rel_grad_norm, zeta;
} orc_opt_result;

/* Projected gradient descent with the Armijo rule (Algorithm 5.4): at most max_iter
 * iterations, each one gradient evaluation at u^n, an Armijo line search and the
 * update; no gradient is evaluated after the last update.  u is updated in place.
 * J_hist (max_iter+1, nullable) receives J(u^n) of every iterate reached. */
int orc_optimize(const orc_problem *P, double *u, const orc_opt_params *o, int nthreads,
                 orc_opt_result *r, double *J_hist);

/* ------------------------------------------------------------------------- */
/* Feedback control (Sec. 2 eq:control_structure; Sec. 5.1-5.2; Sec. 6) for    */
/* d = 2, du = 1, z = (x, v): u(z, t_k) = sum_{i,l} mu[k][i nv + l]               */
/*   phi(x - x^i) phi(v - v^l), centres x^i = (i + 1/2) 2 x_max / nx - x_max (same   */
/* for v), phi the bump exp(-1/(1 - (eps r)^2)) on |r| < 1/eps.  The control acts  */
/* through B u(z) and is evaluated at the left end of every sub-step; the path    */
/* cost is sum_k dt l(X_{k+1}, t_{k+1}) + sum over sub-steps (nu/2) delta_i u(Y_i)^2 */
/* (nu is the paper's alpha), l quadratic or the Gaussian of eq:tracking_cost.    */
/* mu is Nt * L, L = nx nv, row-major [k][i][l].                                   */
/* ------------------------------------------------------------------------- */
#define ORC_FBMAX 16     /* centres per axis */
enum { ORC_TRACK_QUAD = 0, ORC_TRACK_GAUSS = 1, ORC_TRACK_ELLIPSE = 2 };
enum { ORC_FB_EXACT = 0, ORC_FB_SURROGATE = 1 };

typedef struct {
  int nx, nv;             /* centres per axis */
  double x_max, v_max;    /* computational domain (-x_max, x_max) x (-v_max, v_max) */
  double eps;             /* bump shape parameter eps_phi */
  int track;              /* ORC_TRACK_QUAD or ORC_TRACK_GAUSS */
  double sigma_J;         /* Gaussian tracking width */
  int adjoint;            /* ORC_FB_EXACT, or ORC_FB_SURROGATE (Sec. 6.5): the costates run
                             along states drawn from N(z_d(t_k), rate t_k I) */
  double sur_rate;        /* surrogate variance growth per unit time */
  int particles;          /* coupled particles per realization (Sec. 6.4), 0 = independent paths */
  double omega;           /* nearest-neighbour coupling of the ring */
  double ax, av;          /* ellipse half-axes: tracking term ORC_TRACK_ELLIPSE (Eq.
                             phonon_functional_tracking) and the coupled initial states */
} orc_feedback;

/* The bump phi(x, x_c, eps) of r = x - x_c, and its derivative in x. */
double orc_bump(double r, double eps);
double orc_bump_dr(double r, double eps);
/* u(z) under mu_k (L values); du (nullable) gets (u_x, u_v), phi (nullable) the L
 * shape-function values. */
double orc_fb_control(const orc_feedback *F, const double *mu_k, const double *z, double *du,
                      double *phi);
/* One path under feedback: X (Nt+1)*2, lam (Nt+1)*2, G (Nt*L per-path dcost/dmu), cost,
 * njumps (each nullable).  Returns 0 on success.  With F->adjoint == ORC_FB_SURROGATE, G
 * is the surrogate estimate of Sec. 6.5 and lam holds the surrogate costates; the
 * surrogate state of step k is zs_k = z_d(t_k) + sqrt(rate t_k) (xi_0, xi_1), xi the
 * Box-Muller pair of Philox words 0, 1 of counter (k, m, 2 << 24, epoch). */
void orc_fb_surrogate_state(const orc_problem *P, const orc_feedback *F, int k, int64_t m, double zs[2]);
int orc_fb_path(const orc_problem *P, const orc_feedback *F, const double *mu, int64_t m,
                double *X, double *lam, double *G, double *cost, int *njumps);
/* J(mu) and dJ/dmu (Nt*L, nullable), fixed summation order; with F->particles > 0 the
 * interacting-particle rings (orc_fb_coupled_gradient). */
int orc_fb_cost(const orc_problem *P, const orc_feedback *F, const double *mu, int nthreads,
                double *J);
int orc_fb_gradient(const orc_problem *P, const orc_feedback *F, const double *mu, int nthreads,
                    double *J, double *grad);
/* Interacting particles (Sec. 6.4 eq:interacting_model): N = F->particles particles
 * (3 <= N <= ORC_RING_MAX) on a ring, particle i of realization r with the random streams
 * of path index S r + i, S = orc_ring_lanes(N) (32 for N <= 32, the next power of two up
 * to 256, then the next multiple of 256),
 *   dx_i = v_i dt,  dv_i = (u(x_i, v_i, t) - eta x_i - omega (2 x_i - x_{i-1} - x_{i+1})) dt + ...
 * (eta = -A[1][0]; the own term 2 omega x_i with the particle's drift; the neighbours'
 * positions at t_k drive every sub-step of step k).  Particles start equidistant on the
 * ellipse (ax cos(2 pi i/N), av sin(2 pi i/N)).  X (Nt+1)*N*2, lam (Nt+1)*N*2, G (Nt*L,
 * summed over the realization's particles), cost (sum of the particles' path costs); each
 * nullable. */
#define ORC_RING_MAX 2048
int orc_ring_lanes(int N);
int orc_fb_coupled(const orc_problem *P, const orc_feedback *F, const double *mu, int64_t r, double *X,
                   double *lam, double *G, double *cost);
/* J = (1/(R N)) sum over R = M/S realizations and N particles; grad likewise (Nt*L). */
int orc_fb_coupled_gradient(const orc_problem *P, const orc_feedback *F, const double *mu, int nthreads,
                            double *J, double *grad);
/* Gradient descent with the Armijo rule on mu (Algorithm 5.4, unconstrained): the same
 * zeta schedule and stopping tests as orc_optimize; mu (Nt*L) is updated in place. */
int orc_fb_optimize(const orc_problem *P, const orc_feedback *F, double *mu, const orc_opt_params *o,
                    int nthreads, orc_opt_result *r, double *J_hist);

#ifdef __cplusplus
}
#endif
#endif
