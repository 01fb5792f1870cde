"""Pins for the oracle's projected-gradient Armijo optimizer (Algorithm 5.4).

* In the linear-quadratic case J is an exact quadratic in u (sample average over fixed
  draws), so its box-constrained minimum is computed independently: the Hessian is
  assembled from gradients and the QP solved by scipy's L-BFGS-B.  The oracle's
  iterates must decrease J monotonically and approach that minimum.
* Consistency of the discrete optimum with the continuous one (Thm. 3.2): the
  discrete optimal control approaches the continuous LQ optimum (computed on a fine
  grid with scipy) as N_t and M grow.
"""
import numpy as np

import oracle
import workloads
from oracle import closed_forms as cf


def test_lq_optimizer_reaches_discrete_qp_optimum():
    p = workloads.lq_scalar(M=200, Nt=20)
    n = p.Nt
    ustar, H, g0 = cf.discrete_qp_optimum(
        lambda v: oracle.gradient(p, v.reshape(n, 1))[1].ravel(), n, p.u_min, p.u_max)
    Jstar = oracle.cost(p, ustar.reshape(n, 1))
    u, res, hist = oracle.optimize(p, max_iter=300, tol_rel_grad=1e-10)
    assert res["status"] == 0
    assert np.all(np.diff(hist) <= 1e-15)
    assert hist[-1] >= Jstar - 1e-12
    assert hist[-1] - Jstar < 1e-9 * abs(Jstar)
    assert np.abs(u.ravel() - ustar).max() < 1e-3
    # at the optimum some bounds are active (the target needs |u| > 5)
    assert np.isclose(np.abs(ustar).max(), 5.0)


def test_lq_armijo_fifty_iterations_monotone():
    p = workloads.lq_scalar()
    u, res, hist = oracle.optimize(p, max_iter=50, tol_rel_grad=0.0)
    assert res["iters"] == 50 and res["status"] == 0
    assert np.all(np.diff(hist) <= 0)
    assert hist[-1] < 0.5 * hist[0]


def test_discrete_optimum_approaches_continuous_lq_optimum():
    tm, ucont, _ = cf.scalar_lq_continuous_optimum(
        1.0, 1.0, lambda t: np.sin(2 * np.pi * t), 1e-3, -5.0, 5.0, 1.0, n=4000)
    errs = []
    for Nt, M in ((20, 100), (80, 400)):
        p = workloads.lq_scalar(M=M, Nt=Nt)
        u, res, _ = oracle.optimize(p, max_iter=400, tol_rel_grad=1e-8)
        # continuous optimum averaged over each control cell
        cells = ucont.reshape(Nt, -1).mean(axis=1)
        errs.append(np.sqrt(np.mean((u.ravel() - cells) ** 2)) / np.sqrt(np.mean(cells ** 2)))
    assert errs[1] < errs[0]
    assert errs[1] < 0.1


# --- per-iteration resampling (Sec. 5.6 SGD, Algorithm 5.4 with fresh samples) -----------
def test_resampling_without_randomness_is_the_fixed_sample_descent():
    """No noise and no jumps: every sample is the same, so the resampled descent takes the
    fixed-sample iterates exactly."""
    p = workloads.lq_scalar(M=64, Nt=30).replace(sigma=np.array([0.0]), lam=0.0)
    u1, r1, h1 = oracle.optimize(p, max_iter=6)
    u2, r2, h2 = oracle.optimize(p, max_iter=6, resample=True)
    assert np.array_equal(h1, h2) and np.array_equal(u1, u2)


def test_resampling_uses_the_sample_of_each_iteration():
    """Iteration n evaluates its gradient and its Armijo trials on epoch e0 + n: J_hist[n] is
    the cost of u^n on sample e0 + n, and the last entry the accepted trial's cost of u^{N}
    on the sample of the last iteration, e0 + N - 1."""
    p = workloads.lq_scalar(M=300, Nt=30).replace(epoch=5)
    us = [oracle.optimize(p, max_iter=n, resample=True)[0] for n in range(4)]
    _, r, h = oracle.optimize(p, max_iter=3, resample=True)
    assert r["iters"] == 3
    for n in range(3):
        assert h[n] == oracle.cost(p.replace(epoch=5 + n), us[n])
    assert h[3] == oracle.cost(p.replace(epoch=7), us[3]) == r["J"]
    # and the samples differ: the fixed-sample descent takes other iterates
    assert not np.array_equal(oracle.optimize(p, max_iter=3)[2], h)
