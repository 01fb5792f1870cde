"""Pins for the oracle's forward sweep and cost against closed forms.

* sigma = 0, lambda = 0: explicit Euler of an ODE with a textbook solution converges at
  order one (linear: exponential; cubic double well: x0 e^t / sqrt(1 + x0^2 (e^{2t}-1))).
* Linear drift with noise and zero-mean jumps: Monte Carlo mean and covariance of X_k
  against the moment ODEs m' = A m + B u, P' = A P + P A^T + diag(sigma^2) + lambda E[xi xi^T]
  (scalar closed form, and scipy for d = 4), within Monte Carlo error plus O(dt).
* Jump-only dynamics: X_T - X_0 is the compound-Poisson sum, variance lambda T E[xi^2].
* Cost: with sigma = 0 and lambda = 0 the cost is a plain Riemann sum over the grid
  points k = 1..Nt (eq:discrete_functional), evaluated here with the exact ODE solution
  up to the Euler error; its mean under noise equals 1/2 sum dt q (Var + (m - xd)^2).
"""
import numpy as np
import pytest

import oracle
import workloads
from oracle import closed_forms as cf


def _paths(p, u=None, M=None):
    M = M or p.M
    return np.stack([oracle.path(p, u, m, adjoint=False)["X"] for m in range(M)])


def test_linear_ode_euler_order_one():
    errs = []
    for Nt in (50, 100, 200, 400):
        p = workloads.lq_scalar(M=1, Nt=Nt).replace(sigma=np.array([0.0]), lam=0.0)
        u = np.full((Nt, 1), 0.7)
        X = oracle.path(p, u, 0, adjoint=False)["X"][:, 0]
        t = np.arange(Nt + 1) * p.dt
        exact = np.exp(-t) * 1.0 + (1 - np.exp(-t)) * 0.7
        errs.append(np.abs(X - exact).max())
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(ratios - 2.0) < 0.1), ratios


def test_double_well_ode_euler_order_one():
    errs = []
    for Nt in (200, 400, 800, 1600):
        p = workloads.double_well(M=1, Nt=Nt).replace(sigma=np.zeros(2), lam=0.0,
                                                      x0=np.array([0.3, 0.0]))
        X = oracle.path(p, None, 0, adjoint=False)["X"]
        t = np.arange(Nt + 1) * p.dt
        assert np.allclose(X[:, 1], 0.0)
        errs.append(np.abs(X[:, 0] - cf.double_well_ode(0.3, t)).max())
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(ratios - 2.0) < 0.1), ratios


def test_harmonic_oscillator_euler_order_one():
    """The paper's H = [[0, 1], [-eta, 0]] (Sec. 5.4): x' = v, v' = -eta x; exact
    x = cos(w t), v = -w sin(w t) for x0 = (1, 0), w = sqrt(eta).  A transposed A
    gives x' = -eta v, v' = x and misses this solution."""
    eta = 2.0
    w = np.sqrt(eta)
    errs = []
    for Nt in (200, 400, 800, 1600):
        p = workloads.double_well(M=1, Nt=Nt).replace(
            drift=workloads.LINEAR, A=np.array([[0.0, 1.0], [-eta, 0.0]]), sigma=np.zeros(2),
            lam=0.0, x0=np.array([1.0, 0.0]))
        X = oracle.path(p, None, 0, adjoint=False)["X"]
        t = np.arange(Nt + 1) * p.dt
        exact = np.stack([np.cos(w * t), -w * np.sin(w * t)], axis=1)
        errs.append(np.abs(X - exact).max())
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(ratios - 2.0) < 0.15), ratios


def test_scalar_moments_match_closed_form():
    M, Nt = 6000, 200
    p = workloads.lq_scalar(M=M, Nt=Nt).replace(lam=6.0, jump_scale=0.15)
    X = _paths(p)[:, :, 0]
    t = np.arange(Nt + 1) * p.dt
    m, v = cf.scalar_linear_moments(1.0, 1.0, 0.2, p.lam, p.jump_scale ** 2, t)
    for k in (50, 100, 200):
        se_m = np.sqrt(v[k] / M)
        assert abs(X[:, k].mean() - m[k]) < 4.5 * se_m + 2 * p.dt * m[k]
        se_v = v[k] * np.sqrt(2.0 / M) * 1.5   # jumps make the tails heavier
        assert abs(X[:, k].var() - v[k]) < 4.5 * se_v + 2 * p.dt * v[k]


def test_linear4_mean_and_covariance():
    M, Nt = 4000, 100
    p = workloads.linear_family(4, M=M, Nt=Nt, lam=3.0)
    u = np.tile([0.5, -0.25], (Nt, 1))
    X = _paths(p, u)
    t = np.arange(Nt + 1) * p.dt
    mean, P = cf.linear_moments(p.A, p.B, p.sigma, p.lam, p.jump_scale ** 2 * np.eye(4), p.x0,
                                lambda s: np.array([0.5, -0.25]), t)
    for k in (25, 100):
        emp_m = X[:, k].mean(0)
        emp_P = np.cov(X[:, k].T)
        se = np.sqrt(np.diag(P[k]) / M)
        assert np.all(np.abs(emp_m - mean[k]) < 4.5 * se + 3 * p.dt * np.abs(mean[k]) + 1e-12)
        scale = np.sqrt(np.outer(np.diag(P[k]), np.diag(P[k])))
        assert np.all(np.abs(emp_P - P[k]) < 5.0 * scale * np.sqrt(2.0 / M) + 3 * p.dt * scale)


@pytest.mark.parametrize("law", [workloads.JUMP_NORMAL, workloads.JUMP_UNIFORM])
def test_jump_only_compound_poisson(law):
    M, Nt = 6000, 20
    p = workloads.lq_scalar(M=M, Nt=Nt).replace(A=np.array([[0.0]]), sigma=np.array([0.0]),
                                                 lam=3.0, jump_law=law, jump_scale=0.5)
    X = _paths(p)[:, :, 0]
    incr = X[:, -1] - X[:, 0]
    second = 0.25 if law == workloads.JUMP_NORMAL else 0.25 / 3.0
    var = p.lam * p.T * second
    assert abs(incr.mean()) < 4.5 * np.sqrt(var / M)
    assert abs(incr.var() / var - 1) < 4.5 * np.sqrt(2.0 / M) * 2.0
    # probability of no jump at all on [0, T]
    assert abs((incr == 0).mean() - np.exp(-p.lam * p.T)) < 4.5 * np.sqrt(np.exp(-3) / M)


def test_deterministic_cost_riemann_sum():
    Nt = 400
    p = workloads.lq_scalar(M=3, Nt=Nt).replace(sigma=np.array([0.0]), lam=0.0, nu=0.01)
    u = np.full((Nt, 1), 0.3)
    J = oracle.cost(p, u)
    t = np.arange(Nt + 1) * p.dt
    x = np.exp(-t) + (1 - np.exp(-t)) * 0.3
    riemann = np.sum(p.dt * 0.5 * (x[1:] - np.sin(2 * np.pi * t[1:])) ** 2)
    assert abs(J - (riemann + 0.5 * 0.01 * p.dt * Nt * 0.09)) < 5e-3 * riemann


def test_cost_mean_matches_moments():
    M, Nt = 4000, 100
    p = workloads.lq_scalar(M=M, Nt=Nt)
    J = oracle.cost(p)
    t = np.arange(Nt + 1) * p.dt
    m, v = cf.scalar_linear_moments(1.0, 1.0, 0.2, p.lam, p.jump_scale ** 2, t)
    exact = np.sum(p.dt * 0.5 * (v[1:] + (m[1:] - np.sin(2 * np.pi * t[1:])) ** 2))
    assert abs(J - exact) < 0.02 * exact


def test_cost_and_gradient_independent_of_thread_count():
    p = workloads.double_well(M=700, Nt=60)
    u = workloads.random_control(p, scale=0.3)
    J1, g1, _ = oracle.gradient(p, u, nthreads=1)
    J4, g4, _ = oracle.gradient(p, u, nthreads=5)
    assert J1 == J4 and np.array_equal(g1, g4)


def test_keilson_storer_moments_closed_form():
    """Pure velocity resets v <- gamma v + s xi at Poisson times of rate lam (no drift,
    no diffusion): with N(t) ~ Poisson(lam t),
        E v(t)   = v0 exp(-lam (1 - gamma) t),
        E v(t)^2 = v0^2 exp(-lam (1 - gamma^2) t) + s^2 (1 - exp(-lam (1 - gamma^2) t)) / (1 - gamma^2),
    and the position component of z = (x, v) is never moved by a reset."""
    lam, gamma, s, v0, T = 3.0, 0.6, 0.4, 1.5, 1.0
    p = workloads.ks_oscillator(M=20000, Nt=8).replace(
        A=np.zeros((2, 2)), B=np.zeros((2, 1)), sigma=np.zeros(2), x0=np.array([0.25, v0]),
        lam=lam, jump_scale=s, jump_gain=gamma, T=T)
    X = np.stack([oracle.path(p, None, m, adjoint=False)["X"][-1] for m in range(p.M)])
    assert np.all(X[:, 0] == 0.25)
    v = X[:, 1]
    m1 = v0 * np.exp(-lam * (1 - gamma) * T)
    e2 = np.exp(-lam * (1 - gamma ** 2) * T)
    m2 = v0 ** 2 * e2 + s ** 2 * (1 - e2) / (1 - gamma ** 2)
    se1 = np.sqrt(np.var(v) / p.M)
    se2 = np.sqrt(np.var(v ** 2) / p.M)
    assert abs(v.mean() - m1) < 4 * se1, (v.mean(), m1, se1)
    assert abs(np.mean(v ** 2) - m2) < 4 * se2, (np.mean(v ** 2), m2, se2)
