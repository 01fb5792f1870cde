"""Closed forms and independent solvers that pin the oracle (TEST INFRASTRUCTURE ONLY).

Nothing here calls the oracle's C library except ``discrete_qp_optimum``, which only
uses its gradients to assemble the exact Hessian of a quadratic J and then solves the
box-constrained QP with scipy (an independent optimizer).

* Linear drift with additive noise and zero-mean compound-Poisson jumps
  (Sec. 2 eq:compact_forward with linear H, Sec. 5.4 eq:coefficients): the mean obeys
  m' = A m + B u and the covariance P' = A P + P A^T + diag(sigma^2) + lambda E[xi xi^T].
* Pure ODE limits (sigma = 0, lambda = 0) have textbook solutions; explicit Euler
  converges to them at order one (Thm. 3.1 of the paper is the stochastic analogue).
* The continuous LQ optimum for the scalar problem: with additive noise the variance
  does not depend on u, so E[1/2 int (X - xd)^2] = 1/2 int Var + 1/2 int (m - xd)^2 and
  the optimal open-loop control solves a deterministic problem on the mean.
"""
from __future__ import annotations

import numpy as np
from scipy import integrate, linalg, optimize


def scalar_linear_moments(a, x0, sigma, lam, jump_var, t):
    """Mean and variance of dX = -a X dt + sigma dW + dJ, u = 0 (closed form)."""
    t = np.asarray(t, dtype=np.float64)
    m = np.exp(-a * t) * x0
    v = (sigma ** 2 + lam * jump_var) / (2 * a) * (1 - np.exp(-2 * a * t))
    return m, v


def linear_moments(A, B, sigma, lam, jump_cov, x0, u_of_t, t_eval):
    """Mean and covariance of dX = (A X + B u(t)) dt + diag(sigma) dW + dJ by solving
    the moment ODEs with scipy (rtol 1e-11)."""
    d = A.shape[0]
    Qn = np.diag(np.asarray(sigma) ** 2) + lam * np.asarray(jump_cov)

    def rhs(t, y):
        m = y[:d]
        P = y[d:].reshape(d, d)
        dm = A @ m + B @ np.atleast_1d(u_of_t(t))
        dP = A @ P + P @ A.T + Qn
        return np.concatenate([dm, dP.ravel()])

    y0 = np.concatenate([np.asarray(x0, dtype=np.float64), np.zeros(d * d)])
    sol = integrate.solve_ivp(rhs, (0.0, float(t_eval[-1])), y0, t_eval=t_eval, rtol=1e-11,
                              atol=1e-13, method="DOP853")
    m = sol.y[:d].T
    P = sol.y[d:].T.reshape(-1, d, d)
    return m, P


def linear_mean_expm(A, x0, t):
    """m(t) = expm(A t) x0 (u = 0)."""
    return np.stack([linalg.expm(A * tt) @ x0 for tt in np.atleast_1d(t)])


def double_well_ode(x0, t):
    """Exact solution of x' = x - x^3, x(0) = x0."""
    t = np.asarray(t, dtype=np.float64)
    e = np.exp(2 * t)
    return x0 * np.exp(t) / np.sqrt(1 + x0 ** 2 * (e - 1))


def scalar_lq_continuous_optimum(a, x0, target, nu, u_min, u_max, T, n=20000):
    """Optimal open-loop control of min 1/2 int_0^T (m - xd)^2 dt + nu/2 int u^2 dt,
    m' = -a m + u, m(0) = x0, u in [u_min, u_max], on a fine uniform grid of n steps
    (exact exponential propagation per step, control piecewise constant, trapezoid
    quadrature); solved with scipy L-BFGS-B.  Returns (t_mid, u) with u on the n cells."""
    h = T / n
    t = np.arange(n + 1) * h
    xd = target(t)
    ea = np.exp(-a * h)
    gain = (1 - ea) / a

    def fwd(u):
        m = np.empty(n + 1)
        m[0] = x0
        for k in range(n):
            m[k + 1] = ea * m[k] + gain * u[k]
        return m

    w = np.full(n + 1, h)
    w[0] = w[-1] = h / 2

    def fg(u):
        m = fwd(u)
        e = m - xd
        J = 0.5 * np.sum(w * e * e) + 0.5 * nu * h * np.sum(u * u)
        # adjoint of the exact-exponential recursion
        lam = np.zeros(n + 1)
        lam[n] = w[n] * e[n]
        g = np.empty(n)
        for k in range(n - 1, -1, -1):
            g[k] = gain * lam[k + 1] + nu * h * u[k]
            lam[k] = ea * lam[k + 1] + w[k] * e[k]
        return J, g

    res = optimize.minimize(fg, np.zeros(n), jac=True, method="L-BFGS-B",
                            bounds=[(u_min, u_max)] * n,
                            options=dict(maxiter=20000, ftol=1e-15, gtol=1e-12, maxcor=30))
    return t[:-1] + h / 2, res.x, res.fun


def discrete_qp_optimum(grad_fn, n, lo, hi, h=1.0):
    """Box-constrained minimum of a quadratic J whose gradient is grad_fn(u) (n vars).
    The Hessian is assembled exactly (J quadratic) from n+1 gradients; the QP is then
    solved by scipy L-BFGS-B to machine precision.  Returns (u*, Hessian, g0)."""
    g0 = grad_fn(np.zeros(n))
    H = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = h
        H[:, j] = (grad_fn(e) - g0) / h
    H = 0.5 * (H + H.T)

    def fg(u):
        Hu = H @ u
        return 0.5 * u @ Hu + g0 @ u, Hu + g0

    res = optimize.minimize(fg, np.zeros(n), jac=True, method="L-BFGS-B",
                            bounds=[(lo, hi)] * n,
                            options=dict(maxiter=100000, ftol=1e-16, gtol=1e-14, maxcor=50))
    return res.x, H, g0
