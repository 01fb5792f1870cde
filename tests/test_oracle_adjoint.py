"""Pins for the oracle's adjoint sweep and reduced gradient.

The adjoint is the exact derivative of the discrete cost (discretize-then-optimize,
Sec. 4).  It is pinned by quantities computed without it:
  * central finite differences of J (quadratic J in the linear case: exact up to
    rounding for every h);
  * derivatives taken by sympy of the forward recursion on tiny inputs, using the
    draws the oracle reports for each step (jumps forced by a large intensity);
  * lambda_0 = d(path cost)/dX_0 against finite differences in X_0;
  * the parameter gradients (drift direction, sigma, jump scale) against finite
    differences of J in those parameters.
"""
import numpy as np
import pytest
import sympy as sp

import oracle
import workloads


def _fd(fun, x, e, h):
    return (fun(x + h * e) - fun(x - h * e)) / (2 * h)


def test_fd_linear_quadratic_all_coordinates():
    p = workloads.lq_scalar(M=300, Nt=24)
    u = workloads.random_control(p, scale=0.8)
    _, g, _ = oracle.gradient(p, u)
    for k in range(p.Nt):
        e = np.zeros_like(u)
        e[k, 0] = 1.0
        fd = _fd(lambda v: oracle.cost(p, v), u, e, 1e-2)
        assert abs(fd - g[k, 0]) <= 1e-9 * np.abs(g).max(), k


@pytest.mark.parametrize("maker", [workloads.double_well, workloads.double_well_phase])
def test_fd_cubic_random_directions(maker):
    p = maker(M=512, Nt=80)
    u = workloads.random_control(p, scale=0.5)
    _, g, _ = oracle.gradient(p, u)
    rng = np.random.default_rng(3)
    for _ in range(6):
        e = rng.standard_normal(u.shape)
        e /= np.linalg.norm(e)
        dd = float((g * e).sum())
        for h in (1e-3, 1e-4):
            fd = _fd(lambda v: oracle.cost(p, v), u, e, h)
            assert abs(fd - dd) <= 2e-7 * np.linalg.norm(g) + 1e-12, (h, fd, dd)


def test_fd_harmonic_oscillator_nonsymmetric():
    """The paper's H = [[0, 1], [-eta, 0]] (Sec. 5.4 eq:coefficients) with a cubic term:
    a non-symmetric Jacobian, so a transposed A or C in the adjoint fails here."""
    p = workloads.double_well(M=256, Nt=60).replace(
        A=np.array([[0.0, 1.0], [-1.0, -0.2]]), C=np.array([[0.0, 0.0], [-0.5, 0.0]]))
    u = workloads.random_control(p, scale=0.5)
    _, g, _ = oracle.gradient(p, u)
    rng = np.random.default_rng(11)
    for _ in range(4):
        e = rng.standard_normal(u.shape)
        e /= np.linalg.norm(e)
        fd = _fd(lambda v: oracle.cost(p, v), u, e, 1e-4)
        assert abs(fd - (g * e).sum()) <= 2e-7 * np.linalg.norm(g)


def test_fd_linear32_multicontrol():
    p = workloads.linear_family(8, M=128, Nt=30, lam=2.0)
    u = workloads.random_control(p, scale=0.5)
    _, g, _ = oracle.gradient(p, u)
    rng = np.random.default_rng(5)
    for _ in range(4):
        e = rng.standard_normal(u.shape)
        fd = _fd(lambda v: oracle.cost(p, v), u, e, 1e-2)
        assert abs(fd - (g * e).sum()) <= 1e-10 * np.abs(g).sum()


def test_sympy_derivative_tiny_forced_jumps():
    """M = 1, Nt = 3, d = 1 cubic drift, lambda dt = 2 so most steps carry jumps."""
    p = workloads.lq_scalar(M=1, Nt=3).replace(
        drift=workloads.CUBIC, A=np.array([[0.7]]), C=np.array([[-0.4]]), B=np.array([[1.3]]),
        lam=6.0, jump_law=workloads.JUMP_NORMAL, jump_scale=0.3, sigma=np.array([0.25]),
        x0=np.array([0.8]), q=np.array([1.7]))
    draws = [oracle.step_draws(p, k, 0) for k in range(p.Nt)]
    assert sum(dr["n"] for dr in draws) >= 3
    us = sp.symbols("u0:3")
    x = sp.Float(0.8, 30)
    dt = p.dt
    cost = 0
    xs = [x]
    for k, dr in enumerate(draws):
        y = x
        for i in range(dr["n"] + 1):
            de = dr["delta"][i]
            y = y + de * (0.7 * y - 0.4 * y ** 3 + 1.3 * us[k]) + 0.25 * np.sqrt(de) * dr["Z"][i][0]
            if i < dr["n"]:
                y = y + 0.3 * dr["xi_hat"][i][0]
        x = y
        xs.append(x)
        cost = cost + dt * 0.5 * 1.7 * (x - p.xd[k + 1, 0]) ** 2
    u = np.array([[0.4], [-1.1], [0.9]])
    subs = {us[i]: u[i, 0] for i in range(3)}
    r = oracle.path(p, u, 0)
    assert np.allclose(r["X"][:, 0], [float(e.subs(subs)) for e in xs], rtol=1e-13, atol=1e-14)
    assert abs(r["cost"] - float(cost.subs(subs))) < 1e-13
    for k in range(3):
        exact = float(sp.diff(cost, us[k]).subs(subs))
        assert abs(r["G"][k, 0] - exact) < 1e-12 * max(1.0, abs(exact)), k


def test_lambda0_is_derivative_wrt_initial_state():
    # x0 differs from the target at t = 0, so a cost term at k = 0 would show up
    p = workloads.double_well(M=4, Nt=120).replace(x0=np.array([0.5, 0.3]))
    u = workloads.random_control(p, scale=0.4)
    for m in range(3):
        r = oracle.path(p, u, m)
        for c in range(2):
            def pc(x0c):
                x0 = p.x0.copy()
                x0[c] = x0c
                return oracle.path(p.replace(x0=x0), u, m, adjoint=False)["cost"]
            fd = (pc(p.x0[c] + 1e-5) - pc(p.x0[c] - 1e-5)) / 2e-5
            assert abs(fd - r["lam"][0, c]) < 1e-7 * max(1.0, abs(fd))


def test_parameter_gradients_fd():
    base = workloads.double_well_autograd(M=256, Nt=60)
    u = workloads.random_control(base, scale=0.4)
    _, _, gth = oracle.gradient(base, u, theta=True)
    h = 1e-5
    # drift direction: A(theta) = A + theta dA
    fd = (oracle.cost(base.replace(A=base.A + h * base.dA), u)
          - oracle.cost(base.replace(A=base.A - h * base.dA), u)) / (2 * h)
    assert abs(fd - gth[0]) < 1e-7 * max(1.0, abs(fd))
    for c in range(2):
        e = np.zeros(2)
        e[c] = h
        fd = (oracle.cost(base.replace(sigma=base.sigma + e), u)
              - oracle.cost(base.replace(sigma=base.sigma - e), u)) / (2 * h)
        assert abs(fd - gth[1 + c]) < 1e-7 * max(1.0, abs(fd))
    fd = (oracle.cost(base.replace(jump_scale=base.jump_scale + h), u)
          - oracle.cost(base.replace(jump_scale=base.jump_scale - h), u)) / (2 * h)
    assert abs(fd - gth[3]) < 1e-7 * max(1.0, abs(fd))


def test_gradient_is_mean_of_path_sensitivities():
    p = workloads.double_well(M=37, Nt=40)
    u = workloads.random_control(p, scale=0.3)
    J, g, _ = oracle.gradient(p, u)
    rs = [oracle.path(p, u, m) for m in range(p.M)]
    G = np.mean([r["G"] for r in rs], axis=0)
    assert np.allclose(g, p.nu * p.dt * u + G, rtol=1e-13, atol=1e-16)
    c = np.mean([r["cost"] for r in rs])
    assert abs(J - (c + 0.5 * p.nu * p.dt * (u ** 2).sum())) < 1e-13


# --- Keilson-Storer velocity resets (Sec. 5.3 eq:jump_law) -------------------------
def test_fd_keilson_storer():
    """Reset v <- gamma v + s xi: the adjoint crosses each jump as lambda_v <- gamma
    lambda_v.  Central differences in u (random directions), in x0 (lambda_0), and in
    the jump scale s pin it; a dropped gamma, or a gamma applied to the position,
    fails here."""
    p = workloads.ks_oscillator(M=400, Nt=60, gamma=0.7).replace(lam=6.0)
    u = workloads.random_control(p, scale=0.5)
    _, g, gth = oracle.gradient(p, u, theta=True)
    rng = np.random.default_rng(5)
    for _ in range(4):
        e = rng.standard_normal(u.shape)
        e /= np.linalg.norm(e)
        fd = _fd(lambda v: oracle.cost(p, v), u, e, 1e-4)
        assert abs(fd - float((g * e).sum())) <= 1e-8 * np.linalg.norm(g) + 1e-13
    # lambda_0 of one path against differences in the initial state
    r = oracle.path(p, u, 7)
    for c in range(2):
        e = np.zeros(2)
        e[c] = 1.0
        fd = (oracle.path(p.replace(x0=p.x0 + 1e-5 * e), u, 7)["cost"]
              - oracle.path(p.replace(x0=p.x0 - 1e-5 * e), u, 7)["cost"]) / 2e-5
        assert abs(fd - r["lam"][0, c]) <= 1e-7 * max(1.0, abs(fd)), c
    # jump-scale derivative (only the velocity is moved by a reset)
    h = 1e-5
    fd = (oracle.cost(p.replace(jump_scale=p.jump_scale + h), u)
          - oracle.cost(p.replace(jump_scale=p.jump_scale - h), u)) / (2 * h)
    assert abs(fd - gth[3]) <= 1e-6 * max(1.0, abs(fd))
