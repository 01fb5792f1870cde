"""Pins of the oracle's feedback-control form (Sec. 2 eq:control_structure, Sec. 5.1-5.2,
Sec. 5.5, Sec. 6 eq:tracking_cost), each against something other than the oracle:

* the bump function: phi(0) = 1/e, compact support |r| < 1/eps, and its integral, the
  classical constant int_{-1}^{1} exp(-1/(1-t^2)) dt = 0.443993816168079... (scaled by
  1/eps), by scipy quadrature; its derivative by central differences;
* the shape-function layout: a point on a cell centre with eps large enough that only
  that centre's bump reaches it gives u = mu[i, l] / e^2 (cell centres of Sec. 5.1,
  row-major [i][l] with nx != nv); a rank-one mu = a b^T gives u = (a . phi_x)(b . phi_v);
* the controlled forward sweep: first-order convergence of the Euler sweep to scipy's
  high-accuracy solution of z' = A z + B u(z) (no noise, no jumps);
* the cost: exact tracking gives J = -T for the Gaussian cost; a frozen state gives the
  control cost (alpha/2) dt sum_k u_k^2 in closed form;
* the adjoint and the gradient in mu: central differences in random directions of mu,
  in single entries, and in the initial state (lambda_0), with noise and Keilson-Storer
  resets, for both tracking costs; the per-path sensitivities average to the gradient;
* the optimizer (Algorithm 5.4 on mu): monotone Armijo decrease, and on a frozen state
  convergence to the closed-form infimum T l(z0) (the control cost goes to 0).
"""
import numpy as np
import pytest

import oracle
import workloads

scipy = pytest.importorskip("scipy")
from scipy import integrate  # noqa: E402

BUMP_INTEGRAL = 0.44399381616807943782   # int_{-1}^{1} exp(-1/(1-t^2)) dt


def test_bump_values_support_and_integral():
    for eps in (0.5, 0.1, 2.0):
        assert oracle.bump(0.0, eps) == pytest.approx(np.exp(-1.0), rel=1e-15)
        assert oracle.bump(1.0 / eps, eps) == 0.0 and oracle.bump(-1.5 / eps, eps) == 0.0
        r = np.linspace(-0.99 / eps, 0.99 / eps, 7)
        assert np.allclose(oracle.bump(r, eps), oracle.bump(-r, eps), rtol=0, atol=0)
        val, err = integrate.quad(lambda t: oracle.lib().orc_bump(t, eps), -1.0 / eps, 1.0 / eps,
                                  limit=200, epsabs=1e-14, epsrel=1e-13)
        assert val == pytest.approx(BUMP_INTEGRAL / eps, rel=1e-10)


def test_bump_derivative_central_differences():
    eps, h = 0.5, 1e-6
    for r in np.linspace(-1.95, 1.95, 29):
        fd = (oracle.bump(r + h, eps) - oracle.bump(r - h, eps)) / (2 * h)
        assert oracle.bump_dr(r, eps) == pytest.approx(fd, rel=1e-7, abs=1e-12), r
    assert oracle.bump_dr(0.0, eps) == 0.0 and oracle.bump_dr(2.5, eps) == 0.0


def test_centre_layout_single_bump():
    """nx = 4, nv = 3 on (-2, 2) x (-1.5, 1.5): centres x^i = (i + 1/2) - 2, v^l = (l + 1/2) - 1.5.
    eps = 1.2 makes the support radius 0.83 < 1, the centre spacing: only one bump reaches
    a centre, so u = mu[i, l] phi(0)^2 and the gradient vanishes there."""
    fb = workloads.Feedback(nx=4, nv=3, x_max=2.0, v_max=1.5, eps=1.2)
    mu = np.arange(1.0, 13.0)
    for i in range(4):
        for l in range(3):
            z = (i + 0.5 - 2.0, l + 0.5 - 1.5)
            u, du, phi = oracle.fb_control(fb, mu, z)
            assert u == pytest.approx(mu[i * 3 + l] * np.exp(-2.0), rel=1e-14)
            assert np.all(np.abs(du) < 1e-15)
            assert np.count_nonzero(phi) == 1 and phi[i * 3 + l] == pytest.approx(np.exp(-2.0))


def test_rank_one_weights_factor():
    fb = workloads.Feedback(nx=5, nv=3, x_max=2.0, v_max=1.0, eps=0.4)
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal(5), rng.standard_normal(3)
    xc = (np.arange(5) + 0.5) * 0.8 - 2.0
    vc = (np.arange(3) + 0.5) * (2.0 / 3.0) - 1.0
    for z in rng.uniform(-2.5, 2.5, size=(6, 2)):
        u, du, _ = oracle.fb_control(fb, np.outer(a, b).reshape(-1), z)
        px, pv = oracle.bump(z[0] - xc, fb.eps), oracle.bump(z[1] - vc, fb.eps)
        dpx, dpv = oracle.bump_dr(z[0] - xc, fb.eps), oracle.bump_dr(z[1] - vc, fb.eps)
        assert u == pytest.approx((a @ px) * (b @ pv), rel=1e-12, abs=1e-15)
        assert du[0] == pytest.approx((a @ dpx) * (b @ pv), rel=1e-12, abs=1e-15)
        assert du[1] == pytest.approx((a @ px) * (b @ dpv), rel=1e-12, abs=1e-15)


def _deterministic(Nt, eta=1.0):
    p, fb = workloads.feedback_centering(M=1, Nt=Nt, eta=eta)
    return p.replace(sigma=np.zeros(2), lam=0.0), fb


def test_euler_converges_to_the_controlled_ode():
    """Constant weights: z' = A z + B u(z) is autonomous; scipy (DOP853, rtol 1e-12) gives
    z(T).  The Euler error must halve when N_t doubles."""
    rng = np.random.default_rng(11)
    fb = workloads.Feedback(nx=4, nv=4, eps=0.5)
    mu1 = rng.standard_normal(fb.L)
    p0, _ = _deterministic(10)
    A, B = p0.A, p0.B[:, 0]

    def rhs(t, z):
        u, _, _ = oracle.fb_control(fb, mu1, z)
        return A @ z + B * u

    ref = integrate.solve_ivp(rhs, (0.0, p0.T), p0.x0, method="DOP853", rtol=1e-12, atol=1e-14).y[:, -1]
    errs = []
    for Nt in (100, 200, 400):
        p, _ = _deterministic(Nt)
        X = oracle.fb_path(p, fb, np.tile(mu1, (Nt, 1)), 0, adjoint=False)["X"]
        errs.append(np.linalg.norm(X[-1] - ref))
    assert errs[0] > 1e-5
    for e1, e2 in zip(errs, errs[1:]):
        assert 1.8 < e1 / e2 < 2.2, errs


def test_cost_exact_tracking_gaussian():
    p, fb = _deterministic(40)
    p = p.replace(x0=np.zeros(2))                  # z stays at z_d = 0 with mu = 0
    assert oracle.fb_cost(p, fb, np.zeros((40, fb.L)), nthreads=1) == pytest.approx(-p.T, rel=1e-15)


def test_control_cost_frozen_state():
    """B = 0, A = 0: the state stays on the centre (i, l) = (2, 1); with a large eps only
    that bump is on, so u_k = mu[k, (2,1)] / e^2 and the cost is (alpha/2) dt sum u_k^2 plus
    the constant quadratic tracking term."""
    fb = workloads.Feedback(nx=4, nv=3, x_max=2.0, v_max=1.5, eps=1.2, track=workloads.TRACK_QUAD)
    p, _ = _deterministic(25)
    p = p.replace(A=np.zeros((2, 2)), B=np.zeros((2, 1)), x0=np.array([0.5, 0.0]), q=np.array([1.0, 0.0]))
    mu = np.random.default_rng(2).standard_normal((25, fb.L))
    uk = mu[:, 2 * 3 + 1] * np.exp(-2.0)
    dt = p.T / p.Nt
    want = 0.5 * p.nu * dt * np.sum(uk ** 2) + p.Nt * dt * 0.5 * 0.5 ** 2
    assert oracle.fb_cost(p, fb, mu, nthreads=1) == pytest.approx(want, rel=1e-13)


def _fd(fun, x, e, h):
    return (fun(x + h * e) - fun(x - h * e)) / (2 * h)


@pytest.mark.parametrize("track", [workloads.TRACK_GAUSS, workloads.TRACK_QUAD])
def test_gradient_central_differences(track):
    p, fb = workloads.feedback_centering(M=200, Nt=30)
    p = p.replace(lam=8.0)                          # several resets per path
    fb = fb.replace(track=track, sigma_J=0.8)
    mu = workloads.random_mu(p, fb, seed=4, scale=0.7)
    J, g = oracle.fb_gradient(p, fb, mu)
    rng = np.random.default_rng(9)
    for _ in range(3):
        e = rng.standard_normal(mu.shape)
        e /= np.linalg.norm(e)
        fd = _fd(lambda m: oracle.fb_cost(p, fb, m), mu, e, 1e-4)
        assert abs(fd - float((g * e).sum())) <= 1e-7 * np.linalg.norm(g), (fd, (g * e).sum())
    for (k, l) in [(0, 44), (12, 55), (29, 45)]:
        e = np.zeros(mu.shape)
        e[k, l] = 1.0
        fd = _fd(lambda m: oracle.fb_cost(p, fb, m), mu, e, 1e-4)
        assert abs(fd - g[k, l]) <= 1e-7 * np.abs(g).max() + 1e-12, (k, l, fd, g[k, l])


def test_lambda0_is_derivative_wrt_initial_state():
    p, fb = workloads.feedback_centering(M=4, Nt=50)
    p = p.replace(lam=10.0)
    mu = workloads.random_mu(p, fb, seed=5, scale=0.8)
    for m in range(3):
        r = oracle.fb_path(p, fb, mu, m)
        assert r["njumps"].sum() > 0
        for c in range(2):
            e = np.zeros(2)
            e[c] = 1e-6
            fd = (oracle.fb_path(p.replace(x0=p.x0 + e), fb, mu, m, adjoint=False)["cost"]
                  - oracle.fb_path(p.replace(x0=p.x0 - e), fb, mu, m, adjoint=False)["cost"]) / 2e-6
            assert abs(fd - r["lam"][0, c]) <= 1e-7 * max(1.0, abs(fd)), (m, c, fd, r["lam"][0, c])


def test_path_sensitivities_average_to_the_gradient():
    p, fb = workloads.feedback_trajectory(M=300, Nt=12)
    mu = workloads.random_mu(p, fb, seed=6)
    J, g = oracle.fb_gradient(p, fb, mu, nthreads=3)
    rs = [oracle.fb_path(p, fb, mu, m) for m in range(p.M)]
    assert J == pytest.approx(np.mean([r["cost"] for r in rs]), rel=1e-13)
    assert np.allclose(g, np.mean([r["G"] for r in rs], axis=0), rtol=1e-12, atol=1e-16)
    # the thread count does not change the bits
    J1, g1 = oracle.fb_gradient(p, fb, mu, nthreads=1)
    assert J1 == J and np.array_equal(g1, g)


def test_optimizer_decreases_and_satisfies_armijo():
    p, fb = workloads.feedback_centering(M=300, Nt=15)
    mu, r, hist = oracle.fb_optimize(p, fb, max_iter=8)
    assert r["status"] == 0 and r["iters"] == 8
    assert np.all(np.diff(hist) < 0), hist
    # the final iterate's cost is the oracle's cost at the returned weights
    assert oracle.fb_cost(p, fb, mu) == pytest.approx(r["J"], rel=0, abs=0)


def test_optimizer_reaches_the_closed_form_minimum():
    """B = 0, A = 0, no noise, no jumps: the state stays at z0 and only the control cost
    (alpha/2) dt sum_k (mu_k . phi(z0))^2 depends on mu; its infimum is 0, so J converges
    to the constant tracking part N_t dt l(z0) = T l(z0)."""
    p, fb = workloads.feedback_centering(M=4, Nt=10)
    p = p.replace(A=np.zeros((2, 2)), B=np.zeros((2, 1)), sigma=np.zeros(2), lam=0.0, x0=np.array([0.3, -0.2]))
    fb = fb.replace(eps=0.3)
    mu0 = workloads.random_mu(p, fb, seed=2, scale=5.0)
    track = -np.exp(-(0.3 ** 2 + 0.2 ** 2) / (2 * fb.sigma_J ** 2))
    mu, r, hist = oracle.fb_optimize(p, fb, mu0, max_iter=60, tol_rel_grad=1e-12)
    assert hist[0] > p.T * track + 1e-3
    assert r["J"] == pytest.approx(p.T * track, abs=1e-10)


# --- Sec. 6.5: costates along surrogate states -------------------------------------------
def test_surrogate_equals_exact_on_the_forward_trajectory():
    """No noise, no jumps, zero surrogate variance and a target equal to the forward
    trajectory itself (the forward does not depend on the target): the surrogate states
    are the forward states, so the surrogate costates and gradient equal the exact ones
    (the tracking gradients vanish on the target; the drift Jacobian, the feedback terms
    w grad u and the pairing with the forward's phi(Y) remain)."""
    p, fb = workloads.feedback_centering(M=3, Nt=30)
    p = p.replace(sigma=np.zeros(2), lam=0.0)
    mu = workloads.random_mu(p, fb, seed=8, scale=0.7)
    X = oracle.fb_path(p, fb, mu, 0, adjoint=False)["X"]
    for track in (workloads.TRACK_QUAD, workloads.TRACK_GAUSS):
        q, f = p.replace(xd=X), fb.replace(track=track)
        ex = oracle.fb_path(q, f, mu, 0)
        sur = oracle.fb_path(q, f.replace(adjoint=workloads.FB_SURROGATE, sur_rate=0.0), mu, 0)
        assert np.abs(ex["G"]).max() > 1e-6
        assert np.allclose(sur["G"], ex["G"], rtol=1e-13, atol=1e-18)
        assert np.allclose(sur["lam"], ex["lam"], rtol=1e-13, atol=1e-18)


def test_surrogate_state_law():
    """z_d(t_k) + sqrt(rate t_k) xi: mean z_d(t_k), variance rate t_k per component."""
    p, fb = workloads.feedback_trajectory(M=4000, Nt=10)
    fb = fb.replace(adjoint=workloads.FB_SURROGATE, sur_rate=0.3)
    for k in (0, 4, 10):
        Z = np.array([oracle.fb_surrogate_state(p, fb, k, m) for m in range(p.M)])
        var = 0.3 * k * p.T / p.Nt
        if k == 0:
            assert np.all(Z == p.xd[0])
            continue
        se = np.sqrt(var / p.M)
        assert np.all(np.abs(Z.mean(axis=0) - p.xd[k]) < 4 * se)
        assert np.all(np.abs(Z.var(axis=0) - var) < 4 * var * np.sqrt(2.0 / p.M))
        assert abs(np.corrcoef(Z.T)[0, 1]) < 4 / np.sqrt(p.M)


def test_surrogate_costates_do_not_see_the_forward():
    """The surrogate costates depend on the weights, the target and the path's jumps, not
    on the forward states: moving x0 changes the forward (and the gradient) but not them."""
    p, fb = workloads.feedback_centering(M=2, Nt=25)
    p = p.replace(lam=10.0)
    fb = fb.replace(adjoint=workloads.FB_SURROGATE, sur_rate=0.2)
    mu = workloads.random_mu(p, fb, seed=9, scale=0.6)
    a = oracle.fb_path(p, fb, mu, 1)
    b = oracle.fb_path(p.replace(x0=p.x0 + 0.3), fb, mu, 1)
    assert np.array_equal(a["lam"], b["lam"])
    assert not np.allclose(a["G"], b["G"])


def test_surrogate_costates_cross_jumps_with_the_reset_gain():
    """mu = 0 and A = 0: the surrogate costate recursion reduces to
    r_k = diag(1, gamma^{n_k}) r_{k+1} + dt q (zs_k - z_d(t_k)) (k >= 1), n_k the path's jump
    count in step k, r_Nt = dt q (zs_Nt - z_d(t_Nt)); written out here with the oracle's
    surrogate states and jump counts."""
    p, fb = workloads.feedback_centering(M=2, Nt=40)
    p = p.replace(A=np.zeros((2, 2)), lam=9.0, jump_gain=0.6, q=np.array([0.7, 1.3]))
    fb = fb.replace(track=workloads.TRACK_QUAD, adjoint=workloads.FB_SURROGATE, sur_rate=0.4)
    dt = p.T / p.Nt
    lam = oracle.fb_path(p, fb, np.zeros((p.Nt, fb.L)), 1)["lam"]
    r = dt * p.q * (oracle.fb_surrogate_state(p, fb, p.Nt, 1) - p.xd[p.Nt])
    assert np.allclose(lam[p.Nt], r, rtol=1e-14)
    jumps = 0
    for k in range(p.Nt - 1, -1, -1):
        n = oracle.step_draws(p, k, 1)["n"]
        jumps += n
        r = r * np.array([1.0, p.jump_gain ** n])
        if k >= 1:
            r = r + dt * p.q * (oracle.fb_surrogate_state(p, fb, k, 1) - p.xd[k])
        assert np.allclose(lam[k], r, rtol=1e-12, atol=1e-15), k
    assert jumps > 3
