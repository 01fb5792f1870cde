"""Pins of the oracle's interacting-particle form (Sec. 6.4 eq:interacting_model, Eq.
phonon_functional_tracking): rings of N particles (3 <= N <= 2048), particle i of
realization r on the random streams of path index S r + i (S = ring_lanes(N): 32 for
N <= 32, the next power of two up to 256, then the next multiple of 256), the
neighbours' positions at t_k driving the step.  Each pin runs a ring of at most 32
particles and one of more.

* omega = 0 decouples the ring: each particle is the single-particle feedback path from
  its ellipse point (cost and gradient add up);
* the deterministic coupled sweep converges at first order to scipy's solution of the
  2N-dimensional linear ODE with the ring Laplacian;
* the ellipse cost is -1 per unit time on the ellipse and -exp(-E^2/(2 sigma_J^2)) off it;
* the gradient in mu matches central differences with noise, resets and coupling, and the
  initial costates match differences in the ellipse half-axes (which set the initial
  states).
"""
import numpy as np
import pytest

import oracle
import workloads

scipy = pytest.importorskip("scipy")
from scipy import integrate  # noqa: E402


def _ellipse(fb, N):
    th = 2 * np.pi * np.arange(N) / N
    return np.stack([fb.ax * np.cos(th), fb.av * np.sin(th)], axis=1)


def test_ring_lanes():
    assert [oracle.ring_lanes(n) for n in (3, 32, 33, 64, 65, 200, 256, 257, 2000, 2048)] == \
        [32, 32, 64, 64, 128, 256, 256, 512, 2048, 2048]


@pytest.mark.parametrize("N", [5, 40])
def test_zero_coupling_is_independent_particles(N):
    S = oracle.ring_lanes(N)
    p, fb = workloads.feedback_coupled(M=2 * S, Nt=25, particles=N)
    p = p.replace(lam=6.0)
    fb = fb.replace(omega=0.0)
    mu = workloads.random_mu(p, fb, seed=4, scale=0.6)
    Z0 = _ellipse(fb, N)
    for r in (0, 1):
        c = oracle.fb_coupled(p, fb, mu, r)
        cost, G = 0.0, np.zeros_like(c["G"])
        for i in range(N):
            s = oracle.fb_path(p.replace(x0=Z0[i]), fb.replace(particles=0), mu, S * r + i)
            cost += s["cost"]
            G += s["G"]
            assert np.allclose(c["X"][:, i], s["X"], rtol=1e-14, atol=1e-14)
        assert c["cost"] == pytest.approx(cost, rel=1e-13)
        assert np.allclose(c["G"], G, rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("N", [6, 40])
def test_coupled_euler_converges_to_the_ring_ode(N):
    """No noise, no jumps, constant weights: z' = (x', v') with x_i' = v_i,
    v_i' = u(x_i, v_i) - eta x_i - omega (2 x_i - x_{i-1} - x_{i+1})."""
    p0, fb = workloads.feedback_coupled(M=oracle.ring_lanes(N), Nt=10, particles=N)
    fb = fb.replace(nx=4, nv=4, omega=0.7)
    mu1 = np.random.default_rng(12).standard_normal(fb.L) * 0.5
    eta = -p0.A[1, 0]

    def rhs(t, y):
        x, v = y[:N], y[N:]
        u = np.array([oracle.fb_control(fb, mu1, (x[i], v[i]))[0] for i in range(N)])
        lap = 2 * x - np.roll(x, 1) - np.roll(x, -1)
        return np.concatenate([v, u - eta * x - fb.omega * lap])

    Z0 = _ellipse(fb, N)
    ref = integrate.solve_ivp(rhs, (0.0, p0.T), np.concatenate([Z0[:, 0], Z0[:, 1]]), method="DOP853",
                              rtol=1e-12, atol=1e-14).y[:, -1]
    errs = []
    for Nt in (100, 200, 400):
        p = p0.replace(Nt=Nt, sigma=np.zeros(2), lam=0.0, xd=np.zeros((Nt + 1, 2)))
        X = oracle.fb_coupled(p, fb, np.tile(mu1, (Nt, 1)), 0, adjoint=False)["X"][-1]
        errs.append(np.linalg.norm(np.concatenate([X[:, 0], X[:, 1]]) - ref))
    assert errs[0] > 1e-5
    for e1, e2 in zip(errs, errs[1:]):
        assert 1.8 < e1 / e2 < 2.2, errs


def test_ellipse_cost_closed_forms():
    """Held still (A = 0, B = 0, no noise, no jumps, no coupling) on the ellipse the cost is
    -1 per unit time and particle; a single particle held at (1.1 A_x, 0) has
    E = 1.1^2 - 1 = 0.21 and costs -T exp(-E^2 / (2 sigma_J^2))."""
    p, fb = workloads.feedback_coupled(M=64, Nt=20, particles=7)
    p = p.replace(A=np.zeros((2, 2)), B=np.zeros((2, 1)), sigma=np.zeros(2), lam=0.0)
    fb = fb.replace(omega=0.0)
    J, _ = oracle.fb_coupled_gradient(p, fb, np.zeros((p.Nt, fb.L)))
    assert J == pytest.approx(-p.T, rel=1e-14)
    one = oracle.fb_path(p.replace(x0=np.array([1.1 * fb.ax, 0.0])), fb.replace(particles=0),
                         np.zeros((p.Nt, fb.L)), 0, adjoint=False)["cost"]
    assert one == pytest.approx(-p.T * np.exp(-0.21 ** 2 / (2 * fb.sigma_J ** 2)), rel=1e-13)


def _fd(fun, x, e, h):
    return (fun(x + h * e) - fun(x - h * e)) / (2 * h)


@pytest.mark.parametrize("N", [6, 40])
def test_coupled_gradient_central_differences(N):
    p, fb = workloads.feedback_coupled(M=2 * oracle.ring_lanes(N), Nt=20, particles=N)
    p = p.replace(lam=8.0)
    mu = workloads.random_mu(p, fb, seed=5, scale=0.6)
    J, g = oracle.fb_coupled_gradient(p, fb, mu)
    rng = np.random.default_rng(13)
    for _ in range(3):
        e = rng.standard_normal(mu.shape)
        e /= np.linalg.norm(e)
        fd = _fd(lambda m: oracle.fb_coupled_gradient(p, fb, m)[0], mu, e, 1e-4)
        assert abs(fd - float((g * e).sum())) <= 1e-7 * np.linalg.norm(g), (fd, (g * e).sum())


@pytest.mark.parametrize("N", [5, 300])
def test_initial_costates_against_differences_in_the_ellipse_axes(N):
    """With the Gaussian tracking term the cost depends on the half-axes only through the
    initial states (A_x cos th_i, A_v sin th_i): dJ/dA_x = sum_i lambda_x,i(0) cos th_i and
    dJ/dA_v = sum_i lambda_v,i(0) sin th_i, with the coupling (omega = 0.5), noise and
    resets in the adjoint."""
    p, fb = workloads.feedback_coupled(M=oracle.ring_lanes(N), Nt=30, particles=N)
    p = p.replace(lam=5.0)
    fb = fb.replace(track=workloads.TRACK_GAUSS)
    mu = workloads.random_mu(p, fb, seed=6, scale=0.5)
    lam0 = oracle.fb_coupled(p, fb, mu, 0)["lam"][0]
    th = 2 * np.pi * np.arange(N) / N
    h = 1e-6
    for key, comp, w in (("ax", 0, np.cos(th)), ("av", 1, np.sin(th))):
        v = getattr(fb, key)
        cp = oracle.fb_coupled(p, fb.replace(**{key: v + h}), mu, 0, adjoint=False)["cost"]
        cm = oracle.fb_coupled(p, fb.replace(**{key: v - h}), mu, 0, adjoint=False)["cost"]
        fd = (cp - cm) / (2 * h)
        ad = float((lam0[:, comp] * w).sum())
        assert abs(fd - ad) <= 1e-7 * max(1.0, abs(fd)), (key, fd, ad)
