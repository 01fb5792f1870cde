"""GPU parity of the feedback-control form (jd_fb_cost, jd_fb_gradient) against the FP64
oracle (Sec. 2 eq:control_structure, Sec. 5.1-5.2, Sec. 5.5, Sec. 6 eq:tracking_cost).

Bars:
* FP64 path arithmetic: J within 1e-13 relative, dJ/dmu within 1e-12 relative L2 (the
  only differences are summation orders; measured below 1e-15);
* FP32 path arithmetic (FP64 reductions): J within 1e-6 relative, dJ/dmu within 1e-5
  relative L2.  The gradient entries are sums over paths of products of four FP32
  quantities (delta, w, phi_x, phi_v), each carrying the FP32 rounding of the states and
  costates accumulated over the horizon and the exp/reciprocal rounding of the bumps
  (a few 1e-7 relative; measured 5e-8 to 1.4e-7); the bars leave a factor of about 10.
* the same call twice gives the same bits; host and device weights give the same bits;
* at full size (M = 2^20, N_t = 100) the FP64 gradient matches central differences of
  the FP64 cost along random directions (1e-6 relative), and the FP32 gradient matches
  the FP64 one (1e-5 relative L2).
"""
import numpy as np
import pytest

import oracle
import workloads
from paper_2505_04328_gb300 import JdError, JdProblem, build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


CASES = {
    # the paper's 10 x 10 bumps, Gaussian tracking, resets at a raised rate
    "centering": lambda: (lambda p, f: (p.replace(lam=8.0), f))(*workloads.feedback_centering(M=600, Nt=43)),
    # Sec. 6.3 target, eps = 0.1 (every bump reaches every point)
    "trajectory": lambda: workloads.feedback_trajectory(M=333, Nt=40),
    # padded instances: 4 x 3 in the 4 x 4 kernels, 13 x 11 in the 16 x 16 kernels; quadratic
    # tracking, additive normal jumps on a cubic drift
    "small_quad": lambda: (workloads.double_well_phase(M=257, Nt=33).replace(lam=6.0),
                           workloads.Feedback(nx=4, nv=3, x_max=2.0, v_max=1.5, eps=0.6,
                                              track=workloads.TRACK_QUAD)),
    "large_gauss": lambda: (lambda p, f: (p.replace(lam=4.0), f.replace(nx=13, nv=11, eps=0.35, sigma_J=0.7)))(
        *workloads.feedback_centering(M=300, Nt=25)),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cost_and_gradient_parity(case, prec):
    p, fb = CASES[case]()
    mu = workloads.random_mu(p, fb, seed=21, scale=0.6)
    Jo, go = oracle.fb_gradient(p, fb, mu)
    with JdProblem(p, prec=prec) as jp:
        Jc = jp.fb_cost(fb, mu)
        J, g = jp.fb_gradient(fb, mu)
    eJ, eg = abs(J - Jo) / abs(Jo), rel_l2(g, go)
    print(f"{case} {prec}: J {eJ:.2e}  grad {eg:.2e}")
    assert Jc == J
    if prec == "fp64":
        assert eJ <= 1e-13 and eg <= 1e-12
    else:
        assert eJ <= 1e-6 and eg <= 1e-5


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_state_on_the_support_boundary(prec):
    """Centres at -1 and 1 (x_max = 2, nx = 2), eps = 1/2: a state held at (1, 1) (A = 0,
    B = 0, no noise, no jumps) lies exactly on the edge |x - x_c| = 1/eps of the bumps at
    -1, where 1 - eps^2 r^2 == 0.  The bump and its derivative are 0 there, not NaN."""
    p, _ = workloads.feedback_centering(M=96, Nt=12)
    p = p.replace(A=np.zeros((2, 2)), B=np.zeros((2, 1)), sigma=np.zeros(2), lam=0.0, x0=np.array([1.0, 1.0]))
    fb = workloads.Feedback(nx=2, nv=2, x_max=2.0, v_max=2.0, eps=0.5)
    mu = workloads.random_mu(p, fb, seed=25)
    Jo, go = oracle.fb_gradient(p, fb, mu)
    with JdProblem(p, prec=prec) as jp:
        J, g = jp.fb_gradient(fb, mu)
    assert np.isfinite(J) and np.all(np.isfinite(g))
    assert abs(J - Jo) <= 1e-6 * abs(Jo) and rel_l2(g, go) <= 1e-5


def test_repeatable_and_device_weights():
    torch = pytest.importorskip("torch")
    p, fb = CASES["centering"]()
    mu = workloads.random_mu(p, fb, seed=22, scale=0.5)
    with JdProblem(p) as jp:
        J1, g1 = jp.fb_gradient(fb, mu)
        J2, g2 = jp.fb_gradient(fb, mu)
        md = torch.tensor(mu, dtype=torch.float64, device="cuda")
        J3, g3 = jp.fb_gradient(fb, md)
        Jc = jp.fb_cost(fb, md)
    assert J1 == J2 and np.array_equal(g1, g2)
    assert J3 == J1 and np.array_equal(g3.cpu().numpy(), g1) and Jc == J1


def test_unsupported_and_invalid():
    p = workloads.lq_scalar(M=256, Nt=16)
    fb = workloads.Feedback()
    with JdProblem(p) as jp:
        with pytest.raises(JdError) as e:
            jp.fb_cost(fb, np.zeros((16, fb.L)))
        assert e.value.status == 7
    q, fb = workloads.feedback_centering(M=256, Nt=16)
    with JdProblem(q) as jp:
        for bad in (fb.replace(nx=17), fb.replace(eps=0.0), fb.replace(sigma_J=-1.0)):
            with pytest.raises(JdError) as e:
                jp.fb_cost(bad, np.zeros((16, bad.nx * bad.nv)))
            assert e.value.status == 1
        mu = np.zeros((16, fb.L))
        mu[3, 7] = np.nan
        with pytest.raises(JdError):
            jp.fb_cost(fb, mu)


def test_full_size_directional_derivative():
    """M = 2^20, N_t = 100 (the feedback benchmark size)."""
    p, fb = workloads.feedback_centering()
    mu = workloads.random_mu(p, fb, seed=23, scale=0.5)
    rng = np.random.default_rng(24)
    with JdProblem(p, prec="fp64") as jp:
        J, g = jp.fb_gradient(fb, mu)
        h = 1e-3
        for _ in range(2):
            e = rng.standard_normal(mu.shape)
            e /= np.linalg.norm(e)
            fd = (jp.fb_cost(fb, mu + h * e) - jp.fb_cost(fb, mu - h * e)) / (2 * h)
            dd = float((g * e).sum())
            print(f"fd {fd:.10e} adjoint {dd:.10e}")
            assert abs(fd - dd) <= 1e-6 * np.linalg.norm(g)
    with JdProblem(p, prec="fp32") as jp:
        J32, g32 = jp.fb_gradient(fb, mu)
    print(f"fp32 vs fp64: J {abs(J32 - J) / abs(J):.2e} grad {rel_l2(g32, g):.2e}")
    assert abs(J32 - J) <= 1e-6 * abs(J) and rel_l2(g32, g) <= 1e-5


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_optimizer_follows_the_oracle(prec):
    """Algorithm 5.4 on mu: the GPU descent takes the oracle's iterate sequence (the same
    accept/reject decisions); FP64 J history within 1e-10 relative and the final weights
    within 1e-9 of their scale, FP32 within the FP32 bars (1e-6 for J, 1e-5 for mu)."""
    p, fb = workloads.feedback_centering(M=700, Nt=20)
    p = p.replace(lam=6.0)
    muo, ro, ho = oracle.fb_optimize(p, fb, max_iter=6)
    with JdProblem(p, prec=prec) as jp:
        mu, r, h = jp.fb_optimize(fb, max_iter=6)
    print(prec, r, ro)
    assert r["status"] == 0 and r["iters"] == ro["iters"] and r["evals"] == ro["evals"]
    tJ, tm = (1e-10, 1e-9) if prec == "fp64" else (1e-6, 1e-5)
    assert np.max(np.abs(h - ho) / np.abs(ho)) <= tJ
    assert np.max(np.abs(mu - muo)) <= tm * np.max(np.abs(muo))
    assert np.all(np.diff(h) < 0)


@pytest.mark.parametrize("case", ["centering", "trajectory", "small_quad"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_surrogate_gradient_parity(case, prec):
    """Sec. 6.5 surrogate adjoint (costates along states drawn around the target) against
    the oracle's: the same surrogate states (same Philox counter), the same jump counts,
    the same pairing with the forward's sub-steps."""
    p, fb = CASES[case]()
    fb = fb.replace(adjoint=workloads.FB_SURROGATE, sur_rate=0.3)
    mu = workloads.random_mu(p, fb, seed=26, scale=0.6)
    Jo, go = oracle.fb_gradient(p, fb, mu)
    with JdProblem(p, prec=prec) as jp:
        J, g = jp.fb_gradient(fb, mu)
        J2, g2 = jp.fb_gradient(fb, mu)
    eJ, eg = abs(J - Jo) / abs(Jo), rel_l2(g, go)
    print(f"surrogate {case} {prec}: J {eJ:.2e}  grad {eg:.2e}")
    assert J == J2 and np.array_equal(g, g2)
    if prec == "fp64":
        assert eJ <= 1e-13 and eg <= 1e-12
    else:
        assert eJ <= 1e-6 and eg <= 1e-5


@pytest.mark.parametrize("N", [5, 32, 33, 256, 2000])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_coupled_particles_parity(N, prec):
    """Sec. 6.4: rings of N coupled particles, ellipse tracking cost, shared weights;
    against the oracle's rings.  N <= 32: one warp per ring (shuffles); N <= 256: rings
    within a block (shared memory); N > 256: a ring per thread-block cluster (distributed
    shared memory)."""
    S = oracle.ring_lanes(N)
    R = {32: 37, 64: 12, 256: 5, 2048: 3}[S]   # rings (whole blocks beyond one warp)
    p, fb = workloads.feedback_coupled(M=S * R, Nt=30, particles=N)
    p = p.replace(lam=5.0)
    mu = workloads.random_mu(p, fb, seed=27, scale=0.6)
    Jo, go = oracle.fb_coupled_gradient(p, fb, mu)
    with JdProblem(p, prec=prec) as jp:
        Jc = jp.fb_cost(fb, mu)
        J, g = jp.fb_gradient(fb, mu)
    eJ, eg = abs(J - Jo) / abs(Jo), rel_l2(g, go)
    print(f"coupled N={N} {prec}: J {eJ:.2e}  grad {eg:.2e}")
    assert Jc == J
    if prec == "fp64":
        assert eJ <= 1e-13 and eg <= 1e-12
    else:
        assert eJ <= 1e-6 and eg <= 1e-5


@pytest.mark.parametrize("N,R", [(8, 12), (256, 2)])
def test_coupled_optimizer_follows_the_oracle(N, R):
    """Algorithm 5.4 on the shared weights of the coupled rings (FP64): the oracle's iterate
    sequence, J history within 1e-10."""
    p, fb = workloads.feedback_coupled(M=oracle.ring_lanes(N) * R, Nt=20, particles=N)
    p = p.replace(lam=4.0)
    muo, ro, ho = oracle.fb_optimize(p, fb, max_iter=5)
    with JdProblem(p, prec="fp64") as jp:
        mu, r, h = jp.fb_optimize(fb, max_iter=5)
    print("coupled optimizer", r, ro)
    assert r["iters"] == ro["iters"] and r["evals"] == ro["evals"]
    assert np.max(np.abs(h - ho) / np.abs(ho)) <= 1e-10
    assert np.max(np.abs(mu - muo)) <= 1e-9 * np.max(np.abs(muo))
    assert h[-1] < h[0]


def test_feedback_resampling_descent_follows_the_oracle():
    p, fb = workloads.feedback_centering(M=500, Nt=15)
    p = p.replace(lam=6.0, epoch=2)
    muo, ro, ho = oracle.fb_optimize(p, fb, max_iter=5, resample=True)
    with JdProblem(p, prec="fp64") as jp:
        mu, r, h = jp.fb_optimize(fb, max_iter=5, resample=True)
    assert r["iters"] == ro["iters"] and r["evals"] == ro["evals"]
    assert np.max(np.abs(h - ho) / np.abs(ho)) <= 1e-10
    assert np.max(np.abs(mu - muo)) <= 1e-9 * np.max(np.abs(muo))


def test_optimizer_reuses_the_accepted_trial_sweep():
    """With the exact adjoint and a fixed sample each gradient after the first takes the
    accepted trial's sweep as its forward half: forward sweeps = 1 + trials, i.e. evals
    minus the iterations plus one; the resampled descent (new sample per gradient) and the
    surrogate adjoint (its own forward) run one sweep per evaluation.  The J history
    equals the costs of the iterates evaluated afresh."""
    p, fb = workloads.feedback_centering(M=700, Nt=20)
    p = p.replace(lam=6.0)
    with JdProblem(p, prec="fp64") as jp:
        mu, r, h = jp.fb_optimize(fb, max_iter=4, tol_rel_grad=0.0)
        assert r["status"] == 0 and r["iters"] == 4 and r["sweeps"] == r["evals"] - r["iters"] + 1
        assert jp.fb_cost(fb, mu) == pytest.approx(h[-1], rel=1e-13)
        _, rr, _ = jp.fb_optimize(fb, max_iter=3, tol_rel_grad=0.0, resample=True)
        assert rr["sweeps"] == rr["evals"]
        _, rs, _ = jp.fb_optimize(fb.replace(adjoint=workloads.FB_SURROGATE, sur_rate=0.05), max_iter=3,
                                  tol_rel_grad=0.0)
        assert rs["sweeps"] == rs["evals"]
