"""GPU tests of the autograd form J(u, theta) (torch.autograd.Function over jd_forward /
jd_backward), theta = (damping rho, sigma, jump half-width) of the double-well problem.

Bars (the gradient is checked at a seeded random control, not at an optimum):
* FP64 GPU form: adjoint gradients vs central finite differences of the same function
  with h = 1e-4, relative agreement <= 1e-6 (the FD truncation error is O(h^2 J''')).
* FP32 GPU form vs the FP64 oracle's adjoint gradient: relative L2 <= 1e-4 for u and
  for theta.
* FP32 finite differences vs the FP32 adjoint: FP32 rounding of J (about 1e-7 |J|)
  divided by h = 1e-4 gives an FD noise of about 1e-3 |J|; the bar is 5e-3 relative
  to max(|dJ/dtheta_i|, 0.05 |J|).
* Backward results are bitwise equal to jd_gradient's, and equal in the stored and
  recompute plans.
"""
import numpy as np
import pytest

import oracle
import workloads
from paper_2505_04328_gb300 import build
from paper_2505_04328_gb300.autograd import JumpDiffusionCost, compose_theta_grad, theta_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THETA0 = (0.5, 0.3, 0.2)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _setup(M=4096, Nt=200, prec="fp32", mode="recompute"):
    p = workloads.double_well_autograd(M=M, Nt=Nt)
    f = JumpDiffusionCost(p, rho0=0.5, prec=prec, mode=mode)
    u0 = workloads.random_control(p, seed=31, scale=0.5)
    return p, f, u0


def _eval(f, u0, theta, grad=True):
    u = torch.tensor(u0, dtype=torch.float64, device="cuda", requires_grad=grad)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=grad)
    J = f(u, th)
    if not grad:
        return float(J.detach())
    J.backward()
    return float(J.detach()), u.grad.cpu().numpy(), th.grad.numpy()


def test_fp64_against_central_differences():
    p, f, u0 = _setup(M=2048, Nt=128, prec="fp64")
    J, gu, gth = _eval(f, u0, THETA0)
    h = 1e-4
    th0 = np.array(THETA0)
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        fd = (_eval(f, u0, th0 + e, False) - _eval(f, u0, th0 - e, False)) / (2 * h)
        assert abs(fd - gth[i]) <= 1e-6 * max(abs(gth[i]), 1e-3 * abs(J)), (i, fd, gth[i])
    rng = np.random.default_rng(4)
    for _ in range(4):
        e = rng.standard_normal(u0.shape)
        e /= np.linalg.norm(e)
        fd = (_eval(f, u0 + h * e, THETA0, False) - _eval(f, u0 - h * e, THETA0, False)) / (2 * h)
        dd = float(np.sum(gu * e))
        assert abs(fd - dd) <= 1e-6 * max(abs(dd), np.linalg.norm(gu)), (fd, dd)
    f.close()


@pytest.mark.parametrize("mode", ["recompute", "stored"])
def test_fp32_against_oracle_adjoint(mode):
    p, f, u0 = _setup(M=2048, Nt=256, mode=mode)
    J, gu, gth = _eval(f, u0, THETA0)
    pt = theta_problem(p, p.A - 0.5 * p.dA, np.ones(2), THETA0)
    Jo, go, gtho = oracle.gradient(pt, u0, theta=True)
    dth_o = compose_theta_grad(gtho, np.ones(2))
    print(f"{mode}: J {abs(J - Jo) / abs(Jo):.2e}, grad_u relL2 {np.linalg.norm(gu - go) / np.linalg.norm(go):.2e}, "
          f"theta {np.abs(gth - dth_o) / np.abs(dth_o)}")
    assert abs(J - Jo) <= 1e-5 * abs(Jo)
    assert np.linalg.norm(gu - go) <= 1e-4 * np.linalg.norm(go)
    assert np.linalg.norm(gth - dth_o) <= 1e-4 * np.linalg.norm(dth_o)
    f.close()


def test_fp32_central_differences():
    p, f, u0 = _setup(M=8192, Nt=200)
    J, gu, gth = _eval(f, u0, THETA0)
    h = 1e-4
    th0 = np.array(THETA0)
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        fd = (_eval(f, u0, th0 + e, False) - _eval(f, u0, th0 - e, False)) / (2 * h)
        print(f"theta_{i}: adjoint {gth[i]:.6e} fd {fd:.6e}")
        assert abs(fd - gth[i]) <= 5e-3 * max(abs(gth[i]), 0.05 * abs(J))
    f.close()


def test_backward_matches_gradient_and_plans_agree():
    outs = {}
    for mode in ("recompute", "stored"):
        p, f, u0 = _setup(M=3000, Nt=150, mode=mode)
        J, gu, gth = _eval(f, u0, THETA0)
        # jd_gradient on the same problem object and coefficients
        Jg, gg, gthg = f.problem.gradient(u0, theta=True)
        assert J == Jg and np.array_equal(gu, gg)
        assert np.array_equal(gth, compose_theta_grad(gthg, np.ones(2)))
        outs[mode] = (J, gu, gth)
        f.close()
    a, b = outs["recompute"], outs["stored"]
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_interleaved_evaluations():
    """Two forwards, then the first one's backward: the kept states belong to the second
    evaluation, so the function re-runs the first forward before the adjoint."""
    p, f, u0 = _setup(M=2048, Nt=100)
    J1, g1, t1 = _eval(f, u0, THETA0)
    u = torch.tensor(u0, dtype=torch.float64, device="cuda", requires_grad=True)
    th = torch.tensor(THETA0, dtype=torch.float64, requires_grad=True)
    Ja = f(u, th)
    Jb = f(u * 0.5, torch.tensor((0.6, 0.3, 0.2), dtype=torch.float64))
    Ja.backward()
    assert float(Ja.detach()) == J1 and np.array_equal(u.grad.cpu().numpy(), g1) and np.array_equal(th.grad.numpy(), t1)
    assert float(Jb.detach()) != J1
    f.close()


def test_full_size_plans_agree():
    """The autograd workload at full size (M = 2^22, N_t = 4096): the recompute plan
    (checkpoints) and the stored plan (137 GB of states) give bitwise-equal J, dJ/du and
    dJ/dtheta."""
    p = workloads.double_well_autograd()
    u0 = workloads.random_control(p, seed=32, scale=0.5)
    res = []
    for mode, budget in (("recompute", 0), ("stored", 200 << 30)):
        f = JumpDiffusionCost(p, rho0=0.5, mode=mode, mem_budget=budget)
        res.append(_eval(f, u0, THETA0))
        assert f.problem.info()["mode"] == mode
        f.close()
        torch.cuda.synchronize()
    (Ja, ga, ta), (Jb, gb, tb) = res
    assert np.isfinite(Ja) and np.all(np.isfinite(ga)) and np.all(np.isfinite(ta))
    assert Ja == Jb and np.array_equal(ga, gb) and np.array_equal(ta, tb)
