"""Host logic of the autograd form (no GPU): the parameter map theta -> problem and the
chain rule that turns the library's per-coefficient derivatives into dJ/dtheta.

Both are checked through the FP64 oracle: its adjoint parameter derivatives, composed by
compose_theta_grad, must match central finite differences of its cost along theta
(h = 1e-4, the step of the autograd config).  A wrong sign, a dropped sigma component
or a swapped entry of the composition fails here.
"""
import numpy as np
import pytest

import oracle
import workloads
from paper_2505_04328_gb300.autograd import compose_theta_grad, theta_problem

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _base(M=512, Nt=64):
    return workloads.double_well_autograd(M=M, Nt=Nt)


def test_theta_problem_arrays():
    p = _base()
    A_base = p.A - 0.5 * p.dA
    assert np.allclose(A_base, [[1.0, 0.0], [0.0, 0.0]])
    q = theta_problem(p, A_base, np.ones(2), (0.7, 0.25, 0.1))
    assert np.allclose(q.A, [[1.0, 0.0], [0.0, -0.7]])
    assert np.allclose(q.sigma, [0.25, 0.25]) and q.jump_scale == 0.1
    # everything else is the base problem's
    assert q.M == p.M and q.Nt == p.Nt and np.array_equal(q.xd, p.xd) and q.seed == p.seed
    # theta0 = (0.5, 0.3, 0.2) reproduces the base problem
    q0 = theta_problem(p, A_base, np.ones(2), (0.5, 0.3, 0.2))
    assert np.array_equal(q0.A, p.A) and np.array_equal(q0.sigma, p.sigma) and q0.jump_scale == p.jump_scale


def test_compose_layout():
    g = np.array([1.0, 2.0, 3.0, 4.0])       # [dA, sigma_0, sigma_1, jump]
    assert np.allclose(compose_theta_grad(g, np.ones(2)), [1.0, 5.0, 4.0])
    assert np.allclose(compose_theta_grad(g, np.array([0.5, 2.0])), [1.0, 7.0, 4.0])


@pytest.mark.parametrize("sigma_shape", [np.ones(2), np.array([1.0, 0.5])])
def test_chain_rule_against_fd_of_the_oracle(sigma_shape):
    p = _base()
    A_base = p.A - 0.5 * p.dA
    theta = np.array([0.5, 0.3, 0.2])
    u = workloads.random_control(p, seed=3, scale=0.5)
    pt = theta_problem(p, A_base, sigma_shape, theta)
    _, _, gth = oracle.gradient(pt, u, theta=True)
    dtheta = compose_theta_grad(gth, sigma_shape)
    h = 1e-4
    fd = np.zeros(3)
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        jp = oracle.cost(theta_problem(p, A_base, sigma_shape, theta + e), u)
        jm = oracle.cost(theta_problem(p, A_base, sigma_shape, theta - e), u)
        fd[i] = (jp - jm) / (2 * h)
    assert np.allclose(dtheta, fd, rtol=1e-6, atol=1e-9), (dtheta, fd)
