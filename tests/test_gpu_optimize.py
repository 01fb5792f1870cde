"""GPU optimizer (jd_optimize: device-side FP64 Armijo test) against the oracle's
projected-gradient Armijo descent (Algorithm 5.4, eq:Stochastic_Armijo)."""
import numpy as np
import pytest

import oracle
import workloads
from paper_2505_04328_gb300 import JdProblem, build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def test_lq_fp64_fifty_iterations_match_oracle():
    """The scalar LQ workload in FP64 (d=1, M=1000, Nt=100): one gradient plus 50
    projected-gradient iterations from u = 0; the iterates follow the oracle's."""
    p = workloads.lq_scalar()
    uo, ro, ho = oracle.optimize(p, max_iter=50, tol_rel_grad=0.0)
    with JdProblem(p, prec="fp64") as jp:
        u, r, h = jp.optimize(max_iter=50, tol_rel_grad=0.0)
    assert r["iters"] == ro["iters"] == 50 and r["evals"] == ro["evals"]
    assert np.allclose(h, ho, rtol=1e-11, atol=0)
    assert np.max(np.abs(u - uo)) <= 1e-9 * max(1.0, np.abs(uo).max())


def test_double_well_fp32_iterates_follow_oracle():
    p = workloads.double_well(M=2048, Nt=100)
    uo, ro, ho = oracle.optimize(p, max_iter=8, tol_rel_grad=0.0)
    with JdProblem(p, prec="fp32") as jp:
        u, r, h = jp.optimize(max_iter=8, tol_rel_grad=0.0)
    assert r["iters"] == 8
    # Armijo decisions are FP64 comparisons of FP32-evaluated costs; the sequences
    # agree unless a decision margin falls below the FP32 cost error (reported then)
    if r["evals"] == ro["evals"]:
        assert np.allclose(h, ho, rtol=1e-4)
        assert np.max(np.abs(u - uo)) <= 1e-3 * max(1.0, np.abs(uo).max())
    assert np.all(np.diff(h) <= 0)


def test_optimizer_reports_linesearch_failure():
    p = workloads.lq_scalar(M=200, Nt=20)
    with JdProblem(p, prec="fp64") as jp:
        # armijo_c > 1 cannot be satisfied by a descent step on a convex quadratic
        u, r, h = jp.optimize(max_iter=3, tol_rel_grad=0.0, armijo_c=5.0, max_backtracks=3,
                              raise_on_error=False)
    assert r["status"] == 5


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_resampling_descent_follows_the_oracle(prec, tol):
    """Per-iteration resampling (Sec. 5.6): iteration n on epoch e0 + n, for the gradient
    and its Armijo trials; the GPU takes the oracle's iterates, and the problem's epoch is
    unchanged afterwards (the same cost before and after the run)."""
    p = workloads.lq_scalar(M=1000, Nt=50).replace(epoch=3)
    uo, ro, ho = oracle.optimize(p, max_iter=8, resample=True)
    with JdProblem(p, prec=prec) as jp:
        J0 = jp.cost(np.zeros((p.Nt, p.du)))
        u, r, h = jp.optimize(max_iter=8, resample=True)
        assert jp.cost(np.zeros((p.Nt, p.du))) == J0
    assert r["iters"] == ro["iters"] and r["evals"] == ro["evals"]
    assert np.max(np.abs(h - ho) / np.abs(ho)) <= tol
    assert np.max(np.abs(u - uo)) <= 10 * tol * max(1.0, np.max(np.abs(uo)))
