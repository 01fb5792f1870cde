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


def _pair_vs_single(jp, **kw):
    u1, r1, h1 = jp.optimize(tol_rel_grad=0.0, raise_on_error=False, pairs=False, **kw)
    u2, r2, h2 = jp.optimize(tol_rel_grad=0.0, raise_on_error=False, pairs=True, **kw)
    assert r1["status"] == r2["status"]
    assert r1["iters"] == r2["iters"] and r1["evals"] == r2["evals"] and r1["zeta"] == r2["zeta"]
    assert np.array_equal(u1, u2)
    assert np.array_equal(h1, h2, equal_nan=True)
    assert r1["sweeps"] <= r1["evals"]
    return r1, r2


@pytest.mark.parametrize("prec,mode", [("fp32", "stored"), ("fp32", "recompute"), ("fp64", "stored")])
@pytest.mark.parametrize("zeta0", [1.0, 512.0])
def test_paired_trials_take_the_sequential_iterates(prec, mode, zeta0):
    """Armijo trials in pairs (zeta and zeta / 2 in one forward sweep on the same draws,
    tested in backtracking order) against one trial per sweep: bitwise the same iterates,
    J history, evaluation count and final step, in fewer sweeps.  zeta0 = 512 makes the
    first iteration reject both points of its pair and backtrack further with single
    trials."""
    p = workloads.double_well(M=4096 + 77, Nt=150)
    with JdProblem(p, prec=prec, mode=mode) as jp:
        r1, r2 = _pair_vs_single(jp, max_iter=10, zeta0=zeta0)
    assert r1["status"] == 0 and r1["iters"] == 10
    assert r1["evals"] > r1["iters"] + 1   # some iteration backtracked
    assert r2["sweeps"] < r1["sweeps"]


def test_paired_trials_with_resets_and_the_lq_workload():
    """Keilson-Storer resets (jumps through the general jump step) and the FP64 scalar
    workload: the same iterates with and without pairs."""
    p = workloads.ks_oscillator(M=2048, Nt=120)
    with JdProblem(p, prec="fp32") as jp:
        _pair_vs_single(jp, max_iter=8)
    with JdProblem(workloads.lq_scalar(), prec="fp64") as jp:
        _, r2 = _pair_vs_single(jp, max_iter=50)
    assert r2["sweeps"] < r2["evals"]


@pytest.mark.parametrize("max_backtracks", [0, 1, 2, 3, 4])
def test_paired_trials_exhaust_backtracks_like_single_trials(max_backtracks):
    """armijo_c > 1 rejects every trial: both forms stop with LINESEARCH after the same
    evaluations, the pairs never trying a point single trials would not."""
    p = workloads.lq_scalar(M=300, Nt=20)
    with JdProblem(p, prec="fp64") as jp:
        r1, r2 = _pair_vs_single(jp, max_iter=3, armijo_c=5.0, max_backtracks=max_backtracks)
    assert r1["status"] == 5 and r1["evals"] == 1 + max_backtracks + 1


def test_paired_trials_fall_back_when_the_budget_holds_one_set():
    """A memory budget that holds the plan's buffers once: one trial per sweep, the same
    result."""
    p = workloads.double_well(M=4096, Nt=100)
    with JdProblem(p, prec="fp32", mode="stored") as jp:
        jp.gradient(np.zeros((p.Nt, p.du)))
        need = jp.info()["device_bytes"]
    with JdProblem(p, prec="fp32", mode="stored", mem_budget=need + 4096) as jp:
        r1, r2 = _pair_vs_single(jp, max_iter=6)
        assert jp.info()["device_bytes"] == need
    assert r2["sweeps"] == r1["sweeps"]


def test_paired_trials_at_the_benchmark_size():
    """The benchmark workload at full size (d = 2, M = 2^20, N_t = 1000, stored plan): three
    iterations with paired trials and with one trial per sweep give bitwise the same
    iterates and J history; the paired run takes fewer sweeps."""
    p = workloads.double_well()
    with JdProblem(p, prec="fp32", mode="stored") as jp:
        r1, r2 = _pair_vs_single(jp, max_iter=3, zeta0=2.0)
    assert r1["status"] == 0 and r1["iters"] == 3
    assert r2["sweeps"] <= r1["sweeps"]
