"""Small problems take their main-stream and one-jump slot draws from a parallel pre-pass
whose buffers are reused while the draws' key (generator key, epoch, path range, N_t, d,
jump law and thresholds) stays the same.  A result must never depend on what the buffers
held before: the same call twice, a call after the coefficients (jump rate, seed) were
updated, and a full sweep after a sweep over a path range all equal a fresh problem's
result bit for bit, and the updated problem's cost equals the oracle's."""
import numpy as np
import pytest

import oracle
import workloads
from paper_2505_04328_gb300 import JdProblem, build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_reused_draws_follow_the_key(prec):
    p = workloads.double_well(M=3000, Nt=80)
    u = workloads.random_control(p, seed=5, scale=0.5)
    p2 = p.replace(lam=9.0, seed=77)
    with JdProblem(p, prec=prec) as jp:
        J1 = jp.cost(u)
        assert jp.cost(u) == J1                          # reused draws
        jp.update(p2)                                    # new thresholds and generator key
        J2 = jp.cost(u)
        _, g2, _ = jp.gradient(u)
        jp.sample_paths(u, 100, 50)                      # a sweep over another path range
        J3, g3, _ = jp.gradient(u)
    with JdProblem(p2, prec=prec) as fresh:
        Jf = fresh.cost(u)
        Jg, gf, _ = fresh.gradient(u)
    assert J2 == Jf and J2 != J1
    assert J3 == Jg and np.array_equal(g2, gf) and np.array_equal(g3, gf)
    Jo = oracle.cost(p2, u)
    assert abs(J2 - Jo) <= (1e-5 if prec == "fp32" else 1e-12) * abs(Jo)
