"""Path sharding (through the C ABI): one problem's paths split into shards of whole
units (JD_UNIT_PATHS paths) that run as separate problems (m_offset, M), whose unit sums
jd_combine_units joins.  The result must be jd_gradient / jd_cost of the whole problem
bit for bit, for every split, plan and precision, and the shards' own J must be the
means over their paths (the oracle on the same global path indices)."""
import numpy as np
import pytest

import oracle
import workloads
from paper_2505_04328_gb300 import JdError, JdProblem, binding, build

pytestmark = pytest.mark.gpu
U = binding.UNIT_PATHS


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _shards(p, cuts):
    edges = [0] + list(cuts) + [p.M]
    return [p.replace(M=b - a, m_offset=a) for a, b in zip(edges[:-1], edges[1:])]


SPLITS = {"two": [2 * U], "three": [U, 2 * U], "units": [U, 2 * U, 3 * U]}


@pytest.mark.parametrize("prec,mode", [("fp32", "stored"), ("fp32", "recompute"), ("fp64", "stored")])
@pytest.mark.parametrize("split", sorted(SPLITS))
def test_sharded_gradient_equals_whole_problem_bitwise(prec, mode, split):
    p = workloads.double_well(M=3 * U + 777, Nt=57)
    u = workloads.random_control(p, seed=7, scale=0.5)
    with JdProblem(p, prec=prec, mode=mode) as whole:
        J, g, _ = whole.gradient(u)
        Jc = whole.cost(u)
    units, cunits = [], []
    for s in _shards(p, SPLITS[split]):
        with JdProblem(s, prec=prec, mode=mode) as sp:
            units.append(sp.gradient_units(u))
            cunits.append(sp.cost_units(u))
    Js, gs = binding.combine_units(p, u, np.concatenate(units))
    assert Js == J and np.array_equal(gs, g)
    Jcs, _ = binding.combine_units(p, u, np.concatenate(cunits))
    assert Jcs == Jc
    # the gradient units' cost column is the cost units
    assert np.array_equal(np.concatenate(units)[:, :1], np.concatenate(cunits))


def test_shard_is_the_mean_over_its_own_global_paths():
    """A shard's jd_gradient is the oracle's mean over the same global paths: the draws
    are keyed by the global path index m_offset + m."""
    p = workloads.double_well(M=2 * U, Nt=20)
    u = workloads.random_control(p, seed=8, scale=0.5)
    s = p.replace(M=300, m_offset=U)
    with JdProblem(s, prec="fp64") as sp:
        J, g, _ = sp.gradient(u)
    paths = [oracle.path(p, u, m) for m in range(U, U + 300)]
    Jo = np.mean([r["cost"] for r in paths]) + 0.5 * p.nu * p.dt * float(np.sum(u * u))
    go = np.mean([r["G"] for r in paths], axis=0) + p.nu * p.dt * u
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    assert np.linalg.norm(g - go) <= 1e-12 * np.linalg.norm(go)


def test_units_need_a_unit_boundary():
    p = workloads.double_well(M=2 * U, Nt=20)
    u = np.zeros((p.Nt, p.du))
    with JdProblem(p.replace(M=1000, m_offset=100)) as sp:
        with pytest.raises(JdError) as e:
            sp.gradient_units(u)
        assert e.value.status == binding.JD_ERR_INVALID_ARG
        sp.gradient(u)   # a shard at any offset still evaluates its own mean
    with pytest.raises(JdError):
        JdProblem(p.replace(M=1000, m_offset=(1 << 32) - 10))
