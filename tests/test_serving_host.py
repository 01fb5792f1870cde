"""Host side of the serving loop (no GPU): the HBM footprint used for admission
(jd_problem_footprint, host arithmetic in libjd.so) and the request stream of the
serving workload."""
import math

import numpy as np
import pytest

import workloads
from paper_2505_04328_gb300 import JdError, footprint, lib

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    try:
        lib()
    except (RuntimeError, OSError) as e:   # built by build(); the CPU suite builds it
        pytest.skip(f"libjd.so not loadable here: {e}")


def test_footprint_of_the_stored_benchmark_plan():
    """d = 2, M = 2^20, N_t = 1000, FP32: the stored plan is dominated by the trajectory
    ([ceil((N_t+1)/4)][D][M][4] floats = 8.4 GB) plus flags, the jump log and the
    per-warp gradient partials."""
    p = workloads.double_well()
    st = footprint(p, "stored")
    rc = footprint(p, "recompute")
    traj = ((p.Nt + 4) // 4) * 2 * p.M * 4 * 4
    partG = p.Nt * 1 * (p.M // 128 * 4) * 8
    assert traj < st < traj + partG + 1.2e9
    assert rc < st - traj + 0.3e9          # checkpoints are small
    assert 8.0e9 < st < 10.0e9


def test_footprint_scales_with_paths_and_steps():
    p = workloads.double_well(M=1 << 16, Nt=400)
    a = footprint(p, "stored")
    b = footprint(p.replace(M=1 << 17), "stored")
    c = footprint(p.replace(Nt=800), "stored")
    # states grow with M and N_t; the jump log grows with M only (its capacity follows
    # lambda T, not N_t)
    assert 1.95 < b / a < 2.05 and 1.7 < c / a < 2.0
    # FP64 doubles the state storage
    assert footprint(p, "stored", prec="fp64") > 1.8 * a


def test_footprint_errors():
    p32 = workloads.linear_family(32, M=4096, Nt=50)
    assert footprint(p32, "stored") > 32 * 4 * 4096 * 51
    with pytest.raises(JdError):
        footprint(p32, "recompute")           # no recompute adjoint for d > 8
    with pytest.raises(JdError):
        footprint(workloads.double_well(M=1024, Nt=10), "auto")
    bad = workloads.double_well(M=1024, Nt=10)
    bad.sigma = np.array([np.nan, 0.3])
    with pytest.raises(JdError):
        footprint(bad, "stored")


def test_request_stream():
    reqs = workloads.serving_requests(n=4000, rate=200.0)
    t = np.array([a for a, _ in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 200.0) < 4 * (1 / 200.0) / math.sqrt(len(gaps))
    ds = np.array([p.d for _, p in reqs])
    assert set(ds) == {1, 2, 8, 32}
    for d in (1, 2, 8, 32):
        assert abs(np.mean(ds == d) - 0.25) < 0.03
    lm = np.log2([p.M for _, p in reqs])
    assert lm.min() >= 12 - 1e-9 and lm.max() <= 22 + 1e-9 and abs(lm.mean() - 17) < 0.2
    nt = np.array([p.Nt for _, p in reqs])
    assert nt.min() >= 50 and nt.max() <= 2000
    lam = np.array([p.lam for _, p in reqs])
    assert lam.min() >= 0.5 and lam.max() <= 10.0
    assert len({p.seed for _, p in reqs}) == len(reqs)
    # the same seed gives the same stream
    a1, a2 = workloads.serving_requests(n=100), workloads.serving_requests(n=100)
    assert all(a == b and p.M == q.M and p.Nt == q.Nt and p.lam == q.lam and p.d == q.d
               for (a, p), (b, q) in zip(a1, a2))
