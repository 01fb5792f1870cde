"""The sharded path of one problem on CPU: two gloo ranks (127.0.0.1).

Each rank takes its paths of the problem (bench.shard_range: whole units of
JD_UNIT_PATHS paths in rank order), forms its unit sums from the oracle's per-path costs
and sensitivities, and the ranks all-gather them (bench.gather_units); every rank then
combines them with the library's host combine (jd_combine_units, no GPU).  The test
checks that both ranks get the same bits as one process combining all units, and the
oracle's J and gradient of the whole problem.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

U = 16384


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    import workloads
    return workloads.lq_scalar(M=2 * U + 123, Nt=6)


def _control(p):
    import workloads
    return workloads.random_control(p, seed=11, scale=0.7)


def _oracle_units(p, u, m0, n):
    """Unit sums of paths [m0, m0 + n): per unit, the path costs and per-step
    sensitivities summed in path order."""
    import oracle
    rows = []
    for a in range(m0, m0 + n, U):
        J = 0.0
        G = np.zeros(p.Nt * p.du)
        for m in range(a, min(a + U, m0 + n)):
            r = oracle.path(p, u, m)
            J += r["cost"]
            G += r["G"].reshape(-1)
        rows.append(np.concatenate([[J], G]))
    return np.array(rows).reshape(-1, 1 + p.Nt * p.du)


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    from paper_2505_04328_gb300 import binding
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = _problem()
        u = _control(p)
        m0, n = bench.shard_range(p.M, rank, world)
        ne = 1 + p.Nt * p.du
        units = _oracle_units(p, u, m0, n)
        allu = bench.gather_units(dist, units, ne)
        J, g = binding.combine_units(p, u, allu)
        out.put((rank, m0, n, allu, J, g))
    finally:
        dist.destroy_process_group()


def test_shard_ranges_cover_the_paths_in_whole_units():
    import bench
    for M in (1, U, U + 1, 5 * U + 7, 3 * U):
        for world in (1, 2, 3, 8):
            spans = [bench.shard_range(M, r, world) for r in range(world)]
            assert sum(n for _, n in spans) == M
            pos = 0
            for m0, n in spans:
                assert m0 == pos and m0 % U == 0 or n == 0
                pos += n
            # every shard but the last one with paths holds whole units
            full = [s for s in spans if s[1]]
            assert all(n % U == 0 for _, n in full[:-1])


def test_two_shards_on_gloo_combine_to_the_whole_problem():
    from paper_2505_04328_gb300 import binding
    try:
        binding.lib()
    except (RuntimeError, OSError) as e:
        pytest.skip(f"libjd.so not loadable here: {e}")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = {}
    for _ in range(2):
        r, m0, n, allu, J, g = q.get(timeout=600)
        res[r] = (m0, n, allu, J, g)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = _problem()
    u = _control(p)
    assert res[0][:2] == (0, 2 * U) and res[1][:2] == (2 * U, 123)
    # one process combining every unit: the same bits on both ranks
    units = _oracle_units(p, u, 0, p.M)
    J1, g1 = binding.combine_units(p, u, units)
    for r in (0, 1):
        assert np.array_equal(res[r][2], units)
        assert res[r][3] == J1 and np.array_equal(res[r][4], g1)
    # and the oracle's whole-problem result
    import oracle
    Jo, go, _ = oracle.gradient(p, u, nthreads=1)
    assert abs(J1 - Jo) <= 1e-12 * abs(Jo)
    assert np.linalg.norm(g1 - go) <= 1e-12 * np.linalg.norm(go)
