"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1).

With several GPUs every rank solves its own replica of the workload (Philox seed offset
by the rank, no collective on the data path) and only the timing is reduced (maximum over
ranks).  Here each rank evaluates its replica with the oracle on a small sample, and the
test checks that the replicas are independent instances, that the reduced time is the
maximum, that the whole-job value counts every rank's path-steps, and that only rank 0
runs the reference arm.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import oracle
    import workloads
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        p = bench.replica_problem(workloads.double_well(M=256, Nt=40), r)
        J = oracle.cost(p, np.zeros((p.Nt, p.du)), nthreads=1)
        t = bench.max_over_ranks(dist, 10.0 + r)          # rank 1 is the slower one
        value = ws * p.M * p.Nt / (t * 1e-3)
        Js = [None] * world
        dist.all_gather_object(Js, (p.seed, J))
        # the reference arm runs on rank 0 only; other ranks return without work
        class A:
            reference_paths, steps, warmup = 64, 1, 0
        import contextlib
        import io
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            rc = bench.run_reference(A())
        out.put((r, ws, t, value, Js, rc, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_replicas_on_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r, ws, t, value, Js, rc, printed = q.get(timeout=300)
        res[r] = (ws, t, value, Js, rc, printed)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        ws, t, value, Js, rc, printed = res[r]
        assert ws == 2 and t == 11.0                      # max over ranks
        assert value == pytest.approx(2 * 256 * 40 / 11e-3)
        (s0, J0), (s1, J1) = Js
        assert s1 == s0 + 1 and J0 != J1                  # independent replicas
        assert rc == 0
    assert '"impl": "reference"' in res[0][5] and res[1][5] == ""
    # each rank's J is the single-process evaluation of its own replica
    import oracle
    import workloads
    p1 = workloads.double_well(M=256, Nt=40).replace(seed=1)
    assert res[0][3][1][1] == oracle.cost(p1, np.zeros((p1.Nt, p1.du)), nthreads=1)
