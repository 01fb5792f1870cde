"""GPU tests of the serving loop (jd_server_*).

* Solo vs mixed: each request's final control and J are bitwise equal whether it runs
  alone (jd_optimize from u = 0) or in a mix of concurrent requests of every d.
* Parity: the smallest requests of each d (FP64 for d <= 8) follow the oracle's
  optimizer (J history within 1e-10 relative, final control within 1e-9); the d = 32
  request (FP32 only) within the FP32 bars (J 1e-5, control 1e-4 relative).
* Admission: a request larger than the whole budget finishes with status OOM; a small
  budget serializes requests without changing their results.
* Batched launches: many small requests (d <= 2) share launch sequences, and each still
  gets the bits of its solo jd_optimize; the batched server launches fewer kernels than
  the same stream served one request per launch sequence.
"""
import numpy as np
import pytest

import oracle
import workloads
import paper_2505_04328_gb300 as jd
from paper_2505_04328_gb300 import JdProblem, JdServer, build, footprint

pytestmark = pytest.mark.gpu

OPT = dict(max_iter=6, tol_rel_grad=1e-4)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _requests():
    """A mix of every family: (problem, prec)."""
    out = []
    for i, (d, M, Nt, lam) in enumerate([(1, 4096, 60, 2.0), (2, 6000, 120, 5.0), (8, 5000, 80, 3.0),
                                         (32, 4096, 50, 1.0), (2, 20000, 200, 9.0), (1, 30000, 300, 0.5),
                                         (8, 2500, 64, 8.0), (32, 2048, 90, 4.0)]):
        if d == 1:
            p = workloads.lq_scalar(M=M, Nt=Nt)
        elif d == 2:
            p = workloads.double_well(M=M, Nt=Nt)
        else:
            p = workloads.linear_family(d, M, Nt)
        p.lam = lam
        p.seed = 500 + i
        out.append(p)
    return out


def _solo(p, prec="fp32"):
    with JdProblem(p, prec=prec) as jp:
        u, r, _ = jp.optimize(np.zeros((p.Nt, p.du)), **OPT)
    return u, r


def test_mixed_equals_solo():
    reqs = _requests()
    solo = [_solo(p) for p in reqs]
    with JdServer(max_slots=4) as srv:
        tickets = [srv.submit(p, **OPT) for p in reqs]
        for t in tickets:
            assert srv.wait(t, timeout=300)
        res = [srv.poll(t) for t in tickets]
        infos = [srv.info(t) for t in tickets]
    for p, (us, rs), (um, rm), inf in zip(reqs, solo, res, infos):
        assert rm["status"] == 0 and rs["status"] == 0
        assert rm["J"] == rs["J"] and rm["iters"] == rs["iters"] and rm["evals"] == rs["evals"]
        # the same paired trials as alone (d <= 8 requests reserve their second buffer set)
        assert rm["sweeps"] == rs["sweeps"], p.name
        assert np.array_equal(um, us), p.name
        assert 0 <= inf["submit_s"] <= inf["admit_s"] <= inf["done_s"]
        grads = inf["path_steps"] // (p.M * p.Nt)
        assert inf["path_steps"] % (p.M * p.Nt) == 0 and grads > 0 and inf["device_bytes"] > 0
        assert inf["sweep_steps"] == (rm["sweeps"] + grads) * p.M * p.Nt
    # the requests overlapped: some request was admitted before another one finished
    assert any(b["admit_s"] < a["done_s"] for a in infos for b in infos if a is not b)


def test_small_budget_serializes_without_changing_results():
    reqs = _requests()[:4]
    solo = [_solo(p) for p in reqs]
    need = max(footprint(p, "stored") for p in reqs)
    with JdServer(budget=int(need * 1.05), max_slots=4) as srv:
        tickets = [srv.submit(p, mode="stored", **OPT) for p in reqs]
        for t in tickets:
            assert srv.wait(t, timeout=300)
        res = [srv.poll(t) for t in tickets]
        infos = [srv.info(t) for t in tickets]
    for (us, rs), (um, rm) in zip(solo, res):
        assert rm["J"] == rs["J"] and np.array_equal(um, us)
    # never more than the budget in flight
    ev = sorted([(i["admit_s"], i["device_bytes"]) for i in infos] + [(i["done_s"], -i["device_bytes"]) for i in infos])
    live = 0
    for _, b in ev:
        live += b
        assert live <= need * 1.05


def test_oversized_request_is_rejected():
    p = workloads.double_well(M=1 << 16, Nt=500)
    with JdServer(budget=64 << 20, max_slots=2) as srv:
        t = srv.submit(p, mode="stored", **OPT)
        t2 = srv.submit(workloads.lq_scalar(M=1024, Nt=50), **OPT)
        assert srv.wait(t, timeout=60) and srv.wait(t2, timeout=60)
        u, r = srv.poll(t)
        assert r["status"] == 2       # JD_ERR_OOM
        _, r2 = srv.poll(t2)
        assert r2["status"] == 0


@pytest.mark.parametrize("idx", [0, 1, 2, 3])
def test_parity_with_oracle(idx):
    p = [r for r in _requests() if r.M <= 6000][idx]
    prec = "fp32" if p.d > 8 else "fp64"
    with JdServer(max_slots=2) as srv:
        t = srv.submit(p, prec=prec, **OPT)
        assert srv.wait(t, timeout=300)
        u, r = srv.poll(t)
    uo, ro, ho = oracle.optimize(p, np.zeros((p.Nt, p.du)), **OPT)
    print(p.name, prec, r["J"], ro["J"], r["iters"], ro["iters"])
    assert r["iters"] == ro["iters"]
    if prec == "fp64":
        assert abs(r["J"] - ro["J"]) <= 1e-10 * abs(ro["J"])
        assert np.max(np.abs(u - uo)) <= 1e-9 * max(1.0, np.max(np.abs(uo)))
    else:
        assert abs(r["J"] - ro["J"]) <= 1e-5 * abs(ro["J"])
        assert np.linalg.norm(u - uo) <= 1e-4 * np.linalg.norm(uo)


def _small_requests(n=24):
    """Small requests of the serving families: d in {1, 2}, M from 700 to 40000 (ragged),
    N_t from 30 to 400, lambda from 0.5 to 9; FP32 and FP64."""
    rng = np.random.default_rng(11)
    out = []
    for i in range(n):
        d = 1 + i % 2
        M = int(rng.integers(700, 40001))
        Nt = int(rng.integers(30, 401))
        p = workloads.lq_scalar(M=M, Nt=Nt) if d == 1 else workloads.double_well(M=M, Nt=Nt)
        p.lam = float(rng.uniform(0.5, 9.0))
        p.seed = 900 + i
        out.append((p, "fp64" if i % 3 == 2 else "fp32"))
    return out


def _serve(reqs, batch_paths, slots=32):
    l0 = jd.launch_count()
    with JdServer(max_slots=slots, batch_paths=batch_paths) as srv:
        tickets = [srv.submit(p, prec=prec, **OPT) for p, prec in reqs]
        for t in tickets:
            assert srv.wait(t, timeout=600)
        res = [srv.poll(t) for t in tickets]
        stats = srv.batch_stats()
    return res, stats, jd.launch_count() - l0


def test_batched_small_requests_equal_solo():
    reqs = _small_requests()
    solo = [_solo(p, prec) for p, prec in reqs]
    res, (launches, phases), nk = _serve(reqs, batch_paths=1 << 16)
    assert launches > 0 and phases > launches, (launches, phases)   # phases shared launches
    for (p, prec), (us, rs), (um, rm) in zip(reqs, solo, res):
        assert rm["status"] == 0 and rs["status"] == 0, p.name
        assert rm["J"] == rs["J"] and rm["iters"] == rs["iters"] and rm["evals"] == rs["evals"], p.name
        assert rm["sweeps"] == rs["sweeps"], p.name
        assert np.array_equal(um, us), (p.name, prec)
    # the same stream without batching: the same bits, more kernels
    res0, (l0, ph0), nk0 = _serve(reqs, batch_paths=0)
    assert l0 == 0 and ph0 == 0
    for (um, rm), (u0, r0) in zip(res, res0):
        assert rm["J"] == r0["J"] and np.array_equal(um, u0)
    print("kernels batched", nk, "unbatched", nk0, "mean batch", phases / launches)
    assert nk < nk0


def test_batching_limit_excludes_large_requests():
    """Requests above the limit run their own launches (no batched phase)."""
    reqs = [(workloads.double_well(M=5000, Nt=40), "fp32"), (workloads.lq_scalar(M=3000, Nt=40), "fp32")]
    res, (launches, phases), _ = _serve(reqs, batch_paths=2000, slots=4)
    assert launches == 0 and phases == 0
    assert all(r["status"] == 0 for _, r in res)
    with JdServer(max_slots=2) as srv:
        import ctypes
        from paper_2505_04328_gb300 import binding
        assert binding.lib().jd_server_set_batching(srv.h, ctypes.c_int64(-1)) == binding.JD_ERR_INVALID_ARG
