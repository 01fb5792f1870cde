"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (relative error |a - b| / max(|b|, rms over the path of b)):
  * FP32 path arithmetic: pathwise X_k, lambda_k and per-path cost <= 1e-5;
  * FP64 path arithmetic: pathwise <= 1e-12;
  * reduced gradient: relative L2 error <= GRAD_TOL_FP32 in FP32, <= 1e-12 in FP64;
  * discrete decisions (Poisson counts, jump order) are integer comparisons on the
    same 32-bit words in both implementations, so jump patterns agree exactly.
Stored and recompute adjoints run the same FP32 operations and must agree bit for bit.
"""
import numpy as np
import pytest

import oracle
import workloads
from paper_2505_04328_gb300 import JdProblem, build

pytestmark = pytest.mark.gpu

PATH_TOL_FP32 = 1e-5
PATH_TOL_FP64 = 1e-12
GRAD_TOL_FP32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def rel_err(a, b):
    """max |a-b| / max(|b|, rms of b over the path) (per path, then max)."""
    a = np.asarray(a)
    b = np.asarray(b)
    rms = np.sqrt(np.mean(b.reshape(b.shape[0], -1) ** 2, axis=1))
    den = np.maximum(np.abs(b), rms.reshape((-1,) + (1,) * (b.ndim - 1)))
    den = np.where(den == 0, 1.0, den)
    return float(np.max(np.abs(a - b) / den))


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _oracle_paths(p, u, ms):
    rs = [oracle.path(p, u, m) for m in ms]
    return (np.stack([r["X"] for r in rs]), np.stack([r["lam"] for r in rs]),
            np.array([r["cost"] for r in rs]), np.stack([r["njumps"] for r in rs]))


CASES = {
    "double_well": lambda: workloads.double_well(M=300, Nt=203),
    "double_well_phase": lambda: workloads.double_well_phase(M=300, Nt=203),
    "lq_scalar": lambda: workloads.lq_scalar(M=300, Nt=101),
    "linear3_odd": lambda: workloads.linear_family(3, M=200, Nt=77, lam=4.0),
    "linear4": lambda: workloads.linear_family(4, M=200, Nt=77, lam=4.0),
    "linear8": lambda: workloads.linear_family(8, M=200, Nt=77, lam=4.0),
    "d1_two_controls": lambda: workloads.lq_scalar(M=150, Nt=50).replace(du=2, B=np.array([[1.0, -0.5]])),
    "many_jumps": lambda: workloads.double_well(M=130, Nt=40).replace(lam=120.0),
    # Keilson-Storer velocity resets (Sec. 5.3): the paper's beta = 10, gamma = 0.9 at a
    # larger rate so that most paths see several resets; d = 4 has two velocities
    "ks_oscillator": lambda: workloads.ks_oscillator(M=300, Nt=150).replace(lam=12.0),
    "ks_linear4": lambda: workloads.linear_family(4, M=200, Nt=77, lam=6.0).replace(
        jump_law=workloads.JUMP_KS, jump_gain=0.6, jump_scale=0.3),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_pathwise_parity(case, prec):
    p = CASES[case]()
    u = workloads.random_control(p, seed=3, scale=0.7)
    ms = sorted(set(list(range(0, p.M, max(1, p.M // 23))) + [p.M - 1]))
    with JdProblem(p, prec=prec) as jp:
        X, L, c = jp.sample_paths(u, 0, p.M)
    Xo, Lo, co, nj = _oracle_paths(p, u, ms)
    tol = PATH_TOL_FP32 if prec == "fp32" else PATH_TOL_FP64
    assert nj.sum() > 0
    assert rel_err(X[ms], Xo) <= tol
    assert rel_err(L[ms], Lo) <= tol
    assert np.max(np.abs(c[ms] - co) / np.abs(co)) <= tol


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("mode", ["stored", "recompute"])
def test_cost_and_gradient_parity(case, prec, mode):
    p = CASES[case]()
    u = workloads.random_control(p, seed=4, scale=0.7)
    Jo, go, _ = oracle.gradient(p, u)
    with JdProblem(p, prec=prec, mode=mode) as jp:
        J, g, _ = jp.gradient(u)
        Jc = jp.cost(u)
        assert jp.info()["mode"] == mode
    tol = GRAD_TOL_FP32 if prec == "fp32" else 1e-12
    assert abs(J - Jo) <= tol * abs(Jo)
    assert abs(Jc - Jo) <= tol * abs(Jo)
    assert rel_l2(g, go) <= tol


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("law", ["normal", "ks"])
def test_stored_equals_recompute_bitwise(prec, law):
    if law == "normal":
        p = workloads.double_well(M=1000, Nt=333).replace(lam=20.0)
    else:
        p = workloads.ks_oscillator(M=1000, Nt=333).replace(lam=20.0)
    u = workloads.random_control(p, seed=5)
    with JdProblem(p, prec=prec, mode="stored") as a, JdProblem(p, prec=prec, mode="recompute") as b:
        Ja, ga, ta = a.gradient(u, theta=True)
        Jb, gb, tb = b.gradient(u, theta=True)
        Jc = a.cost(u)
    assert Ja == Jb
    assert np.array_equal(ga, gb)
    assert np.array_equal(ta, tb)
    # the cost and checkpoint sweeps draw with the parameter block's Philox round keys,
    # the single store sweep bumps the key per round: the same words, so the same cost
    assert Jc == Ja


def test_repeatable_bitwise():
    p = workloads.double_well(M=5000, Nt=100)
    u = workloads.random_control(p, seed=6)
    with JdProblem(p) as jp:
        r1 = jp.gradient(u)
        r2 = jp.gradient(u)
    assert r1[0] == r2[0] and np.array_equal(r1[1], r2[1])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-4)])
@pytest.mark.parametrize("law", ["uniform", "ks"])
def test_parameter_gradient_parity(prec, tol, law):
    if law == "uniform":
        p = workloads.double_well_autograd(M=600, Nt=120)
    else:   # reset law: the jump-scale derivative sums over the velocity half only
        p = workloads.ks_oscillator(M=600, Nt=120).replace(lam=10.0, dA=np.array([[0.0, 0.0], [0.0, -1.0]]))
    u = workloads.random_control(p, seed=8, scale=0.5)
    _, _, tho = oracle.gradient(p, u, theta=True)
    with JdProblem(p, prec=prec, mode="recompute") as jp:
        _, _, th = jp.gradient(u, theta=True)
    assert np.max(np.abs(th - tho) / np.maximum(np.abs(tho), 1e-3 * np.abs(tho).max())) <= tol


@pytest.mark.parametrize("over", [
    dict(M=1, Nt=1), dict(M=1, Nt=9), dict(M=129, Nt=1), dict(lam=0.0),
    dict(jump_law=workloads.JUMP_NONE), dict(M=37, Nt=31), dict(sigma=np.zeros(2))])
def test_edge_cases(over):
    p = workloads.double_well(M=257, Nt=65).replace(**over)
    u = workloads.random_control(p, seed=9)
    Jo, go, _ = oracle.gradient(p, u)
    for prec, tol in (("fp32", GRAD_TOL_FP32), ("fp64", 1e-12)):
        for mode in ("stored", "recompute"):
            with JdProblem(p, prec=prec, mode=mode) as jp:
                J, g, _ = jp.gradient(u)
            assert abs(J - Jo) <= tol * abs(Jo), (prec, mode)
            assert rel_l2(g, go) <= tol, (prec, mode)


def test_full_size_double_well_sampled_paths():
    """The benchmark's workload (d=2, M=2^20, Nt=1000): paths at both ends of the
    range against the oracle, and stored == recompute at full size."""
    p = workloads.double_well()
    u = workloads.random_control(p, seed=10, scale=0.5)
    ms = [0, 1, 777, p.M // 2 + 3, p.M - 2, p.M - 1]
    Xo, Lo, co, _ = _oracle_paths(p, u, ms)
    with JdProblem(p, prec="fp32", mode="stored") as jp:
        for m, xo, lo, c in zip(ms, Xo, Lo, co):
            X, L, cc = jp.sample_paths(u, m, 1)
            assert rel_err(X, xo[None]) <= PATH_TOL_FP32
            assert rel_err(L, lo[None]) <= PATH_TOL_FP32
            assert abs(cc[0] - c) <= PATH_TOL_FP32 * abs(c)
        Js, gs, _ = jp.gradient(u)
    with JdProblem(p, prec="fp32", mode="recompute") as jp:
        Jr, gr, _ = jp.gradient(u)
    assert Js == Jr and np.array_equal(gs, gr)
    assert np.all(np.isfinite(gs)) and Js > 0


def test_device_tensor_gradient_matches_host():
    torch = pytest.importorskip("torch")
    p = workloads.double_well(M=2000, Nt=64)
    u = workloads.random_control(p, seed=12)
    with JdProblem(p) as jp:
        J, g, _ = jp.gradient(u)
        ud = torch.tensor(u, dtype=torch.float64, device="cuda").reshape(-1)
        gd = torch.empty_like(ud)
        J2, _ = jp.gradient_into(ud, gd)
        torch.cuda.synchronize()
    assert J2 == J
    assert np.array_equal(gd.cpu().numpy().reshape(g.shape), g)
