"""GPU parity of the d = 32 linear-drift path (128-path tiles; CUDA cores or tcgen05).

* use_tensor_cores = 0 (FP32 on the CUDA cores) meets the FP32 bars of the generic path:
  pathwise <= 1e-5, J and grad relative L2 <= 1e-5.
* use_tensor_cores = 1 (BF16 inputs, FP32 accumulation): the drift sees 8-bit mantissas
  (unit roundoff u = 2^-9), so each step's drift carries a relative error ~u and the
  state drifts by about T |A| u |x| ~ 4e-3 over the horizon: the stated bounds are
  pathwise <= 1e-2, J and gradient relative L2 <= 1e-2 (measured values are printed).
* use_tensor_cores = 2 (BF16 high + low parts, three products, ~16 mantissa bits):
  pathwise <= 2e-5, gradient relative L2 <= 5e-5.
* use_tensor_cores = 3 (the forward of 0, the adjoint of 2): the states of 0 bit for bit,
  the adjoint and gradient within the bounds of 2.
Steps with jumps run on the CUDA cores in every mode.
"""
import numpy as np
import pytest

import oracle
import workloads
from paper_2505_04328_gb300 import JdProblem, build

pytestmark = pytest.mark.gpu

BOUNDS = {0: (1e-5, 1e-5), 1: (1e-2, 1e-2), 2: (2e-5, 5e-5), 3: (2e-5, 5e-5)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def rel_err(a, b):
    rms = np.sqrt(np.mean(b.reshape(b.shape[0], -1) ** 2, axis=1)).reshape((-1,) + (1,) * (b.ndim - 1))
    den = np.maximum(np.abs(b), rms)
    return float(np.max(np.abs(a - b) / np.where(den == 0, 1.0, den)))


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = {
    "linear32": lambda: workloads.linear_family(32, M=300, Nt=61, lam=1.0),
    "linear16": lambda: workloads.linear_family(16, M=200, Nt=40, lam=2.0),
    "linear32_jumpy": lambda: workloads.linear_family(32, M=130, Nt=20, lam=60.0),
    # uniform jump sizes (2 u - 1 per word) through the warp-wide one-jump steps
    "linear32_uniform": lambda: workloads.linear_family(32, M=160, Nt=30, lam=20.0).replace(
        jump_law=workloads.JUMP_UNIFORM, jump_scale=0.2),
}


@pytest.mark.parametrize("tc", [0, 1, 2, 3])
@pytest.mark.parametrize("case", sorted(CASES))
def test_d32_paths_and_gradient(case, tc):
    p = CASES[case]()
    u = workloads.random_control(p, seed=21, scale=0.5)
    path_tol, grad_tol = BOUNDS[tc]
    ms = sorted(set([0, 1, 57, p.M // 2, p.M - 1]))
    rs = [oracle.path(p, u, m) for m in ms]
    Xo = np.stack([r["X"] for r in rs])
    Lo = np.stack([r["lam"] for r in rs])
    Jo, go, _ = oracle.gradient(p, u)
    with JdProblem(p, prec="fp32", use_tensor_cores=tc) as jp:
        X, L, _ = jp.sample_paths(u, 0, p.M)
        J, g, _ = jp.gradient(u)
        Jc = jp.cost(u)
        assert jp.info()["mode"] == "stored"
    ex, el = rel_err(X[ms], Xo), rel_err(L[ms], Lo)
    eg = rel_l2(g, go)
    print(f"{case} tc={tc}: pathwise X {ex:.2e} lambda {el:.2e}; J {abs(J - Jo) / abs(Jo):.2e}; "
          f"grad relL2 {eg:.2e}")
    assert ex <= path_tol and el <= path_tol
    assert abs(J - Jo) <= grad_tol * abs(Jo) and abs(Jc - J) <= 1e-6 * abs(J)
    assert eg <= grad_tol


@pytest.mark.parametrize("tc", [0, 2])
def test_d32_full_size_sampled_paths(tc):
    """The d = 32 workload at full size (M = 2^18, Nt = 500): sampled paths at both ends
    of the range against the oracle, and a finite gradient."""
    p = workloads.linear32()
    u = workloads.random_control(p, seed=22, scale=0.5)
    ms = [0, 4097, p.M - 1]
    with JdProblem(p, prec="fp32", use_tensor_cores=tc) as jp:
        for m in ms:
            r = oracle.path(p, u, m)
            X, L, c = jp.sample_paths(u, m, 1)
            assert rel_err(X, r["X"][None]) <= BOUNDS[tc][0]
            assert rel_err(L, r["lam"][None]) <= BOUNDS[tc][0]
        J, g, _ = jp.gradient(u)
    assert np.isfinite(J) and np.all(np.isfinite(g))


def test_d32_rejects_unbuilt_combinations():
    from paper_2505_04328_gb300 import JdError
    p = workloads.linear_family(32, M=256, Nt=10)
    with pytest.raises(JdError):
        JdProblem(p, prec="fp64")
    with JdProblem(p, mode="recompute") as jp:
        with pytest.raises(JdError):
            jp.gradient(workloads.random_control(p))
    with JdProblem(p) as jp:
        with pytest.raises(JdError):
            jp.gradient(workloads.random_control(p), theta=True)


@pytest.mark.parametrize("tc", [0, 1])
def test_d32_block_wise_stored_plan_is_bitwise_equal(tc):
    """A memory budget below the full stored plan makes the d = 32 problem store its
    paths block by block (multiples of 128 paths, the last block ragged); J, the gradient
    and an optimizer run are bitwise equal to the single-block plan."""
    from paper_2505_04328_gb300 import footprint
    p = workloads.linear_family(32, M=1000, Nt=40, lam=3.0)
    u = workloads.random_control(p, seed=23, scale=0.5)
    full = footprint(p, "stored")
    out = []
    for budget in (0, int(full * 0.55), int(full * 0.2)):
        with JdProblem(p, prec="fp32", use_tensor_cores=tc, mem_budget=budget) as jp:
            J, g, _ = jp.gradient(u)
            info = jp.info()
            ub, r, hist = jp.optimize(np.zeros((p.Nt, p.du)), max_iter=3, tol_rel_grad=0.0)
            if budget:
                assert info["device_bytes"] <= budget < full
            out.append((J, g, ub, r["J"], hist))
    for J, g, ub, Jr, hist in out[1:]:
        assert J == out[0][0] and np.array_equal(g, out[0][1])
        assert np.array_equal(ub, out[0][2]) and Jr == out[0][3] and np.array_equal(hist, out[0][4])


def test_d32_adjoint_only_mode_keeps_the_cuda_core_forward():
    """Mode 3 runs the CUDA-core forward of mode 0: states, per-path costs and J bit for
    bit (its BF16 x3 adjoint is checked against the oracle above)."""
    p = CASES["linear32"]()
    u = workloads.random_control(p, seed=22, scale=0.5)
    out = {}
    for tc in (0, 3):
        with JdProblem(p, prec="fp32", use_tensor_cores=tc) as jp:
            X, _, c = jp.sample_paths(u, 0, p.M, lam=False)
            J, g, _ = jp.gradient(u)
        out[tc] = (X, c, J, g)
    assert np.array_equal(out[3][0], out[0][0]) and np.array_equal(out[3][1], out[0][1])
    assert out[3][2] == out[0][2]
