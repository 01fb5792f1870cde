"""Checkpoint spacing of the recompute adjoint chosen from the memory budget: 16 steps
when the checkpoints fit, else 32 or 64 (S ~ sqrt(N_t) for N_t near 4096).  Whatever the
spacing, the recompute plan replays the same steps with the same arithmetic: J, the
gradient and the parameter gradients equal the stored plan's bit for bit."""
import numpy as np
import pytest

import workloads
from paper_2505_04328_gb300 import JdError, JdProblem, build, footprint

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _ckpt(p, S, es):
    return (-(-p.Nt // S) + 1) * p.d * p.M * es


# FP64 d = 2 stops at 32: the parameter-gradient replay of 64 steps (states and normals,
# 2 x 64 x 2 x 128 doubles) would not fit a block's shared memory
@pytest.mark.parametrize("prec,es,S", [("fp32", 4, 16), ("fp32", 4, 32), ("fp32", 4, 64),
                                       ("fp64", 8, 16), ("fp64", 8, 32)])
def test_spacing_from_the_budget_keeps_the_stored_plans_bits(S, prec, es):
    p = workloads.double_well(M=3001, Nt=301).replace(lam=12.0)
    u = workloads.random_control(p, seed=9, scale=0.5)
    with JdProblem(p, prec=prec, mode="stored") as st:
        J0, g0, t0 = st.gradient(u, theta=True)
    base = footprint(p, "recompute", prec=prec) - _ckpt(p, 16, es)
    budget = base + _ckpt(p, S, es) + 1024   # holds spacing S, not S / 2
    with JdProblem(p, prec=prec, mode="recompute", mem_budget=budget) as rc:
        J, g, t = rc.gradient(u, theta=True)
        Jc = rc.cost(u)
        info = rc.info()
    assert info["mode"] == "recompute" and info["device_bytes"] == base + _ckpt(p, S, es)
    assert J == J0 and np.array_equal(g, g0) and np.array_equal(t, t0)
    assert Jc == J0


@pytest.mark.parametrize("prec,es,widest", [("fp32", 4, 64), ("fp64", 8, 32)])
def test_budget_below_the_widest_spacing_is_out_of_memory(prec, es, widest):
    p = workloads.double_well(M=3001, Nt=301)
    base = footprint(p, "recompute", prec=prec) - _ckpt(p, 16, es)
    with JdProblem(p, prec=prec, mode="recompute", mem_budget=base + _ckpt(p, widest, es) - 4096) as rc:
        with pytest.raises(JdError):
            rc.gradient(np.zeros((p.Nt, p.du)))
