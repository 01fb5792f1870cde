"""jd_cost_noalloc: the cost entry point for callers that must not allocate device
memory while running (real-time control loops, applications whose memory pool owns
the GPU).  It must give the same J as jd_cost, call after call, while using only its
fixed scratch array.  This file is collected last so that, if it fails, a run that
stops at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import workloads
from paper_2505_04328_gb300 import JdProblem, binding, build

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("maker", [lambda: workloads.double_well(M=70001, Nt=333),
                                   lambda: workloads.lq_scalar(M=5000, Nt=100)])
def test_noalloc_cost_matches_jd_cost_two_calls(prec, maker):
    torch = pytest.importorskip("torch")
    p = maker()
    L = binding.lib()
    with JdProblem(p, prec=prec) as jp:
        for seed in (1, 2):   # two calls in a row share the scratch array
            u = workloads.random_control(p, seed=seed, scale=0.5)
            J_ref = jp.cost(u)
            ud = torch.tensor(u.reshape(-1), dtype=torch.float64, device="cuda")
            Jd = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            st = L.jd_cost_noalloc(ctypes.byref(jp.desc), ctypes.c_void_p(ud.data_ptr()),
                                   ctypes.c_void_p(Jd.data_ptr()))
            assert st == binding.JD_OK
            torch.cuda.synchronize()
            J = float(Jd.item())
            assert abs(J - J_ref) <= TOL[prec] * abs(J_ref), (seed, J, J_ref)


def test_noalloc_rejects_beyond_scratch_and_unsupported_sizes():
    torch = pytest.importorskip("torch")
    L = binding.lib()
    ud = torch.zeros(1000, dtype=torch.float64, device="cuda")
    Jd = torch.zeros(1, dtype=torch.float64, device="cuda")
    big = workloads.double_well(M=1 << 30, Nt=1000)       # 64 MiB of partials
    with JdProblem(big.replace(M=1 << 10)) as jp:
        d = jp.desc
        d.M = 1 << 30
        assert L.jd_cost_noalloc(ctypes.byref(d), ctypes.c_void_p(ud.data_ptr()),
                                 ctypes.c_void_p(Jd.data_ptr())) == binding.JD_ERR_OOM
    lin = workloads.linear_family(4, M=1024, Nt=1000)
    with JdProblem(lin) as jp:
        assert L.jd_cost_noalloc(ctypes.byref(jp.desc), ctypes.c_void_p(ud.data_ptr()),
                                 ctypes.c_void_p(Jd.data_ptr())) == binding.JD_ERR_UNSUPPORTED
