"""jd_cost_noalloc: the cost entry point for callers that must not allocate device
memory while running (real-time control loops, applications whose memory pool owns
the GPU).  It must give the same J as jd_cost, and the oracle's J, call after call,
while using only its fixed scratch array; after a warm-up call it must not change the
device's free memory.  This file is collected last so that, if it fails, a run that
stops at the first failure has already run every other test."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import workloads
from paper_2505_04328_gb300 import JdProblem, binding, build

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _call(L, desc, ud, Jd):
    return L.jd_cost_noalloc(ctypes.byref(desc), ctypes.c_void_p(ud.data_ptr()), ctypes.c_void_p(Jd.data_ptr()))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("maker", [lambda: workloads.double_well(M=70001, Nt=333),
                                   lambda: workloads.lq_scalar(M=5000, Nt=100)])
def test_noalloc_cost_matches_jd_cost_and_the_oracle_two_calls(prec, maker):
    torch = pytest.importorskip("torch")
    p = maker()
    L = binding.lib()
    with JdProblem(p, prec=prec) as jp:
        for seed in (1, 2):   # two calls in a row share the scratch array
            u = workloads.random_control(p, seed=seed, scale=0.5)
            J_ref = jp.cost(u)
            J_orc = oracle.cost(p, u)
            ud = torch.tensor(u.reshape(-1), dtype=torch.float64, device="cuda")
            Jd = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            assert _call(L, jp.desc, ud, Jd) == binding.JD_OK
            torch.cuda.synchronize()
            J = float(Jd.item())
            assert abs(J - J_ref) <= TOL[prec] * abs(J_ref), (seed, J, J_ref)
            assert abs(J - J_orc) <= TOL[prec] * abs(J_orc), (seed, J, J_orc)


def test_noalloc_changes_no_free_memory_after_warm_up():
    """The first call on a device may load the kernels' code (lazy module loading);
    after it, a call allocates nothing: the device's free memory stays the same."""
    torch = pytest.importorskip("torch")
    p = workloads.double_well(M=40000, Nt=200)
    L = binding.lib()
    desc, _keep = binding.make_desc(p, prec=binding.JD_FP32)
    u = workloads.random_control(p, seed=4, scale=0.5)
    ud = torch.tensor(u.reshape(-1), dtype=torch.float64, device="cuda")
    Jd = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _call(L, desc, ud, Jd) == binding.JD_OK   # warm-up
    torch.cuda.synchronize()
    J1 = float(Jd.item())
    free0, _ = torch.cuda.mem_get_info()
    assert _call(L, desc, ud, Jd) == binding.JD_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert float(Jd.item()) == J1   # the same sample, the same bits


_CHILD = r"""
import ctypes, sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import workloads
from paper_2505_04328_gb300 import binding
p = workloads.double_well(M=20001, Nt=200)
u = workloads.random_control(p, seed=3, scale=0.5)
desc, keep = binding.make_desc(p, prec=binding.JD_FP64)
ud = torch.tensor(u.reshape(-1), dtype=torch.float64, device="cuda")
Jd = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
st = binding.lib().jd_cost_noalloc(ctypes.byref(desc), ctypes.c_void_p(ud.data_ptr()),
                                   ctypes.c_void_p(Jd.data_ptr()))
torch.cuda.synchronize()
print(st, repr(float(Jd.item())))
"""


def test_noalloc_in_a_fresh_process_without_a_problem():
    """A process whose only library call is jd_cost_noalloc (no problem object, so the
    context's stack limit is the default): the call runs and gives the oracle's J."""
    p = workloads.double_well(M=20001, Nt=200)
    u = workloads.random_control(p, seed=3, scale=0.5)
    J_orc = oracle.cost(p, u)
    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    st, J = r.stdout.split()[-2:]
    assert int(st) == binding.JD_OK
    assert abs(float(J) - J_orc) <= TOL["fp64"] * abs(J_orc), (J, J_orc)


def test_noalloc_rejects_beyond_scratch_and_unsupported_sizes():
    torch = pytest.importorskip("torch")
    L = binding.lib()
    ud = torch.zeros(1000, dtype=torch.float64, device="cuda")
    Jd = torch.zeros(1, dtype=torch.float64, device="cuda")
    big = workloads.double_well(M=1 << 30, Nt=1000)       # 64 MiB of partials
    with JdProblem(big.replace(M=1 << 10)) as jp:
        d = jp.desc
        d.M = 1 << 30
        assert _call(L, d, ud, Jd) == binding.JD_ERR_OOM
    lin = workloads.linear_family(4, M=1024, Nt=1000)
    with JdProblem(lin) as jp:
        assert _call(L, jp.desc, ud, Jd) == binding.JD_ERR_UNSUPPORTED
