"""C-ABI checks that need no GPU: the library loads, exports every function that
include/jd.h declares, the ctypes mirror of jd_problem_desc matches the C layout, and
invalid descriptors are rejected before any CUDA call."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import workloads
from paper_2505_04328_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "jd.h")


@pytest.fixture(scope="module")
def jdlib():
    import paper_2505_04328_gb300 as pkg
    pkg.build()
    return binding.lib()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(jd_[a-z_]+)\s*\(", text)))


def test_header_declarations_match_binding_list():
    assert _declared_functions() == sorted(binding.ABI_SYMBOLS)


def test_library_exports_every_declared_symbol(jdlib):
    out = subprocess.run(["nm", "-D", "--defined-only", binding.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    for name in _declared_functions():
        assert name in exported, name
        assert hasattr(jdlib, name)


def test_desc_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    fields = [f[0] for f in binding.ProblemDesc._fields_]
    cname = {"lam": "lambda"}
    body = "\n".join(f'  printf("{f} %zu\\n", offsetof(jd_problem_desc, {cname.get(f, f)}));' for f in fields)
    src.write_text(f"""#include <stdio.h>
#include <stddef.h>
#include "jd.h"
int main(void) {{
  printf("size %zu\\n", sizeof(jd_problem_desc));
  printf("opt %zu %zu\\n", sizeof(jd_opt_params), sizeof(jd_opt_result));
{body}
  return 0;
}}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    vals = dict((ln.split()[0], ln.split()[1:]) for ln in lines if ln)
    assert int(vals["size"][0]) == ctypes.sizeof(binding.ProblemDesc)
    assert int(vals["opt"][0]) == ctypes.sizeof(binding.OptParams)
    assert int(vals["opt"][1]) == ctypes.sizeof(binding.OptResult)
    for f in fields:
        assert int(vals[f][0]) == getattr(binding.ProblemDesc, f).offset, f


def test_feedback_desc_layout_matches_c(tmp_path):
    src = tmp_path / "fb_layout.c"
    fields = [f[0] for f in binding.FeedbackDesc._fields_]
    body = "\n".join(f'  printf("{f} %zu\\n", offsetof(jd_feedback_desc, {f}));' for f in fields)
    src.write_text(f"""#include <stdio.h>
#include <stddef.h>
#include "jd.h"
int main(void) {{
  printf("size %zu\\n", sizeof(jd_feedback_desc));
{body}
  return 0;
}}
""")
    exe = tmp_path / "fb_layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    vals = dict((ln.split()[0], ln.split()[1:]) for ln in lines if ln)
    assert int(vals["size"][0]) == ctypes.sizeof(binding.FeedbackDesc)
    for f in fields:
        assert int(vals[f][0]) == getattr(binding.FeedbackDesc, f).offset, f


def _create(desc):
    h = ctypes.c_void_p()
    st = binding.lib().jd_problem_create(ctypes.byref(desc), ctypes.byref(h))
    return st, h


def _desc(**over):
    p = workloads.double_well(M=256, Nt=16)
    keep = []

    def arr(a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        keep.append(a)
        return a.ctypes.data_as(ctypes.c_void_p)

    kw = dict(d=2, du=1, T=2.0, Nt=16, M=256, drift=1, A=arr(p.A), C=arr(p.C), B=arr(p.B), dA=None,
              sigma=arr(p.sigma), lam=5.0, jump_law=2, jump_scale=0.2, x0=arr(p.x0), q=arr(p.q),
              xd=arr(p.xd), nu=1e-3, u_min=-5.0, u_max=5.0, seed=0, epoch=0, prec=0, mode=0,
              use_tensor_cores=0, mem_budget_bytes=0, cuda_stream=None)
    kw.update(over)
    d = binding.ProblemDesc(**kw)
    d._keep = keep
    return d


@pytest.mark.parametrize("over,status", [
    (dict(d=0), binding.JD_ERR_INVALID_ARG),
    (dict(du=0), binding.JD_ERR_INVALID_ARG),
    (dict(d=40), binding.JD_ERR_UNSUPPORTED),
    (dict(du=5), binding.JD_ERR_UNSUPPORTED),
    (dict(Nt=0), binding.JD_ERR_INVALID_ARG),
    (dict(M=0), binding.JD_ERR_INVALID_ARG),
    (dict(M=1 << 33), binding.JD_ERR_INVALID_ARG),
    (dict(T=-1.0), binding.JD_ERR_INVALID_ARG),
    (dict(T=float("nan")), binding.JD_ERR_INVALID_ARG),
    (dict(lam=-1.0), binding.JD_ERR_INVALID_ARG),
    (dict(jump_law=7), binding.JD_ERR_INVALID_ARG),
    (dict(jump_law=3, jump_gain=float("nan")), binding.JD_ERR_INVALID_ARG),
    (dict(d=16, drift=0, jump_law=3, jump_gain=0.5), binding.JD_ERR_UNSUPPORTED),
    (dict(drift=3), binding.JD_ERR_INVALID_ARG),
    (dict(u_min=1.0, u_max=0.0), binding.JD_ERR_INVALID_ARG),
    (dict(C=None), binding.JD_ERR_INVALID_ARG),
    (dict(sigma=None), binding.JD_ERR_INVALID_ARG),
    (dict(prec=4), binding.JD_ERR_INVALID_ARG),
    (dict(use_tensor_cores=1), binding.JD_ERR_UNSUPPORTED),
    (dict(use_tensor_cores=4), binding.JD_ERR_INVALID_ARG),
])
def test_invalid_descriptors_rejected_before_cuda(jdlib, over, status):
    st, h = _create(_desc(**over))
    assert st == status
    assert not h.value
    assert binding.lib().jd_last_error().decode()


def test_nonfinite_coefficient_rejected(jdlib):
    A = np.array([[1.0, np.nan], [0.0, -0.5]])
    d = _desc(A=A.ctypes.data_as(ctypes.c_void_p))
    d._keep.append(A)
    st, _ = _create(d)
    assert st == binding.JD_ERR_INVALID_ARG


def test_status_strings(jdlib):
    for s in range(9):
        assert binding.lib().jd_status_string(s).decode()
    assert binding.lib().jd_status_string(99).decode() == "unknown status"


def test_null_arguments(jdlib):
    L = binding.lib()
    J = ctypes.c_double()
    assert L.jd_problem_create(None, None) == binding.JD_ERR_INVALID_ARG
    assert L.jd_cost(None, None, 0, ctypes.byref(J)) == binding.JD_ERR_INVALID_ARG
    assert L.jd_gradient(None, None, 0, None, None, 0, None) == binding.JD_ERR_INVALID_ARG
    assert L.jd_problem_destroy(None) == binding.JD_OK
