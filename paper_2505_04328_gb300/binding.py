"""ctypes binding of the C ABI in include/jd.h (argument marshalling only).

Every numeric step runs in libjd.so's CUDA kernels; this module only converts numpy
arrays / torch tensors into pointers and sizes.  There is no CPU fallback: if the
library is missing or cannot be loaded, the first call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libjd.so")
_lib = None
_lock = threading.Lock()

JD_OK, JD_ERR_INVALID_ARG, JD_ERR_OOM, JD_ERR_CUDA, JD_ERR_NONFINITE = 0, 1, 2, 3, 4
JD_ERR_LINESEARCH, JD_ERR_TIMEOUT, JD_ERR_UNSUPPORTED, JD_ERR_BUSY = 5, 6, 7, 8
JD_FP32, JD_FP64 = 0, 1
JD_ADJ_AUTO, JD_ADJ_STORED, JD_ADJ_RECOMPUTE = 0, 1, 2
JD_MEM_HOST, JD_MEM_DEVICE = 0, 1
_CUDA_STREAM_LEGACY = 0x1   # cudaStreamLegacy

# Every function declared in include/jd.h.
ABI_SYMBOLS = (
    "jd_problem_create", "jd_problem_destroy", "jd_cost", "jd_gradient", "jd_sample_paths",
    "jd_forward", "jd_backward", "jd_problem_update",
    "jd_optimize", "jd_problem_info", "jd_kernel_launch_count", "jd_profile_enable",
    "jd_profile_read", "jd_cost_noalloc", "jd_problem_footprint", "jd_server_create",
    "jd_server_submit", "jd_server_poll", "jd_server_wait", "jd_server_info", "jd_server_destroy",
    "jd_status_string", "jd_last_error", "jd_fb_cost", "jd_fb_gradient", "jd_fb_optimize",
    "jd_gradient_units", "jd_cost_units", "jd_combine_units", "jd_server_set_batching",
    "jd_server_batch_stats",
)

UNIT_PATHS = 16384   # JD_UNIT_PATHS: paths per unit of the path reduction (path sharding)


class JdError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        super().__init__(f"{where}: status {status} ({detail})")


class ProblemDesc(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("du", ctypes.c_int), ("T", ctypes.c_double), ("Nt", ctypes.c_int),
        ("M", ctypes.c_int64), ("drift", ctypes.c_int),
        ("A", ctypes.c_void_p), ("C", ctypes.c_void_p), ("B", ctypes.c_void_p), ("dA", ctypes.c_void_p),
        ("sigma", ctypes.c_void_p), ("lam", ctypes.c_double), ("jump_law", ctypes.c_int),
        ("jump_scale", ctypes.c_double), ("x0", ctypes.c_void_p), ("q", ctypes.c_void_p),
        ("xd", ctypes.c_void_p), ("nu", ctypes.c_double), ("u_min", ctypes.c_double),
        ("u_max", ctypes.c_double), ("seed", ctypes.c_uint64), ("epoch", ctypes.c_uint32),
        ("prec", ctypes.c_int), ("mode", ctypes.c_int), ("use_tensor_cores", ctypes.c_int),
        ("mem_budget_bytes", ctypes.c_size_t), ("cuda_stream", ctypes.c_void_p),
        ("jump_gain", ctypes.c_double), ("m_offset", ctypes.c_int64),
    ]


class FeedbackDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("nv", ctypes.c_int), ("x_max", ctypes.c_double),
                ("v_max", ctypes.c_double), ("eps", ctypes.c_double), ("track", ctypes.c_int),
                ("sigma_J", ctypes.c_double), ("adjoint", ctypes.c_int), ("sur_rate", ctypes.c_double),
                ("particles", ctypes.c_int), ("omega", ctypes.c_double), ("ax", ctypes.c_double),
                ("av", ctypes.c_double)]


def make_feedback(fb) -> FeedbackDesc:
    """The jd_feedback_desc of a workloads.Feedback (duck-typed)."""
    return FeedbackDesc(nx=int(fb.nx), nv=int(fb.nv), x_max=float(fb.x_max), v_max=float(fb.v_max),
                        eps=float(fb.eps), track=int(fb.track), sigma_J=float(fb.sigma_J),
                        adjoint=int(getattr(fb, "adjoint", 0)), sur_rate=float(getattr(fb, "sur_rate", 0.0)),
                        particles=int(getattr(fb, "particles", 0)), omega=float(getattr(fb, "omega", 0.0)),
                        ax=float(getattr(fb, "ax", 1.0)), av=float(getattr(fb, "av", 1.0)))


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double)]


class OptParams(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int), ("tol_rel_grad", ctypes.c_double),
                ("tol_step", ctypes.c_double), ("armijo_c", ctypes.c_double),
                ("zeta0", ctypes.c_double), ("zeta_max", ctypes.c_double),
                ("max_backtracks", ctypes.c_int), ("resample", ctypes.c_int),
                ("one_trial_per_sweep", ctypes.c_int)]


class OptResult(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("evals", ctypes.c_int), ("J", ctypes.c_double),
                ("rel_grad_norm", ctypes.c_double), ("zeta", ctypes.c_double),
                ("status", ctypes.c_int), ("sweeps", ctypes.c_int)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("plan", ctypes.c_int), ("done", ctypes.c_int),
                ("path_steps", ctypes.c_int64), ("sweep_steps", ctypes.c_int64)]


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Load libjd.so (built by paper_2505_04328_gb300._build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(
                f"{_LIB_PATH} is missing: build it with paper_2505_04328_gb300._build.build() "
                "(CUDA toolkit required; there is no CPU fallback)")
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER
        vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p
        L.jd_problem_create.argtypes = [P(ProblemDesc), P(ctypes.c_void_p)]
        L.jd_problem_destroy.argtypes = [vp]
        L.jd_cost.argtypes = [vp, dp, ctypes.c_int, P(ctypes.c_double)]
        L.jd_gradient.argtypes = [vp, dp, ctypes.c_int, dp, dp, ctypes.c_int, dp]
        L.jd_forward.argtypes = [vp, dp, ctypes.c_int, dp, ctypes.c_int]
        L.jd_backward.argtypes = [vp, dp, ctypes.c_int, dp]
        L.jd_problem_update.argtypes = [vp, P(ProblemDesc)]
        L.jd_sample_paths.argtypes = [vp, dp, ctypes.c_int, i64, i64, dp, dp, dp]
        L.jd_optimize.argtypes = [vp, dp, ctypes.c_int, P(OptParams), P(OptResult), dp]
        L.jd_problem_info.argtypes = [vp, P(ctypes.c_size_t), P(ctypes.c_int)]
        L.jd_cost_noalloc.argtypes = [P(ProblemDesc), dp, dp]
        L.jd_gradient_units.argtypes = [vp, dp, ctypes.c_int, dp, ctypes.c_int]
        L.jd_cost_units.argtypes = [vp, dp, ctypes.c_int, dp, ctypes.c_int]
        L.jd_combine_units.argtypes = [i64, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp,
                                       i64, ctypes.c_int, dp, dp]
        L.jd_fb_cost.argtypes = [vp, P(FeedbackDesc), dp, ctypes.c_int, dp]
        L.jd_fb_gradient.argtypes = [vp, P(FeedbackDesc), dp, ctypes.c_int, dp, dp]
        L.jd_fb_optimize.argtypes = [vp, P(FeedbackDesc), dp, ctypes.c_int, P(OptParams), P(OptResult), dp]
        L.jd_problem_footprint.argtypes = [P(ProblemDesc), ctypes.c_int, P(ctypes.c_size_t)]
        L.jd_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int, P(ctypes.c_void_p)]
        L.jd_server_submit.argtypes = [vp, P(ProblemDesc), P(OptParams), P(ctypes.c_uint64)]
        L.jd_server_poll.argtypes = [vp, ctypes.c_uint64, dp, P(OptResult)]
        L.jd_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_double]
        L.jd_server_info.argtypes = [vp, ctypes.c_uint64, P(RequestInfo)]
        L.jd_server_destroy.argtypes = [vp]
        L.jd_server_set_batching.argtypes = [vp, ctypes.c_int64]
        L.jd_server_batch_stats.argtypes = [vp, P(ctypes.c_int64), P(ctypes.c_int64)]
        L.jd_kernel_launch_count.restype = ctypes.c_uint64
        L.jd_profile_enable.argtypes = [ctypes.c_int]
        L.jd_profile_enable.restype = None
        L.jd_profile_read.argtypes = [P(KernelStat), ctypes.c_int]
        L.jd_profile_read.restype = ctypes.c_int
        L.jd_status_string.argtypes = [ctypes.c_int]
        L.jd_status_string.restype = ctypes.c_char_p
        L.jd_last_error.restype = ctypes.c_char_p
        for f in ABI_SYMBOLS:
            if f not in ("jd_kernel_launch_count", "jd_status_string", "jd_last_error",
                         "jd_profile_enable", "jd_profile_read"):
                getattr(L, f).restype = ctypes.c_int
        _lib = L
        return L


def launch_count() -> int:
    return int(lib().jd_kernel_launch_count())


def profile_enable(on: bool = True):
    """Start (clearing old records) or stop per-kernel CUDA-event timing."""
    lib().jd_profile_enable(1 if on else 0)


def profile_read():
    """{kernel class: (launches, total ms)} of the recorded launches."""
    arr = (KernelStat * 16)()
    n = lib().jd_profile_read(arr, 16)
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(n)}


def _check(status: int, where: str):
    if status != JD_OK:
        L = lib()
        raise JdError(status, where, f"{L.jd_status_string(status).decode()}: {L.jd_last_error().decode()}")


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _u_arg(u, n: int):
    """Returns (pointer, memspace, keepalive) for a control given as numpy or torch."""
    if _is_torch(u):
        import torch
        if u.dtype != torch.float64 or not u.is_contiguous() or u.numel() != n:
            raise ValueError(f"control tensor must be contiguous float64 with {n} entries")
        if u.is_cuda:
            return ctypes.c_void_p(u.data_ptr()), JD_MEM_DEVICE, u
        return ctypes.c_void_p(u.data_ptr()), JD_MEM_HOST, u
    a = _f64(u).reshape(-1)
    if a.size != n:
        raise ValueError(f"control must have {n} entries, got {a.size}")
    return _ptr(a), JD_MEM_HOST, a


_PREC = {"fp32": JD_FP32, "fp64": JD_FP64, JD_FP32: JD_FP32, JD_FP64: JD_FP64}
_MODE = {"auto": JD_ADJ_AUTO, "stored": JD_ADJ_STORED, "recompute": JD_ADJ_RECOMPUTE,
         JD_ADJ_AUTO: JD_ADJ_AUTO, JD_ADJ_STORED: JD_ADJ_STORED, JD_ADJ_RECOMPUTE: JD_ADJ_RECOMPUTE}


def make_desc(problem, prec=JD_FP32, mode=JD_ADJ_AUTO, use_tensor_cores=0, mem_budget_bytes=0,
              stream_handle=None):
    """(ProblemDesc, arrays): the descriptor of a workloads Problem and the float64
    arrays it points to (keep them alive while the descriptor is in use)."""
    d = problem.d
    C = problem.C if problem.C is not None else np.zeros((d, d))
    a = dict(
        A=_f64(problem.A).reshape(-1), C=_f64(C).reshape(-1), B=_f64(problem.B).reshape(-1),
        dA=None if problem.dA is None else _f64(problem.dA).reshape(-1),
        sigma=_f64(problem.sigma).reshape(-1), x0=_f64(problem.x0).reshape(-1),
        q=_f64(problem.q).reshape(-1), xd=_f64(problem.xd).reshape(-1))
    desc = ProblemDesc(
        d=d, du=problem.du, T=float(problem.T), Nt=problem.Nt, M=problem.M, drift=int(problem.drift),
        A=_ptr(a["A"]), C=_ptr(a["C"]), B=_ptr(a["B"]), dA=_ptr(a["dA"]), sigma=_ptr(a["sigma"]),
        lam=float(problem.lam), jump_law=int(problem.jump_law), jump_scale=float(problem.jump_scale),
        x0=_ptr(a["x0"]), q=_ptr(a["q"]), xd=_ptr(a["xd"]), nu=float(problem.nu),
        u_min=float(problem.u_min), u_max=float(problem.u_max), seed=int(problem.seed),
        epoch=int(problem.epoch), prec=_PREC[prec], mode=_MODE[mode],
        use_tensor_cores=int(use_tensor_cores), mem_budget_bytes=int(mem_budget_bytes),
        cuda_stream=stream_handle, jump_gain=float(getattr(problem, "jump_gain", 1.0)),
        m_offset=int(getattr(problem, "m_offset", 0)))
    return desc, a


def combine_units(problem, u, units, M_total=None):
    """(J, grad (Nt, du) or None) from the unit sums of all shards in path order
    (jd_combine_units: host arithmetic, the same bits as jd_gradient on the whole
    problem).  units: [ceil(M_total / UNIT_PATHS), ne] with ne = 1 (cost) or 1 + Nt du."""
    M_total = int(problem.M if M_total is None else M_total)
    units = np.ascontiguousarray(units, dtype=np.float64)
    ne = units.shape[1]
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1))
    J = ctypes.c_double()
    g = np.zeros((problem.Nt, problem.du)) if ne > 1 else None
    _check(lib().jd_combine_units(M_total, problem.Nt, problem.du, float(problem.T), float(problem.nu), _ptr(u),
                                  _ptr(units), units.shape[0], ne, ctypes.byref(J), _ptr(g)), "jd_combine_units")
    return J.value, g


def footprint(problem, plan="stored", prec="fp32") -> int:
    """Device bytes of ``problem`` under an adjoint plan (jd_problem_footprint; no GPU)."""
    desc, _keep = make_desc(problem, prec=prec)
    b = ctypes.c_size_t()
    _check(lib().jd_problem_footprint(ctypes.byref(desc), _MODE[plan], ctypes.byref(b)), "jd_problem_footprint")
    return b.value


class JdProblem:
    """One problem on the current CUDA device (see jd_problem_create).

    ``problem`` is any object with the fields of workloads.Problem (d, du, T, Nt, M,
    drift, A, C, B, dA, sigma, lam, jump_law, jump_scale, jump_gain, x0, q, xd, nu, u_min, u_max,
    seed, epoch).  ``stream``: a torch.cuda.Stream, a raw cudaStream_t int, or None for
    torch's current stream (a library-owned stream when torch has no CUDA).
    ``use_tensor_cores`` (8 < d <= 32): 0 CUDA cores, 1 BF16 tensor cores, 2 BF16 x3,
    3 CUDA-core forward with the BF16 x3 tensor-core adjoint.
    """

    def __init__(self, problem, prec="fp32", mode="auto", stream=None, mem_budget: int = 0,
                 use_tensor_cores: int = 0):
        self.p = problem
        self.Nt, self.du, self.d, self.M = problem.Nt, problem.du, problem.d, problem.M
        self.stream_handle = self._stream(stream)
        self._opts = dict(prec=prec, mode=mode, use_tensor_cores=int(use_tensor_cores),
                          mem_budget_bytes=int(mem_budget))
        self.desc = self._make_desc(problem)
        h = ctypes.c_void_p()
        _check(lib().jd_problem_create(ctypes.byref(self.desc), ctypes.byref(h)), "jd_problem_create")
        self.h = h

    def _make_desc(self, problem) -> ProblemDesc:
        """Descriptor of ``problem``; the arrays it points to are kept in self._arrays."""
        desc, self._arrays = make_desc(problem, stream_handle=self.stream_handle, **self._opts)
        return desc

    def update(self, problem):
        """Move the problem's coefficients to those of ``problem`` (jd_problem_update);
        sizes, drift family and precision must not change."""
        desc = self._make_desc(problem)
        _check(lib().jd_problem_update(self.h, ctypes.byref(desc)), "jd_problem_update")
        self.p, self.desc = problem, desc

    def forward_into(self, u, J_out=None):
        """jd_forward: forward sweep keeping the adjoint plan's states.  J_out: a CUDA
        float64 tensor with one element (written in stream order, no synchronization),
        or None to return J as a float (synchronizes)."""
        up, us, _keep = _u_arg(u, self.n)
        if J_out is None:
            J = ctypes.c_double()
            _check(lib().jd_forward(self.h, up, us, ctypes.byref(J), JD_MEM_HOST), "jd_forward")
            return J.value
        if not (_is_torch(J_out) and J_out.is_cuda and J_out.numel() == 1):
            raise ValueError("J_out must be a CUDA tensor with one element")
        _check(lib().jd_forward(self.h, up, us, ctypes.c_void_p(J_out.data_ptr()), JD_MEM_DEVICE),
               "jd_forward")
        return None

    def backward_into(self, grad_out, theta_out=None):
        """jd_backward into CUDA float64 tensors grad_out (Nt*du) and theta_out (d+2) or
        None; does not synchronize."""
        for t, n in ((grad_out, self.n), (theta_out, self.d + 2)):
            if t is not None and not (_is_torch(t) and t.is_cuda and t.is_contiguous() and t.numel() == n):
                raise ValueError(f"outputs must be contiguous CUDA float64 tensors of {n} entries")
        _check(lib().jd_backward(self.h, ctypes.c_void_p(grad_out.data_ptr()), JD_MEM_DEVICE,
                                 None if theta_out is None else ctypes.c_void_p(theta_out.data_ptr())),
               "jd_backward")

    def backward(self, theta: bool = False):
        """jd_backward to host memory: (grad (Nt, du), grad_theta (d+2) or None)."""
        g = np.zeros((self.Nt, self.du))
        gth = np.zeros(self.d + 2) if theta else None
        _check(lib().jd_backward(self.h, _ptr(g), JD_MEM_HOST, _ptr(gth)), "jd_backward")
        return g, gth

    @staticmethod
    def _stream(stream):
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream()
            except ImportError:
                pass
            if stream is None:
                return None
        handle = stream if isinstance(stream, int) else stream.cuda_stream
        # torch's default stream has handle 0, which the C ABI reads as "make a private
        # stream": pass the legacy default stream (cudaStreamLegacy) instead, so the
        # library's work stays ordered with torch's on that stream
        return ctypes.c_void_p(handle if handle else _CUDA_STREAM_LEGACY)

    @property
    def n(self) -> int:
        return self.Nt * self.du

    def close(self):
        if getattr(self, "h", None):
            lib().jd_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def cost(self, u) -> float:
        up, us, _keep = _u_arg(u, self.n)
        J = ctypes.c_double()
        _check(lib().jd_cost(self.h, up, us, ctypes.byref(J)), "jd_cost")
        return J.value

    def gradient(self, u, theta: bool = False):
        """(J, grad (Nt, du) numpy, grad_theta (d+2) or None)."""
        up, us, _keep = _u_arg(u, self.n)
        J = ctypes.c_double()
        g = np.zeros((self.Nt, self.du))
        gth = np.zeros(self.d + 2) if theta else None
        _check(lib().jd_gradient(self.h, up, us, ctypes.byref(J), _ptr(g), JD_MEM_HOST, _ptr(gth)),
               "jd_gradient")
        return J.value, g, gth

    def gradient_into(self, u, grad_out, want_J: bool = True, theta: bool = False):
        """Gradient written into a device tensor grad_out (float64, Nt*du); returns
        (J or None, grad_theta or None).  Without J/theta the call does not synchronize."""
        up, us, _keep = _u_arg(u, self.n)
        if not (_is_torch(grad_out) and grad_out.is_cuda):
            raise ValueError("grad_out must be a CUDA tensor")
        J = ctypes.c_double()
        gth = np.zeros(self.d + 2) if theta else None
        _check(lib().jd_gradient(self.h, up, us, ctypes.byref(J) if want_J else None,
                                 ctypes.c_void_p(grad_out.data_ptr()), JD_MEM_DEVICE, _ptr(gth)),
               "jd_gradient")
        return (J.value if want_J else None), gth

    # --- path sharding: unit sums of this problem's paths ------------------------------
    def gradient_units(self, u):
        """Unit sums [ceil(M / UNIT_PATHS), 1 + Nt du] (jd_gradient_units, host)."""
        up, us, _keep = _u_arg(u, self.n)
        out = np.zeros((-(-self.M // UNIT_PATHS), 1 + self.n))
        _check(lib().jd_gradient_units(self.h, up, us, _ptr(out), JD_MEM_HOST), "jd_gradient_units")
        return out

    def cost_units(self, u):
        """Cost unit sums [ceil(M / UNIT_PATHS), 1] (jd_cost_units, host)."""
        up, us, _keep = _u_arg(u, self.n)
        out = np.zeros((-(-self.M // UNIT_PATHS), 1))
        _check(lib().jd_cost_units(self.h, up, us, _ptr(out), JD_MEM_HOST), "jd_cost_units")
        return out

    # --- feedback control u(z, t) = mu(t)^T phi(z) (d = 2, du = 1) ---------------------
    def fb_cost(self, fb, mu) -> float:
        """J(mu) of the feedback form; mu (Nt, nx*nv) numpy/torch float64."""
        mp, ms, _keep = _u_arg(mu, self.Nt * fb.nx * fb.nv)
        J = ctypes.c_double()
        F = make_feedback(fb)
        _check(lib().jd_fb_cost(self.h, ctypes.byref(F), mp, ms, ctypes.byref(J)), "jd_fb_cost")
        return J.value

    def fb_gradient(self, fb, mu):
        """(J, dJ/dmu (Nt, nx*nv) numpy) for host mu; for a CUDA tensor mu the gradient is a
        CUDA tensor too."""
        n = self.Nt * fb.nx * fb.nv
        mp, ms, _keep = _u_arg(mu, n)
        J = ctypes.c_double()
        F = make_feedback(fb)
        if ms == JD_MEM_DEVICE:
            import torch
            g = torch.empty((self.Nt, fb.nx * fb.nv), dtype=torch.float64, device=mu.device)
            gp = ctypes.c_void_p(g.data_ptr())
        else:
            g = np.zeros((self.Nt, fb.nx * fb.nv))
            gp = _ptr(g)
        _check(lib().jd_fb_gradient(self.h, ctypes.byref(F), mp, ms, ctypes.byref(J), gp), "jd_fb_gradient")
        return J.value, g

    def fb_optimize(self, fb, mu0=None, max_iter=20, tol_rel_grad=1e-4, tol_step=0.0, armijo_c=1e-4,
                    zeta0=1.0, zeta_max=1e3, max_backtracks=40, resample=False):
        """Armijo descent on the feedback weights: (mu (Nt, L) numpy, result dict, J history)."""
        L = fb.nx * fb.nv
        mu = np.zeros((self.Nt, L)) if mu0 is None else _f64(mu0).reshape(self.Nt, L).copy()
        o = OptParams(max_iter=max_iter, tol_rel_grad=tol_rel_grad, tol_step=tol_step, armijo_c=armijo_c,
                      zeta0=zeta0, zeta_max=zeta_max, max_backtracks=max_backtracks, resample=int(resample))
        r = OptResult()
        hist = np.full(max_iter + 1, np.nan)
        F = make_feedback(fb)
        st = lib().jd_fb_optimize(self.h, ctypes.byref(F), _ptr(mu), JD_MEM_HOST, ctypes.byref(o), ctypes.byref(r),
                                  _ptr(hist))
        if st not in (JD_OK, JD_ERR_LINESEARCH):
            _check(st, "jd_fb_optimize")
        res = dict(iters=r.iters, evals=r.evals, status=r.status, J=r.J, rel_grad_norm=r.rel_grad_norm, zeta=r.zeta,
                   sweeps=r.sweeps)
        return mu, res, hist[: r.iters + 1]

    def sample_paths(self, u, m0: int, count: int, lam: bool = True):
        """(X (count, Nt+1, d), lam (count, Nt+1, d) or None, cost (count))."""
        up, us, _keep = _u_arg(u, self.n)
        X = np.zeros((count, self.Nt + 1, self.d))
        L = np.zeros((count, self.Nt + 1, self.d)) if lam else None
        c = np.zeros(count)
        _check(lib().jd_sample_paths(self.h, up, us, int(m0), int(count), _ptr(X), _ptr(L), _ptr(c)),
               "jd_sample_paths")
        return X, L, c

    def optimize(self, u0=None, max_iter=50, tol_rel_grad=1e-4, tol_step=0.0, armijo_c=1e-4,
                 zeta0=1.0, zeta_max=1e3, max_backtracks=40, raise_on_error=True, resample=False,
                 pairs=True):
        """Projected-gradient Armijo descent (jd_optimize); returns (u, result dict, J history).
        ``pairs``: paired Armijo trials in one sweep where memory allows (same iterates)."""
        u = np.zeros((self.Nt, self.du)) if u0 is None else _f64(u0).reshape(self.Nt, self.du).copy()
        o = OptParams(max_iter=max_iter, tol_rel_grad=tol_rel_grad, tol_step=tol_step,
                      armijo_c=armijo_c, zeta0=zeta0, zeta_max=zeta_max, max_backtracks=max_backtracks,
                      resample=int(resample), one_trial_per_sweep=int(not pairs))
        r = OptResult()
        hist = np.full(max_iter + 2, np.nan)
        st = lib().jd_optimize(self.h, _ptr(u), JD_MEM_HOST, ctypes.byref(o), ctypes.byref(r), _ptr(hist))
        if raise_on_error:
            _check(st, "jd_optimize")
        res = dict(iters=r.iters, evals=r.evals, status=r.status, J=r.J,
                   rel_grad_norm=r.rel_grad_norm, zeta=r.zeta, sweeps=r.sweeps)
        return u, res, hist[: r.iters + 1]

    def info(self):
        b = ctypes.c_size_t()
        m = ctypes.c_int()
        _check(lib().jd_problem_info(self.h, ctypes.byref(b), ctypes.byref(m)), "jd_problem_info")
        return dict(device_bytes=b.value, mode={0: "auto", 1: "stored", 2: "recompute"}[m.value])


class JdServer:
    """The serving loop (jd_server_*): submit problems, poll results.

    ``budget``: device bytes for admitted requests (0 = 80% of free memory);
    ``max_slots``: requests in flight at most; ``batch_paths``: small requests (d <= 2,
    du = 1, stored plan) with at most this many paths share batched launches (None = the
    library's default, 0 = off)."""

    def __init__(self, budget: int = 0, max_slots: int = 16, batch_paths=None):
        h = ctypes.c_void_p()
        _check(lib().jd_server_create(int(budget), int(max_slots), ctypes.byref(h)), "jd_server_create")
        self.h = h
        self._shapes = {}
        if batch_paths is not None:
            _check(lib().jd_server_set_batching(self.h, int(batch_paths)), "jd_server_set_batching")

    def batch_stats(self):
        """(batched launch sequences, request phases they ran)."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().jd_server_batch_stats(self.h, ctypes.byref(a), ctypes.byref(b)), "jd_server_batch_stats")
        return a.value, b.value

    def submit(self, problem, prec="fp32", mode="auto", use_tensor_cores=0, max_iter=200,
               tol_rel_grad=1e-4, tol_step=0.0, armijo_c=1e-4, zeta0=1.0, zeta_max=1e3,
               max_backtracks=40) -> int:
        desc, _keep = make_desc(problem, prec=prec, mode=mode, use_tensor_cores=use_tensor_cores)
        o = OptParams(max_iter=max_iter, tol_rel_grad=tol_rel_grad, tol_step=tol_step,
                      armijo_c=armijo_c, zeta0=zeta0, zeta_max=zeta_max, max_backtracks=max_backtracks)
        t = ctypes.c_uint64()
        _check(lib().jd_server_submit(self.h, ctypes.byref(desc), ctypes.byref(o), ctypes.byref(t)),
               "jd_server_submit")
        self._shapes[t.value] = (problem.Nt, problem.du)
        return t.value

    def poll(self, ticket: int):
        """None while running; then (u (Nt, du), result dict)."""
        Nt, du = self._shapes[ticket]
        u = np.zeros((Nt, du))
        r = OptResult()
        st = lib().jd_server_poll(self.h, ticket, _ptr(u), ctypes.byref(r))
        if st == JD_ERR_BUSY:
            return None
        _check(st, "jd_server_poll")
        return u, dict(iters=r.iters, evals=r.evals, status=r.status, J=r.J,
                       rel_grad_norm=r.rel_grad_norm, zeta=r.zeta, sweeps=r.sweeps)

    def wait(self, ticket: int, timeout: float = 0.0) -> bool:
        st = lib().jd_server_wait(self.h, ticket, float(timeout))
        if st == JD_ERR_BUSY:
            return False
        _check(st, "jd_server_wait")
        return True

    def info(self, ticket: int):
        i = RequestInfo()
        _check(lib().jd_server_info(self.h, ticket, ctypes.byref(i)), "jd_server_info")
        return dict(submit_s=i.submit_s, admit_s=i.admit_s, done_s=i.done_s, device_bytes=i.device_bytes,
                    plan={0: "auto", 1: "stored", 2: "recompute"}[i.plan], done=bool(i.done),
                    path_steps=i.path_steps, sweep_steps=i.sweep_steps)

    def close(self):
        if getattr(self, "h", None):
            lib().jd_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
