"""FP64 CPU oracle for the jump-diffusion adjoint method (TEST INFRASTRUCTURE ONLY).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.

The C library ``jd_oracle.c`` follows the paper step by step:
  * forward sweep: Algorithm 5.1 / 5.2 with additive jumps (Sec. 5.3-5.4,
    eq:SDE_splitted_drift_Euler) on the jump-adapted grid (Sec. 3);
  * cost: eq:discrete_functional (Sec. 3);
  * adjoint and reduced gradient: eq:AdjointModel, eq:definition_Gradient (Sec. 4)
    and eq:adjoint_eq_approximation (Sec. 5.5), read as the exact derivative of the
    discrete cost;
  * optimizer: Algorithm 5.4 with eq:Stochastic_Armijo (Sec. 5.6), projected onto
    the control bounds.
``closed_forms.py`` holds the linear-quadratic closed forms used as pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libjd_oracle.so")
_lib = None
_lock = threading.Lock()

NMAX = 16
DMAX = 64


def build(force: bool = False) -> str:
    """Compile jd_oracle.c into libjd_oracle.so next to it (gcc, -O2, no -march)."""
    src = os.path.join(_HERE, "jd_oracle.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)
            and os.path.getmtime(_SO) >= os.path.getmtime(os.path.join(_HERE, "jd_oracle.h"))):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
           "-o", tmp, src, "-lm", "-lpthread"]
    subprocess.check_call(cmd, cwd=_HERE)
    os.replace(tmp, _SO)
    return _SO


class _Problem(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("du", ctypes.c_int), ("Nt", ctypes.c_int),
        ("M", ctypes.c_int64), ("T", ctypes.c_double), ("drift", ctypes.c_int),
        ("A", ctypes.c_void_p), ("C", ctypes.c_void_p), ("B", ctypes.c_void_p),
        ("dA", ctypes.c_void_p), ("sigma", ctypes.c_void_p), ("lam", ctypes.c_double),
        ("jump_law", ctypes.c_int), ("jump_scale", ctypes.c_double),
        ("x0", ctypes.c_void_p), ("q", ctypes.c_void_p), ("xd", ctypes.c_void_p),
        ("nu", ctypes.c_double), ("u_min", ctypes.c_double), ("u_max", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("epoch", ctypes.c_uint32), ("jump_gain", ctypes.c_double),
    ]


class _Feedback(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("nv", ctypes.c_int), ("x_max", ctypes.c_double),
                ("v_max", ctypes.c_double), ("eps", ctypes.c_double), ("track", ctypes.c_int),
                ("sigma_J", ctypes.c_double), ("adjoint", ctypes.c_int), ("sur_rate", ctypes.c_double),
                ("particles", ctypes.c_int), ("omega", ctypes.c_double), ("ax", ctypes.c_double),
                ("av", ctypes.c_double)]


def _fb(f) -> _Feedback:
    return _Feedback(nx=int(f.nx), nv=int(f.nv), x_max=float(f.x_max), v_max=float(f.v_max),
                     eps=float(f.eps), track=int(f.track), sigma_J=float(f.sigma_J),
                     adjoint=int(getattr(f, "adjoint", 0)), sur_rate=float(getattr(f, "sur_rate", 0.0)),
                     particles=int(getattr(f, "particles", 0)), omega=float(getattr(f, "omega", 0.0)),
                     ax=float(getattr(f, "ax", 1.0)), av=float(getattr(f, "av", 1.0)))


class _Draws(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("theta", ctypes.c_double * NMAX),
        ("delta", ctypes.c_double * (NMAX + 1)),
        ("Z", (ctypes.c_double * DMAX) * (NMAX + 1)),
        ("xi_hat", (ctypes.c_double * DMAX) * NMAX),
    ]


class _OptParams(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int), ("tol_rel_grad", ctypes.c_double),
                ("tol_step", ctypes.c_double), ("armijo_c", ctypes.c_double),
                ("zeta0", ctypes.c_double), ("zeta_max", ctypes.c_double),
                ("max_backtracks", ctypes.c_int), ("resample", ctypes.c_int)]


class _OptResult(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("evals", ctypes.c_int), ("status", ctypes.c_int),
                ("J", ctypes.c_double), ("rel_grad_norm", ctypes.c_double),
                ("zeta", ctypes.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.POINTER
            L.orc_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
            L.orc_u01.argtypes = [ctypes.c_uint32]
            L.orc_u01.restype = ctypes.c_double
            L.orc_poisson_thresholds.argtypes = [ctypes.c_double, P(ctypes.c_uint64)]
            L.orc_poisson_count.argtypes = [ctypes.c_uint32, P(ctypes.c_uint64)]
            L.orc_normal_pair.argtypes = [ctypes.c_uint32, ctypes.c_uint32, P(ctypes.c_double)]
            L.orc_step_draws.argtypes = [P(_Problem), ctypes.c_int, ctypes.c_int64, P(_Draws)]
            L.orc_path.argtypes = [P(_Problem), ctypes.c_void_p, ctypes.c_int64] + [ctypes.c_void_p] * 6
            L.orc_cost.argtypes = [P(_Problem), ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
            L.orc_gradient.argtypes = [P(_Problem), ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 3
            L.orc_optimize.argtypes = [P(_Problem), ctypes.c_void_p, P(_OptParams), ctypes.c_int,
                                       P(_OptResult), ctypes.c_void_p]
            L.orc_bump.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_bump.restype = ctypes.c_double
            L.orc_bump_dr.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_bump_dr.restype = ctypes.c_double
            L.orc_fb_control.argtypes = [P(_Feedback)] + [ctypes.c_void_p] * 4
            L.orc_fb_control.restype = ctypes.c_double
            L.orc_fb_path.argtypes = [P(_Problem), P(_Feedback), ctypes.c_void_p, ctypes.c_int64] + [ctypes.c_void_p] * 5
            L.orc_fb_cost.argtypes = [P(_Problem), P(_Feedback), ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
            L.orc_fb_gradient.argtypes = [P(_Problem), P(_Feedback), ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 2
            L.orc_fb_surrogate_state.argtypes = [P(_Problem), P(_Feedback), ctypes.c_int, ctypes.c_int64,
                                                 ctypes.c_void_p]
            L.orc_fb_coupled.argtypes = [P(_Problem), P(_Feedback), ctypes.c_void_p, ctypes.c_int64] + [ctypes.c_void_p] * 4
            L.orc_ring_lanes.argtypes = [ctypes.c_int]
            L.orc_fb_coupled_gradient.argtypes = [P(_Problem), P(_Feedback), ctypes.c_void_p, ctypes.c_int,
                                                  ctypes.c_void_p, ctypes.c_void_p]
            L.orc_fb_optimize.argtypes = [P(_Problem), P(_Feedback), ctypes.c_void_p, P(_OptParams), ctypes.c_int,
                                          P(_OptResult), ctypes.c_void_p]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class OracleProblem:
    """Marshals a workloads.Problem (duck-typed) into the C struct; keeps the
    arrays alive for the lifetime of this object."""

    def __init__(self, p):
        self.p = p
        a = p.arrays()
        self._arrays = a
        self.s = _Problem(
            d=p.d, du=p.du, Nt=p.Nt, M=p.M, T=p.T, drift=p.drift,
            A=_ptr(a["A"]), C=_ptr(a["C"]), B=_ptr(a["B"]), dA=_ptr(a["dA"]),
            sigma=_ptr(a["sigma"]), lam=p.lam, jump_law=p.jump_law, jump_scale=p.jump_scale,
            x0=_ptr(a["x0"]), q=_ptr(a["q"]), xd=_ptr(a["xd"]), nu=p.nu, u_min=p.u_min,
            u_max=p.u_max, seed=p.seed, epoch=p.epoch, jump_gain=getattr(p, "jump_gain", 1.0))

    def _u(self, u):
        p = self.p
        if u is None:
            u = np.zeros((p.Nt, p.du))
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(p.Nt, p.du)
        return u


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def philox(key, ctr):
    """One Philox4x32-10 block as 4 uint32."""
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xffffffff for x in key])
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xffffffff for x in ctr])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(k, c, o)
    return [int(x) for x in o]


def u01(w: int) -> float:
    return lib().orc_u01(int(w) & 0xffffffff)


def poisson_thresholds(mu: float):
    t = (ctypes.c_uint64 * NMAX)()
    lib().orc_poisson_thresholds(float(mu), t)
    return [int(x) for x in t]


def poisson_count(w: int, thr) -> int:
    t = (ctypes.c_uint64 * NMAX)(*[int(x) for x in thr])
    return lib().orc_poisson_count(int(w) & 0xffffffff, t)


def normal_pair(wa: int, wb: int):
    z = (ctypes.c_double * 2)()
    lib().orc_normal_pair(int(wa) & 0xffffffff, int(wb) & 0xffffffff, z)
    return float(z[0]), float(z[1])


def step_draws(p, k: int, m: int):
    """Draws of step k of path m: dict(n, theta, delta, Z (n+1,d), xi_hat (n,d))."""
    op = OracleProblem(p)
    D = _Draws()
    rc = lib().orc_step_draws(ctypes.byref(op.s), int(k), int(m), ctypes.byref(D))
    assert rc == 0
    n = D.n
    d = p.d
    Z = np.array([[D.Z[i][c] for c in range(d)] for i in range(n + 1)])
    xi = np.array([[D.xi_hat[i][c] for c in range(d)] for i in range(n)]).reshape(n, d)
    return dict(n=n, theta=np.array(D.theta[:n]), delta=np.array(D.delta[:n + 1]), Z=Z, xi_hat=xi)


def path(p, u=None, m: int = 0, adjoint: bool = True, theta: bool = False):
    """One path: dict(X (Nt+1,d), lam (Nt+1,d), G (Nt,du), cost, gtheta (d+2), njumps (Nt))."""
    op = OracleProblem(p)
    u = op._u(u)
    X = np.zeros((p.Nt + 1, p.d))
    lam = np.zeros((p.Nt + 1, p.d)) if adjoint else None
    G = np.zeros((p.Nt, p.du)) if adjoint else None
    gth = np.zeros(p.d + 2) if theta else None
    cost = np.zeros(1)
    nj = np.zeros(p.Nt, dtype=np.int32)
    rc = lib().orc_path(ctypes.byref(op.s), _ptr(u), int(m), _ptr(X), _ptr(lam), _ptr(G),
                        _ptr(cost), _ptr(gth), _ptr(nj))
    if rc:
        raise ValueError(f"orc_path failed ({rc})")
    return dict(X=X, lam=lam, G=G, cost=float(cost[0]), gtheta=gth, njumps=nj)


def cost(p, u=None, nthreads: int | None = None) -> float:
    op = OracleProblem(p)
    u = op._u(u)
    J = np.zeros(1)
    rc = lib().orc_cost(ctypes.byref(op.s), _ptr(u), nthreads or default_threads(), _ptr(J))
    if rc:
        raise ValueError(f"orc_cost failed ({rc})")
    return float(J[0])


def gradient(p, u=None, nthreads: int | None = None, theta: bool = False):
    """(J, grad (Nt,du), gtheta (d+2) or None); grad is the Euclidean dJ/du_k."""
    op = OracleProblem(p)
    u = op._u(u)
    J = np.zeros(1)
    g = np.zeros((p.Nt, p.du))
    gth = np.zeros(p.d + 2) if theta else None
    rc = lib().orc_gradient(ctypes.byref(op.s), _ptr(u), nthreads or default_threads(),
                            _ptr(J), _ptr(g), _ptr(gth))
    if rc:
        raise ValueError(f"orc_gradient failed ({rc})")
    return float(J[0]), g, gth


def optimize(p, u0=None, max_iter=50, tol_rel_grad=1e-4, tol_step=0.0, armijo_c=1e-4,
             zeta0=1.0, zeta_max=1e3, max_backtracks=40, nthreads=None, resample=False):
    """Projected-gradient Armijo descent; returns (u, result dict, J history)."""
    op = OracleProblem(p)
    u = op._u(u0).copy()
    o = _OptParams(max_iter=max_iter, tol_rel_grad=tol_rel_grad, tol_step=tol_step,
                   armijo_c=armijo_c, zeta0=zeta0, zeta_max=zeta_max,
                   max_backtracks=max_backtracks, resample=int(resample))
    r = _OptResult()
    hist = np.full(max_iter + 2, np.nan)
    lib().orc_optimize(ctypes.byref(op.s), _ptr(u), ctypes.byref(o), nthreads or default_threads(),
                       ctypes.byref(r), _ptr(hist))
    res = dict(iters=r.iters, evals=r.evals, status=r.status, J=r.J,
               rel_grad_norm=r.rel_grad_norm, zeta=r.zeta)
    return u, res, hist[: r.iters + 1]


# --- feedback control (Sec. 2 eq:control_structure, Sec. 5.1-5.2, Sec. 6) -------------
def bump(r, eps):
    """phi(x, x_c, eps) at r = x - x_c (vectorised over r)."""
    f = np.vectorize(lambda t: lib().orc_bump(float(t), float(eps)))
    return f(r)


def bump_dr(r, eps):
    f = np.vectorize(lambda t: lib().orc_bump_dr(float(t), float(eps)))
    return f(r)


def _mu(p, fb, mu):
    L = fb.nx * fb.nv
    if mu is None:
        mu = np.zeros((p.Nt, L))
    return np.ascontiguousarray(mu, dtype=np.float64).reshape(p.Nt, L)


def fb_control(fb, mu_k, z):
    """(u, (u_x, u_v), phi (L)) at the phase-space point z under the weights mu_k (L)."""
    mk = np.ascontiguousarray(mu_k, dtype=np.float64).reshape(-1)
    zz = np.ascontiguousarray(z, dtype=np.float64).reshape(2)
    du = np.zeros(2)
    phi = np.zeros(fb.nx * fb.nv)
    F = _fb(fb)
    u = lib().orc_fb_control(ctypes.byref(F), _ptr(mk), _ptr(zz), _ptr(du), _ptr(phi))
    return float(u), du, phi


def fb_path(p, fb, mu=None, m: int = 0, adjoint: bool = True):
    """One path under feedback: dict(X (Nt+1,2), lam, G (Nt,L), cost, njumps)."""
    op = OracleProblem(p)
    F = _fb(fb)
    mu = _mu(p, fb, mu)
    X = np.zeros((p.Nt + 1, 2))
    lam = np.zeros((p.Nt + 1, 2)) if adjoint else None
    G = np.zeros((p.Nt, fb.nx * fb.nv)) if adjoint else None
    cost = np.zeros(1)
    nj = np.zeros(p.Nt, dtype=np.int32)
    rc = lib().orc_fb_path(ctypes.byref(op.s), ctypes.byref(F), _ptr(mu), int(m), _ptr(X),
                           _ptr(lam), _ptr(G), _ptr(cost), _ptr(nj))
    if rc:
        raise ValueError(f"orc_fb_path failed ({rc})")
    return dict(X=X, lam=lam, G=G, cost=float(cost[0]), njumps=nj)


def fb_cost(p, fb, mu=None, nthreads: int | None = None) -> float:
    op = OracleProblem(p)
    F = _fb(fb)
    mu = _mu(p, fb, mu)
    J = np.zeros(1)
    rc = lib().orc_fb_cost(ctypes.byref(op.s), ctypes.byref(F), _ptr(mu), nthreads or default_threads(), _ptr(J))
    if rc:
        raise ValueError(f"orc_fb_cost failed ({rc})")
    return float(J[0])


def fb_gradient(p, fb, mu=None, nthreads: int | None = None):
    """(J, dJ/dmu (Nt, L))."""
    op = OracleProblem(p)
    F = _fb(fb)
    mu = _mu(p, fb, mu)
    J = np.zeros(1)
    g = np.zeros((p.Nt, fb.nx * fb.nv))
    rc = lib().orc_fb_gradient(ctypes.byref(op.s), ctypes.byref(F), _ptr(mu), nthreads or default_threads(),
                               _ptr(J), _ptr(g))
    if rc:
        raise ValueError(f"orc_fb_gradient failed ({rc})")
    return float(J[0]), g


def fb_optimize(p, fb, mu0=None, max_iter=20, tol_rel_grad=1e-4, tol_step=0.0, armijo_c=1e-4,
                zeta0=1.0, zeta_max=1e3, max_backtracks=40, nthreads=None, resample=False):
    """Armijo gradient descent on the feedback weights; returns (mu, result dict, J history)."""
    op = OracleProblem(p)
    F = _fb(fb)
    mu = _mu(p, fb, mu0).copy()
    o = _OptParams(max_iter=max_iter, tol_rel_grad=tol_rel_grad, tol_step=tol_step,
                   armijo_c=armijo_c, zeta0=zeta0, zeta_max=zeta_max, max_backtracks=max_backtracks,
                   resample=int(resample))
    r = _OptResult()
    hist = np.full(max_iter + 2, np.nan)
    lib().orc_fb_optimize(ctypes.byref(op.s), ctypes.byref(F), _ptr(mu), ctypes.byref(o),
                          nthreads or default_threads(), ctypes.byref(r), _ptr(hist))
    res = dict(iters=r.iters, evals=r.evals, status=r.status, J=r.J,
               rel_grad_norm=r.rel_grad_norm, zeta=r.zeta)
    return mu, res, hist[: r.iters + 1]


def fb_surrogate_state(p, fb, k: int, m: int):
    """The surrogate state z_d(t_k) + sqrt(rate t_k) xi of step k, path m (Sec. 6.5)."""
    op = OracleProblem(p)
    F = _fb(fb)
    z = np.zeros(2)
    lib().orc_fb_surrogate_state(ctypes.byref(op.s), ctypes.byref(F), int(k), int(m), _ptr(z))
    return z


def ring_lanes(N: int) -> int:
    """Path-index stride of a ring of N particles (orc_ring_lanes)."""
    return int(lib().orc_ring_lanes(int(N)))


def fb_coupled(p, fb, mu=None, r: int = 0, adjoint: bool = True):
    """Realization r of the coupled particles: dict(X (Nt+1,N,2), lam, G (Nt,L) summed over
    the particles, cost summed over the particles)."""
    op = OracleProblem(p)
    F = _fb(fb)
    mu = _mu(p, fb, mu)
    N = fb.particles
    X = np.zeros((p.Nt + 1, N, 2))
    lam = np.zeros((p.Nt + 1, N, 2)) if adjoint else None
    G = np.zeros((p.Nt, fb.nx * fb.nv)) if adjoint else None
    cost = np.zeros(1)
    rc = lib().orc_fb_coupled(ctypes.byref(op.s), ctypes.byref(F), _ptr(mu), int(r), _ptr(X), _ptr(lam),
                              _ptr(G), _ptr(cost))
    if rc:
        raise ValueError(f"orc_fb_coupled failed ({rc})")
    return dict(X=X, lam=lam, G=G, cost=float(cost[0]))


def fb_coupled_gradient(p, fb, mu=None):
    """(J, dJ/dmu (Nt, L)) over the M/S realizations of the coupled particles
    (S = ring_lanes(particles))."""
    op = OracleProblem(p)
    F = _fb(fb)
    mu = _mu(p, fb, mu)
    J = np.zeros(1)
    g = np.zeros((p.Nt, fb.nx * fb.nv))
    rc = lib().orc_fb_coupled_gradient(ctypes.byref(op.s), ctypes.byref(F), _ptr(mu), 1, _ptr(J), _ptr(g))
    if rc:
        raise ValueError(f"orc_fb_coupled_gradient failed ({rc})")
    return float(J[0]), g
