"""Seeded synthetic inputs for the jump-diffusion control problems.

This module only builds problem data (coefficients, targets, sizes, seeds).  It holds
none of the method's arithmetic, and both the CUDA path and the FP64 oracle take their
inputs from it.  The shapes follow the paper's experiments (Sec. 6: particle systems
in phase space, N = 2000 particles, N_t = 50..100 steps) scaled to the sizes of the
GPU workloads below.

Every builder returns a :class:`Problem`, a plain container of numpy arrays.

Workloads (named by what they are):
  * ``lq_scalar``      d=1 linear-quadratic jump diffusion dX=(u-X)dt+0.2dW+dJ,
                       lambda=2, jumps N(0,0.1^2), X0=1, T=1, N_t=100, M=1000,
                       target sin(2 pi t), nu=1e-3, |u|<=5, seed 0.
  * ``double_well``    d=2 cubic drift f1=x1-x1^3, f2=-0.5 x2+u, sigma=(0.3,0.3),
                       lambda=5, jumps uniform in [-0.2,0.2]^2, X0=(1,0), T=2,
                       N_t=1000, M=2^20, target (1, sin 2 pi t), nu=1e-3, |u|<=5.
  * ``double_well_phase``  the phase-space reading of the same model:
                       f1=x2, f2=x1-x1^3-0.5x2+u (mirrors the paper's H=[[0,1],[-eta,0]]).
  * ``double_well_autograd``  double_well with M=2^22, N_t=4096 and the damping
                       direction dA = -e2 e2^T for the drift-coefficient gradient.
  * ``linear32``       d=32 linear drift A = Q diag(ev) Q^T, ev ~ U[-2,-0.1], B 32x4
                       N(0,1/32) (numpy default_rng(1)), sigma=0.1, lambda=1, jumps
                       N(0,0.05^2 I), X0=1, target 0, T=1, N_t=500, M=2^18.
  * ``ks_oscillator``  d=2 phase-space particle x'=v, v'=-x+u with Keilson-Storer
                       velocity resets (beta=10, gamma=0.9), M=2^20, N_t=500.
  * ``feedback_centering``  the paper's feedback problem (Sec. 6.1): z=(x,v),
                       x'=v, v'=-eta x+u(z,t), eta=1, u = mu(t)^T phi(z) with 10x10
                       bump shape functions on (-2,2)^2, eps=0.5, Keilson-Storer resets
                       (beta=10, gamma=0.9), Gaussian tracking of z_d=(0,0), sigma_J=1,
                       alpha=1e-2, b=(0.1,0.1), z0=(0.75,0.75), T=1, N_t=100, M=2^20.
  * ``feedback_trajectory``  Sec. 6.3: the same model with eta=0, eps=0.1, following
                       z_d(t) = (-x_max/2 + x_max t/T, v_max/2 - |v_max t/(2T)|).
  * ``feedback_coupled``  Sec. 6.4: rings of 32 coupled oscillators (eta=1, omega=0.5)
                       on the ellipse A_x=1.5, A_v=1.7071, ellipse tracking cost, M=2^20
                       (2^15 realizations), N_t=100.
  * ``serving_requests``  a stream of requests (d in {1,2,8,32}, M log-uniform in
                       [2^12,2^22], N_t uniform in [50,2000], lambda uniform in
                       [0.5,10]) with Poisson arrivals, numpy default_rng(5).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

LINEAR, CUBIC = 0, 1
JUMP_NONE, JUMP_NORMAL, JUMP_UNIFORM, JUMP_KS = 0, 1, 2, 3


@dataclasses.dataclass
class Problem:
    d: int
    du: int
    T: float
    Nt: int
    M: int
    drift: int
    A: np.ndarray
    B: np.ndarray
    sigma: np.ndarray
    x0: np.ndarray
    q: np.ndarray
    xd: np.ndarray
    C: Optional[np.ndarray] = None
    dA: Optional[np.ndarray] = None
    lam: float = 0.0
    jump_law: int = JUMP_NONE
    jump_scale: float = 0.0
    jump_gain: float = 1.0        # JUMP_KS: velocity gain gamma (v <- gamma v + jump_scale xi)
    nu: float = 1e-3
    u_min: float = -5.0
    u_max: float = 5.0
    seed: int = 0
    epoch: int = 0
    name: str = ""
    m_offset: int = 0             # global index of the first path (one shard of a larger sample)

    def replace(self, **kw) -> "Problem":
        """A copy with some fields changed; the target is resampled if Nt changes."""
        p = dataclasses.replace(self, **kw)
        if "Nt" in kw and "xd" not in kw and kw["Nt"] != self.Nt:
            p.xd = _target(self.name, p.T, p.Nt, p.d)
        return p

    @property
    def dt(self) -> float:
        return self.T / self.Nt

    def arrays(self):
        """All array fields as contiguous float64, C = zeros when absent."""
        d = self.d
        C = self.C if self.C is not None else np.zeros((d, d))
        return dict(
            A=np.ascontiguousarray(self.A, dtype=np.float64).reshape(d, d),
            C=np.ascontiguousarray(C, dtype=np.float64).reshape(d, d),
            B=np.ascontiguousarray(self.B, dtype=np.float64).reshape(d, self.du),
            dA=None if self.dA is None else np.ascontiguousarray(self.dA, dtype=np.float64).reshape(d, d),
            sigma=np.ascontiguousarray(self.sigma, dtype=np.float64).reshape(d),
            x0=np.ascontiguousarray(self.x0, dtype=np.float64).reshape(d),
            q=np.ascontiguousarray(self.q, dtype=np.float64).reshape(d),
            xd=np.ascontiguousarray(self.xd, dtype=np.float64).reshape(self.Nt + 1, d),
        )


def _target(name: str, T: float, Nt: int, d: int) -> np.ndarray:
    """Target samples xd(t_k), k = 0..Nt, for each named family."""
    t = np.arange(Nt + 1) * (T / Nt)
    if name.startswith("lq_scalar"):
        return np.sin(2 * np.pi * t).reshape(Nt + 1, 1)
    if name.startswith("double_well"):
        return np.stack([np.ones_like(t), np.sin(2 * np.pi * t)], axis=1)
    if name.startswith("ks_oscillator"):
        return np.stack([0.5 * np.cos(np.pi * t), -0.5 * np.pi * np.sin(np.pi * t)], axis=1)
    return np.zeros((Nt + 1, d))


def lq_scalar(M: int = 1000, Nt: int = 100, seed: int = 0) -> Problem:
    return Problem(
        name="lq_scalar", d=1, du=1, T=1.0, Nt=Nt, M=M, drift=LINEAR,
        A=np.array([[-1.0]]), B=np.array([[1.0]]), sigma=np.array([0.2]),
        x0=np.array([1.0]), q=np.array([1.0]), xd=_target("lq_scalar", 1.0, Nt, 1),
        lam=2.0, jump_law=JUMP_NORMAL, jump_scale=0.1, nu=1e-3, u_min=-5.0, u_max=5.0,
        seed=seed)


def double_well(M: int = 1 << 20, Nt: int = 1000, seed: int = 0) -> Problem:
    return Problem(
        name="double_well", d=2, du=1, T=2.0, Nt=Nt, M=M, drift=CUBIC,
        A=np.array([[1.0, 0.0], [0.0, -0.5]]), C=np.array([[-1.0, 0.0], [0.0, 0.0]]),
        B=np.array([[0.0], [1.0]]), sigma=np.array([0.3, 0.3]), x0=np.array([1.0, 0.0]),
        q=np.array([1.0, 1.0]), xd=_target("double_well", 2.0, Nt, 2),
        lam=5.0, jump_law=JUMP_UNIFORM, jump_scale=0.2, nu=1e-3, u_min=-5.0, u_max=5.0,
        seed=seed)


def double_well_phase(M: int = 1 << 20, Nt: int = 1000, seed: int = 0) -> Problem:
    p = double_well(M, Nt, seed)
    p.name = "double_well_phase"
    p.A = np.array([[0.0, 1.0], [1.0, -0.5]])
    p.C = np.array([[0.0, 0.0], [-1.0, 0.0]])
    return p


def double_well_autograd(M: int = 1 << 22, Nt: int = 4096, seed: int = 0) -> Problem:
    """double_well with theta = (damping rho, sigma, jump half-width): the damping
    enters A[1][1] = -rho, so the drift-coefficient direction is dA = -e2 e2^T."""
    p = double_well(M, Nt, seed)
    p.name = "double_well_autograd"
    p.dA = np.array([[0.0, 0.0], [0.0, -1.0]])
    return p


def ks_oscillator(M: int = 1 << 20, Nt: int = 500, seed: int = 0, beta: float = 10.0,
                  gamma: float = 0.9) -> Problem:
    """The paper's phase-space particle with Keilson-Storer velocity resets (Sec. 5.3,
    Sec. 6 parameters beta = 10, gamma = 0.9): z = (x, v), harmonic drift x' = v,
    v' = -x + u, jumps at rate sqrt(beta/pi) resetting v <- gamma v + N(0, 1/(2 beta)),
    small diffusion, tracking a half-amplitude circle."""
    return Problem(
        name="ks_oscillator", d=2, du=1, T=1.0, Nt=Nt, M=M, drift=LINEAR,
        A=np.array([[0.0, 1.0], [-1.0, 0.0]]), B=np.array([[0.0], [1.0]]),
        sigma=np.array([0.05, 0.1]), x0=np.array([1.0, 0.0]), q=np.array([1.0, 1.0]),
        xd=_target("ks_oscillator", 1.0, Nt, 2), lam=float(np.sqrt(beta / np.pi)), jump_law=JUMP_KS,
        jump_scale=float(1.0 / np.sqrt(2.0 * beta)), jump_gain=gamma, nu=1e-3, u_min=-5.0, u_max=5.0,
        seed=seed)


def linear_family(d: int, M: int, Nt: int, lam: float = 1.0, seed: int = 0,
                  matrix_seed: int = 1, T: float = 1.0) -> Problem:
    """Random stable linear drift: A = Q diag(ev) Q^T with Q from the QR of a
    standard-normal matrix and ev ~ U[-2,-0.1]; B entries N(0, 1/d); the number of
    controls is min(4, d/2) (at least 1)."""
    rng = np.random.default_rng(matrix_seed)
    G = rng.standard_normal((d, d))
    Q, _ = np.linalg.qr(G)
    ev = rng.uniform(-2.0, -0.1, size=d)
    A = (Q * ev) @ Q.T
    du = max(1, min(4, d // 2))
    B = rng.standard_normal((d, du)) / np.sqrt(d)
    return Problem(
        name=f"linear{d}", d=d, du=du, T=T, Nt=Nt, M=M, drift=LINEAR, A=A, B=B,
        sigma=np.full(d, 0.1), x0=np.ones(d), q=np.ones(d), xd=np.zeros((Nt + 1, d)),
        lam=lam, jump_law=JUMP_NORMAL, jump_scale=0.05, nu=1e-3, u_min=-5.0, u_max=5.0,
        seed=seed)


def linear32(M: int = 1 << 18, Nt: int = 500, seed: int = 0) -> Problem:
    return linear_family(32, M, Nt, lam=1.0, seed=seed, matrix_seed=1)


def random_control(p: Problem, seed: int = 7, scale: float = 1.0) -> np.ndarray:
    """A seeded control u (Nt x du) inside the bounds, for evaluating gradients away
    from u = 0."""
    rng = np.random.default_rng(seed)
    u = scale * rng.standard_normal((p.Nt, p.du))
    return np.clip(u, p.u_min, p.u_max)


def serving_requests(n: int = 10000, rate: float = 200.0, seed: int = 5):
    """Request stream: (arrival_time, Problem).  d uniform in {1,2,8,32}; M
    log-uniform in [2^12, 2^22]; N_t uniform in [50, 2000]; lambda uniform in
    [0.5, 10]; each request gets its own Philox seed."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    out = []
    for i in range(n):
        d = int(rng.choice([1, 2, 8, 32]))
        M = int(np.round(2.0 ** rng.uniform(12, 22)))
        Nt = int(rng.integers(50, 2001))
        lam = float(rng.uniform(0.5, 10.0))
        if d == 1:
            p = lq_scalar(M=M, Nt=Nt)
        elif d == 2:
            p = double_well(M=M, Nt=Nt)
        else:
            p = linear_family(d, M, Nt)
        p.lam = lam
        p.seed = 1000 + i
        p.name = f"{p.name}#req{i}"
        out.append((float(t[i]), p))
    return out


# --- feedback control (Sec. 2 eq:control_structure, Sec. 5.1-5.2, Sec. 6) --------------
TRACK_QUAD, TRACK_GAUSS, TRACK_ELLIPSE = 0, 1, 2
FB_EXACT, FB_SURROGATE = 0, 1


@dataclasses.dataclass
class Feedback:
    """Shape functions of u(z, t) = mu(t)^T phi(z): nx x nv bump products centred on the
    cell centres of (-x_max, x_max) x (-v_max, v_max); tracking cost quadratic or Gaussian
    with width sigma_J."""
    nx: int = 10
    nv: int = 10
    x_max: float = 2.0
    v_max: float = 2.0
    eps: float = 0.5
    track: int = TRACK_GAUSS
    sigma_J: float = 1.0
    adjoint: int = 0          # FB_EXACT, or FB_SURROGATE (Sec. 6.5)
    sur_rate: float = 0.0     # surrogate states N(z_d(t), sur_rate t I)
    particles: int = 0        # coupled particles per realization on a ring (Sec. 6.4), 0 = none
    omega: float = 0.0        # nearest-neighbour coupling
    ax: float = 1.0           # ellipse half-axes (TRACK_ELLIPSE, coupled initial states)
    av: float = 1.0

    @property
    def L(self) -> int:
        return self.nx * self.nv

    def replace(self, **kw) -> "Feedback":
        return dataclasses.replace(self, **kw)


def feedback_centering(M: int = 1 << 20, Nt: int = 100, seed: int = 0, eta: float = 1.0,
                       beta: float = 10.0, gamma: float = 0.9):
    """(Problem, Feedback) of Sec. 6.1: center the particles at z_d = (0, 0)."""
    p = Problem(
        name="feedback_centering", d=2, du=1, T=1.0, Nt=Nt, M=M, drift=LINEAR,
        A=np.array([[0.0, 1.0], [-eta, 0.0]]), B=np.array([[0.0], [1.0]]),
        sigma=np.array([0.1, 0.1]), x0=np.array([0.75, 0.75]), q=np.array([1.0, 1.0]),
        xd=np.zeros((Nt + 1, 2)), lam=float(np.sqrt(beta / np.pi)), jump_law=JUMP_KS,
        jump_scale=float(1.0 / np.sqrt(2.0 * beta)), jump_gain=gamma, nu=1e-2,
        u_min=-np.inf, u_max=np.inf, seed=seed)
    return p, Feedback()


def feedback_trajectory(M: int = 1 << 20, Nt: int = 100, seed: int = 0):
    """(Problem, Feedback) of Sec. 6.3: eta = 0, eps = 0.1, a piecewise-linear target."""
    p, fb = feedback_centering(M=M, Nt=Nt, seed=seed, eta=0.0)
    t = np.linspace(0.0, p.T, Nt + 1)
    xd = np.stack([-fb.x_max / 2 + fb.x_max * t / p.T, fb.v_max / 2 - np.abs(fb.v_max * t / (2 * p.T))], axis=1)
    return p.replace(name="feedback_trajectory", xd=xd), fb.replace(eps=0.1)


def random_mu(p: Problem, fb: Feedback, seed: int = 7, scale: float = 1.0) -> np.ndarray:
    """Seeded feedback weights mu (Nt, L) for gradient tests."""
    return scale * np.random.default_rng(seed).standard_normal((p.Nt, fb.L))


def feedback_coupled(M: int = 1 << 20, Nt: int = 100, seed: int = 0, particles: int = 32):
    """(Problem, Feedback) of Sec. 6.4: rings of `particles` coupled oscillators (eta = 1,
    omega = 0.5) started equidistant on the ellipse A_x = 1.5, A_v = 1.7071067811865475,
    ellipse tracking cost (sigma_J = 1), 10x10 bumps (eps = 0.5), Keilson-Storer resets;
    M = S x realizations, S the ring's lane count (32 for up to 32 particles, the next
    power of two up to 256, then the next multiple of 256; lanes beyond `particles` idle)."""
    p, fb = feedback_centering(M=M, Nt=Nt, seed=seed)
    fb = fb.replace(track=TRACK_ELLIPSE, particles=particles, omega=0.5, ax=1.5, av=1.7071067811865475)
    return p.replace(name="feedback_coupled"), fb
