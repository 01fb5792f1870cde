"""torch.autograd form of the reduced cost: J(u, theta) whose backward is the adjoint kernel.

The forward pass is jd_forward (the forward sweep, keeping the stored states or the
checkpoints of the recompute plan on the device), the backward pass is jd_backward (the
backward sweep of the discrete adjoint, Sec. 4 eq:AdjointModel and Sec. 5.5
eq:adjoint_eq_approximation, with the cross-path reductions of eq:definition_Gradient).
Nothing is computed in Python: this module moves parameters into the problem and
composes the kernel's parameter derivatives by the chain rule.

Parameters theta = (rho, s_sigma, s_jump) act on a base problem as

    A(theta)          = A_base + rho * dA        (a drift coefficient along the direction dA)
    sigma(theta)      = s_sigma * sigma_shape     (diffusion scale; sigma_shape = 1 for a
                                                   scalar sigma shared by all components)
    jump_scale(theta) = s_jump                    (std of NORMAL / half-width of UNIFORM sizes)

and the library returns, for the current coefficients, dJ/dtheta_A along dA, dJ/dsigma_i
per component and dJ/djump_scale, so that

    dJ/drho = g_A,   dJ/ds_sigma = sum_i sigma_shape_i g_sigma_i,   dJ/ds_jump = g_jump.

The jump intensity lambda is not pathwise differentiable (the Poisson count jumps) and is
not a parameter here.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from .binding import JdProblem


def theta_problem(base, A_base, sigma_shape, theta):
    """The problem at theta = (rho, s_sigma, s_jump): a copy of ``base`` (a workloads
    Problem with dA set) with A, sigma and jump_scale replaced."""
    rho, s_sigma, s_jump = (float(v) for v in theta)
    return dataclasses.replace(
        base, A=np.asarray(A_base, dtype=np.float64) + rho * np.asarray(base.dA, dtype=np.float64),
        sigma=s_sigma * np.asarray(sigma_shape, dtype=np.float64), jump_scale=s_jump)


def compose_theta_grad(grad_theta, sigma_shape):
    """(dJ/drho, dJ/ds_sigma, dJ/ds_jump) from the library's d+2 parameter derivatives
    [along dA, sigma_0 .. sigma_{d-1}, jump scale] (numpy or torch, same layout)."""
    d = len(sigma_shape)
    if isinstance(grad_theta, torch.Tensor):
        shape = torch.as_tensor(np.asarray(sigma_shape, dtype=np.float64), device=grad_theta.device)
        return torch.stack([grad_theta[0], (grad_theta[1:1 + d] * shape).sum(), grad_theta[d + 1]])
    g = np.asarray(grad_theta, dtype=np.float64)
    return np.array([g[0], float(np.dot(g[1:1 + d], sigma_shape)), g[d + 1]])


class _CostFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, theta, owner):
        owner._move_to(theta)
        J = torch.empty(1, dtype=torch.float64, device=u.device)
        owner.problem.forward_into(u.detach().contiguous().view(-1), J)
        owner._forwards += 1
        ctx.owner, ctx.eval_id = owner, owner._forwards
        ctx.theta_values = owner._theta
        ctx.save_for_backward(u.detach())
        return J.view(())

    @staticmethod
    def backward(ctx, gJ):
        owner = ctx.owner
        (u,) = ctx.saved_tensors
        if owner._forwards != ctx.eval_id or owner._theta != ctx.theta_values:
            # another evaluation replaced the kept states: redo this one's forward sweep
            owner._move_to(ctx.theta_values)
            owner.problem.forward_into(u.contiguous().view(-1), torch.empty(1, dtype=torch.float64,
                                                                             device=u.device))
            owner._forwards += 1
            ctx.eval_id = owner._forwards
        g = torch.empty(u.numel(), dtype=torch.float64, device=u.device)
        gth = torch.empty(owner.problem.d + 2, dtype=torch.float64, device=u.device)
        owner.problem.backward_into(g, gth)
        dtheta = compose_theta_grad(gth, owner.sigma_shape)
        return (gJ * g).view_as(u), (gJ * dtheta).to(owner._theta_device), None


class JumpDiffusionCost:
    """J(u, theta) as a differentiable torch function on the current CUDA device.

    ``base``: a workloads Problem with the direction dA set; ``A_base`` is A at rho = 0
    (default: base.A - rho0 dA for the rho0 given); ``sigma_shape`` defaults to ones
    (scalar sigma).  ``mode`` "recompute" keeps only checkpoints (the sqrt(Nt)-style
    checkpointing of the no-storage variant), "stored" keeps every X_k.

    Call with u (CUDA float64, shape (Nt, du)) and theta (float64 tensor of 3 entries,
    any device; its values are read on the host at each call).  Returns J as a 0-d CUDA
    tensor; J.backward() runs the adjoint kernel.
    """

    def __init__(self, base, A_base=None, rho0: float = 0.0, sigma_shape=None, prec="fp32",
                 mode="recompute", stream=None, mem_budget: int = 0):
        if base.dA is None:
            raise ValueError("the base problem needs a drift direction dA")
        self.base = base
        self.A_base = (np.asarray(base.A, dtype=np.float64) - rho0 * np.asarray(base.dA, dtype=np.float64)
                       if A_base is None else np.asarray(A_base, dtype=np.float64))
        self.sigma_shape = np.ones(base.d) if sigma_shape is None else np.asarray(sigma_shape, np.float64)
        self.problem = JdProblem(base, prec=prec, mode=mode, stream=stream, mem_budget=mem_budget)
        self._theta = None
        self._theta_device = torch.device("cpu")
        self._forwards = 0

    def _move_to(self, theta):
        if isinstance(theta, torch.Tensor):
            self._theta_device = theta.device
            values = tuple(float(v) for v in theta.detach().cpu().tolist())
        else:
            values = tuple(float(v) for v in theta)
        if len(values) != 3:
            raise ValueError("theta has three entries (rho, s_sigma, s_jump)")
        if values != self._theta:
            self.problem.update(theta_problem(self.base, self.A_base, self.sigma_shape, values))
            self._theta = values

    def __call__(self, u: torch.Tensor, theta: torch.Tensor) -> torch.Tensor:
        if not (u.is_cuda and u.dtype == torch.float64):
            raise ValueError("u must be a CUDA float64 tensor")
        return _CostFn.apply(u, theta, self)

    def close(self):
        self.problem.close()
