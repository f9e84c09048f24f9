"""torch.autograd.Function over the discrete adjoint: J(theta) = an observable at T (kinetic energy
or mixing-layer width) of the Kelvin-Helmholtz samples with perturbation parameters theta;
backward returns grad_output[:, None] * dJ/dtheta computed by the hand-written adjoint kernels (the
gradient is produced together with J in forward, so backward only scales it)."""
from __future__ import annotations

import torch


class KHObservable(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, solver, T, observable):
        J, grad = solver.adjoint(theta.detach(), T, observable)
        solver.stream.synchronize()
        ctx.save_for_backward(grad.to(theta.device))
        return J.to(theta.device, theta.dtype)

    @staticmethod
    def backward(ctx, gJ):
        (grad,) = ctx.saved_tensors
        return (gJ.to(grad.dtype)[:, None] * grad).to(gJ.dtype), None, None, None


def kinetic_energy(theta, solver, T):
    """Differentiable kinetic energy J(theta) at T for a solver configured for the adjoint (2D Euler
    KH, periodic, PC/MC + Rusanov, SSP-RK2/RK3)."""
    return KHObservable.apply(theta, solver, T, "ke")


def mixing_width(theta, solver, T):
    """Differentiable mixing-layer width sum 4 (rho - 1)(2 - rho) dV at T (same solver setup)."""
    return KHObservable.apply(theta, solver, T, "mixing")


