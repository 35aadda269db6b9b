"""torch.autograd interface to the polarization solve and the permanent-multipole energy.

``polarization_energy(solver, xyz, q, dip, quad, alpha, thole, mol)`` returns
the polarization energy (kcal/mol, 0-dim float64 CUDA tensor). Its backward is
the hand-written adjoint of the CUDA library (``amp_forces``): because the
energy is stationary in the induced dipoles, the gradients are evaluated at
the converged dipoles with no second solve. Gradients flow to xyz (= -forces),
q, dip and quad; alpha, thole and mol are parameters without gradients.

``multipole_energy(solver, xyz, q, dip, quad, alpha, thole, mol)`` returns the
energy of the permanent multipoles with each other (``amp_multipole_energy``);
its forward call computes the gradients too, and backward scales them. The
gradient with respect to quad is projected onto traceless changes (the mean
of the three diagonal entries removed).
"""
from __future__ import annotations

import torch

from .amoebapol import Polarization


class _PolarizationEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xyz, q, dip, quad, solver, alpha, thole, mol):
        solver.set_system(xyz.detach(), q.detach(), dip.detach(), quad.detach(), alpha, thole, mol)
        E0 = solver.permanent_field()
        mu, it, rms = solver.solve(E0)
        U = solver.energy(mu, E0)
        ctx.solver = solver
        ctx.inputs = (xyz.detach(), q.detach(), dip.detach(), quad.detach(), alpha, thole, mol)
        ctx.generation = solver.generation
        ctx.save_for_backward(mu)
        ctx.info = (it, rms)
        return torch.tensor(U, dtype=torch.float64, device=xyz.device)

    @staticmethod
    def backward(ctx, grad_u):
        (mu,) = ctx.saved_tensors
        solver = ctx.solver
        if solver.generation != ctx.generation:
            solver.set_system(*ctx.inputs)  # geometry state replaced since forward
        F, gq, gd, gt = solver.forces(mu)
        g = grad_u.to(torch.float64)
        return (-F * g, gq * g, gd * g, gt * g, None, None, None, None)


def polarization_energy(solver: Polarization, xyz, q, dip, quad, alpha, thole, mol):
    """Differentiable polarization energy of one system (see module doc)."""
    return _PolarizationEnergy.apply(xyz, q, dip, quad, solver, alpha, thole, mol)


class _MultipoleEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xyz, q, dip, quad, solver, alpha, thole, mol):
        solver.set_system(xyz.detach(), q.detach(), dip.detach(), quad.detach(), alpha, thole, mol)
        U, F, gq, gd, gt = solver.multipole_energy()
        ctx.save_for_backward(F, gq, gd, gt)
        return torch.tensor(U, dtype=torch.float64, device=xyz.device)

    @staticmethod
    def backward(ctx, grad_u):
        F, gq, gd, gt = ctx.saved_tensors
        g = grad_u.to(torch.float64)
        return (-F * g, gq * g, gd * g, gt * g, None, None, None, None)


def multipole_energy(solver: Polarization, xyz, q, dip, quad, alpha, thole, mol):
    """Differentiable permanent-multipole energy of one system (see module doc)."""
    return _MultipoleEnergy.apply(xyz, q, dip, quad, solver, alpha, thole, mol)
