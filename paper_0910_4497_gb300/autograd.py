"""torch.autograd.Function over one force evaluation.

Forward: the Mermin free energy plus repulsion, A + E_rep (the variational
quantity at kT > 0), computed by the C-ABI pipeline for the positions given.
Backward: the hand-written force kernels' output, dE/dR = -F (Sec. 2,
<F> = Tr[rho F]).  That is the exact gradient when every cluster contains the
whole system and the Krylov space is invariant; for truncated clusters it is
the Hellmann-Feynman force of the local method.
"""
import torch

from .system import TBSystem


class TBEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, system):
        if not isinstance(system, TBSystem):
            raise TypeError("system must be a TBSystem")
        with torch.no_grad():
            x = torch.remainder(pos.detach().to(system.pos.device, torch.float64), system.L)
            x = torch.where(x >= system.L, torch.zeros_like(x), x)
            system.pos.copy_(x)
            system.evaluate()
            energy = system.energies[4].clone()
            forces = system.F.clone()
        ctx.save_for_backward(forces)
        return energy.to(pos.dtype)

    @staticmethod
    def backward(ctx, grad_energy):
        (forces,) = ctx.saved_tensors
        return (-forces * grad_energy).to(grad_energy.dtype), None


def energy(pos, system):
    """A + E_rep of `pos` (N x 3) with gradient -F."""
    return TBEnergy.apply(pos, system)
