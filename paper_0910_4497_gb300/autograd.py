"""torch.autograd.Functions over one force evaluation.

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


class TBLocalEnergy(torch.autograd.Function):
    """The truncated local free energy at r = r_min, A_loc + E_rep, with its
    exact gradient (Daleckii-Krein) as the backward.

    Forward: dense spectra of every cluster Hamiltonian, mu, energies
    (tb_local_forward).  Backward: tb_local_gradient, reading the eigenvectors
    the forward stored when the system was reserved with store_basis=True,
    else recomputing them.  The system holds one forward's state: a second
    forward before this backward makes the backward raise."""

    @staticmethod
    def forward(ctx, pos, system):
        if not isinstance(system, TBSystem):
            raise TypeError("system must be a TBSystem")
        if not hasattr(system, "lam_loc"):
            raise RuntimeError("call system.reserve_local() first")
        with torch.no_grad():
            x = torch.remainder(pos.detach().to(system.pos.device, torch.float64), system.L)
            x = torch.where(x >= system.L, torch.zeros_like(x), x)
            system.pos.copy_(x)
            system.local_forward()
            energy = system.energies_loc[4].clone()
        ctx.system = system
        ctx.version = system.local_version
        return energy.to(pos.dtype)

    @staticmethod
    def backward(ctx, grad_energy):
        system = ctx.system
        if system.local_version != ctx.version:
            raise RuntimeError("the system ran another forward before this backward")
        with torch.no_grad():
            system.local_gradient()
            F = system.F_loc.clone()
        return (-F * grad_energy).to(grad_energy.dtype), None


def local_energy(pos, system):
    """A_loc + E_rep of `pos` (N x 3) with its exact gradient."""
    return TBLocalEnergy.apply(pos, system)
