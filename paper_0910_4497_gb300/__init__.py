"""GB300 (sm_103a) linear-scaling tight-binding forces: local block-Krylov
density-matrix columns per target atom, global chemical potential, pair
Hellmann-Feynman forces and velocity-Verlet MD, behind the C ABI of
include/tb.h.  The Python layer only marshals arguments; importing the package
loads libtb.so and raises if it has not been built.
"""
from . import binding
from .binding import (TBParams, TBError, make_params, tb_ctx_create, tb_ctx_destroy,
                      tb_ctx_reserve, tb_ctx_workspace_bytes, tb_get_status,
                      tb_build_neighbors, tb_assemble_H, tb_krylov_density, tb_find_mu,
                      tb_forces, tb_md_step, tb_virial, tb_ctx_reserve_local, tb_local_forward,
                      tb_local_gradient, tb_version)
from .system import TBSystem
from .autograd import TBEnergy, TBLocalEnergy, energy, local_energy

binding.lib()   # fail loudly now if the CUDA library is missing

__all__ = ["TBParams", "TBError", "make_params", "tb_ctx_create", "tb_ctx_destroy",
           "tb_ctx_reserve", "tb_ctx_workspace_bytes", "tb_get_status",
           "tb_build_neighbors", "tb_assemble_H", "tb_krylov_density", "tb_find_mu",
           "tb_forces", "tb_md_step", "tb_virial", "tb_ctx_reserve_local", "tb_local_forward",
           "tb_local_gradient", "tb_version", "TBSystem", "TBEnergy", "TBLocalEnergy",
           "energy", "local_energy"]
