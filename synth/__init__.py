"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds workload definitions (structure generators and the constant
tables of each workload) and nothing of the tight-binding method's arithmetic:
no Hamiltonian, no Krylov step, no occupation function.  Both the CPU oracle and
the CUDA path take their inputs from here; neither imports the other.
"""
from .configs import (CONFIGS, DIAMOND_EOS, LONGRANGE, NPT, TB_CONSTANTS,
                      TB_CONSTANTS_LONGRANGE, workload_params)
from .c60 import (c60_cage, fcc_c60_crystal, maxwell_boltzmann_velocities,
                  linear_chain, dimer, diamond_cell)

__all__ = ["CONFIGS", "LONGRANGE", "NPT", "TB_CONSTANTS", "TB_CONSTANTS_LONGRANGE",
           "workload_params", "c60_cage",
           "fcc_c60_crystal", "maxwell_boltzmann_velocities", "linear_chain",
           "dimer", "diamond_cell"]
