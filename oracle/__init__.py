"""FP64 CPU oracle of the linear-scaling tight-binding force evaluation.

TEST INFRASTRUCTURE ONLY.  Only the tests, the package entry point's smoke
check and the benchmark's CPU-baseline leg may import this package.  The
product path (the CUDA library and its Python binding) never imports it, and it
imports nothing from the product path.

It is a plain, slow, readable restatement of the method in NumPy float64,
following the paper's steps in order:

* Eq. (1): orthogonal sp3 tight-binding Hamiltonian (``model``),
* Sec. 2: locality - each target atom sees only the atoms within the cutoff
  radius (``neighbors``, ``hamiltonian``),
* Sec. 3, Eq. (Krylov) and the block form of Eq. (lanczos_blas3): block Krylov
  space seeded with the target atom's four orbitals, block Lanczos with full
  reorthogonalisation, the projected matrix T = V^T H V and its eigenpairs
  (``krylov``), and its m-target Level-3 form on the union cluster of a
  group of targets (``grouping``),
* Sec. 2: density matrix rho = sum_m |m> f(e_m) <m| and the force
  <F_i> = Tr[rho F_i] (``density``),
* plus the velocity-Verlet step of the MD workload (``md``), the exact
  O(N^3) whole-cell diagonalisation used as a limit check (``exact``), and
  the exact gradient of the truncated local free energy at r = r_min
  (``local_exact``).

Library primitives used as single steps: numpy matmul, numpy.linalg.eigh.
"""
from . import model, neighbors, hamiltonian, krylov, density, md, exact, local_exact, virial, grouping  # noqa: F401
from .pipeline import force_evaluation, OracleResult  # noqa: F401
