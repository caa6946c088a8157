"""Virial stress and pressure of the pair-decomposed forces (used for the
equation of state of diamond, Sec. 5).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Reading (the paper computes the pressure of a diamond supercell but does not
say how): every force of the method is a sum over directed bonds k -> j,
F_k = sum_{j in H(k)} f_kj, with the bond term

  f_kj = 2 sum_{a,b} [rho^(k)_{j b, k a} + rho^(j)_{k a, j b}] dH_ab/dd + phi'(r) d / r,
  d = R_j - R_k (minimum image),

and f_jk = -f_kj.  The configurational virial is then the pair form

  W = sum_k R_k (x) F_k = -1/2 sum_{directed bonds} d (x) f_kj     (eV),

which is defined under periodic boundaries, and the static pressure is
P = tr W / (3V); a kinetic term 2 KE / (3V) is added for a moving system.
When every cluster is complete the forces are the exact gradient of the
energy, and P = -dE/dV under uniform scaling of the cell and its contents.

Library primitives used as single steps: numpy.einsum.
"""
import numpy as np

from . import model


def bond_forces(bonds, rho, hlists, rep_der):
    """f_kj for every directed bond (same order as the bond table), n_bonds x 3."""
    nb = len(bonds.src)
    f = np.zeros((nb, 3))
    for k in range(bonds.n):
        for q, j in enumerate(hlists[k]):
            b = bonds.off[k] + q
            rq = int(np.searchsorted(hlists[j], k))
            R_sum = rho[k][1 + q] + rho[j][1 + rq].T       # [b, a]
            f[b] = 2.0 * np.einsum('ba,kab->k', R_sum, bonds.g[b])
            r = np.sqrt(bonds.d[b] @ bonds.d[b])
            f[b] += rep_der[b] * bonds.d[b] / r
    return f


def virial(bonds, f):
    """W_ab = -1/2 sum over directed bonds of d_a f_b."""
    return -0.5 * np.einsum('pa,pb->ab', bonds.d, f)


def evaluation_virial(res, p):
    """Virial of an oracle.force_evaluation result (its bonds, rho, lists)."""
    r_b = np.sqrt(np.sum(res.bonds.d * res.bonds.d, axis=1))
    _, dphi = model.pair_repulsion(r_b, p)
    f = bond_forces(res.bonds, res.rho, res.hlists, dphi)
    return virial(res.bonds, f)


def exact_virial(ex, bonds, p):
    """Virial of the whole-cell exact density matrix (oracle.exact.whole_cell),
    from the same pair formula with rho the full symmetric matrix."""
    rho = ex["rho"]
    r_b = np.sqrt(np.sum(bonds.d * bonds.d, axis=1))
    _, dphi = model.pair_repulsion(r_b, p)
    f = np.zeros((len(bonds.src), 3))
    for b in range(len(bonds.src)):
        k, j = int(bonds.src[b]), int(bonds.dst[b])
        blk = rho[4 * j:4 * j + 4, 4 * k:4 * k + 4] + rho[4 * k:4 * k + 4, 4 * j:4 * j + 4].T
        f[b] = 2.0 * np.einsum('ba,kab->k', blk, bonds.g[b]) + dphi[b] * bonds.d[b] / r_b[b]
    return virial(bonds, f)


def pressure(W, L, kinetic=0.0):
    """(tr W + 2 KE) / (3 V) in eV/A^3."""
    return (np.trace(W) + 2.0 * kinetic) / (3.0 * L ** 3)


EV_PER_A3_IN_GPA = 160.21766208
