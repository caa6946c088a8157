"""Exact O(N^3) references (Sec. 2: the density matrix from the eigenstates of
the whole Hamiltonian; its cost is the reason for the local method).

* whole-cell diagonalisation of the 4N x 4N Gamma-point Hamiltonian:
  rho = U f(E) U^T, mu by the same bisection with unit weight per eigenstate,
  forces from the same pair formula (rho is symmetric here);
* dense diagonalisation of one cluster Hamiltonian H_c: the target's columns
  rho E_i = sum_m f(e_m) m m^T E_i, which the Krylov result must reproduce once
  the block Krylov space is invariant (Sec. 3: r at the minimal-polynomial
  degree).
"""
import numpy as np

from . import model
from .neighbors import neighbor_lists
from .hamiltonian import BondTable, full_hamiltonian, cluster_hamiltonian
from .density import fermi, find_mu, band_terms


def whole_cell(pos, L, p):
    n = len(pos)
    hl = neighbor_lists(pos, L, p["rm"])
    bonds = BondTable(pos, L, hl, p)
    H = full_hamiltonian(bonds)
    eps, U = np.linalg.eigh(H)
    kT = p["kT"]
    w = np.ones_like(eps)
    mu = find_mu(eps, w, kT, p["n_electrons_per_atom"] * n)
    eb, ee, ne = band_terms(eps, w, mu, kT)
    f = fermi((eps - mu) / kT)
    rho = (U * f[None, :]) @ U.T
    r_b = np.sqrt(np.sum(bonds.d * bonds.d, axis=1))
    phi, dphi = model.pair_repulsion(r_b, p)
    F = np.zeros((n, 3))
    for k in range(n):
        for q, j in enumerate(hl[k]):
            b = bonds.off[k] + q
            blk = rho[4 * j:4 * j + 4, 4 * k:4 * k + 4] + rho[4 * k:4 * k + 4, 4 * j:4 * j + 4].T
            F[k] += 2.0 * np.einsum('ba,kab->k', blk, bonds.g[b])
            F[k] += dphi[b] * bonds.d[b] / r_b[b]
    return dict(mu=mu, E_band=eb, E_entropy=ee, n_electrons=ne,
                E_rep=0.5 * np.sum(phi), F=F, eps=eps, rho=rho, hlists=hl)


def cluster_columns(bonds, clist, mu, kT):
    """Dense-diagonalisation columns rho[:, target orbitals] of H_c, plus the
    target's (E_band, -TS, N_e) contributions."""
    Hc = cluster_hamiltonian(bonds, clist)
    eps, U = np.linalg.eigh(Hc)
    f = fermi((eps - mu) / kT)
    cols = (U * f[None, :]) @ U[0:4, :].T          # (4n, 4)
    w = np.sum(U[0:4, :] ** 2, axis=0)
    return cols, band_terms(eps, w, mu, kT)
