"""Global periodic Hamiltonian of Eq. (1) in 4x4 blocks and the cluster
Hamiltonian H_c of one target atom.

H_c is the principal submatrix of the minimum-image (Gamma-point) Hamiltonian
on the atoms of the target's cluster (Sec. 2: only atoms within the cutoff
radius of the target are taken into account), orbitals ordered atom-major
(cluster slot), then s, px, py, pz.
"""
import numpy as np

from . import model
from .neighbors import minimum_image


class BondTable:
    """Directed bonds i -> j (j in the Hamiltonian list of i) with their
    hopping blocks t (4x4) and gradients dt/dd (3x4x4), d = R_j - R_i."""

    def __init__(self, pos, L, hlists, p):
        self.n = len(pos)
        self.hlists = hlists
        self.off = np.zeros(self.n + 1, dtype=np.int64)
        self.off[1:] = np.cumsum([len(h) for h in hlists])
        nb = int(self.off[-1])
        self.src = np.zeros(nb, dtype=np.int64)
        self.dst = np.zeros(nb, dtype=np.int64)
        self.d = np.zeros((nb, 3))
        self.t = np.zeros((nb, 4, 4))
        self.g = np.zeros((nb, 3, 4, 4))
        for i in range(self.n):
            for q, j in enumerate(hlists[i]):
                b = self.off[i] + q
                d = minimum_image(pos[j] - pos[i], L)
                self.src[b], self.dst[b], self.d[b] = i, j, d
                self.t[b] = model.sk_block(d, p)
                self.g[b] = model.sk_block_grad(d, p)
        self.onsite = model.onsite_block(p)

    def block_index(self, i, j):
        """Row-block position of j in i's list, or -1."""
        h = self.hlists[i]
        q = np.searchsorted(h, j)
        return int(self.off[i] + q) if q < len(h) and h[q] == j else -1


def cluster_hamiltonian(bonds, cluster):
    """Dense H_c (4n x 4n) on the atoms `cluster` (slot order as given)."""
    n = len(cluster)
    slot = {int(a): s for s, a in enumerate(cluster)}
    H = np.zeros((n, 4, n, 4))
    for s, a in enumerate(cluster):
        H[s, :, s, :] = bonds.onsite
        for q, b in enumerate(bonds.hlists[a]):
            t = slot.get(int(b))
            if t is not None:
                H[s, :, t, :] = bonds.t[bonds.off[a] + q]
    return H.reshape(4 * n, 4 * n)


def full_hamiltonian(bonds):
    """Dense 4N x 4N Gamma-point Hamiltonian of the whole periodic cell."""
    return cluster_hamiltonian(bonds, np.arange(bonds.n))
