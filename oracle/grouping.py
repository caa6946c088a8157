"""Groups of m target atoms for the m-target (Level-3) form of the recursion,
Sec. 3, Eq. (lanczos_blas3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper rearranges the N atoms into small groups of m atoms and runs the m
recursions of a group together: L_k = H V_k - A_k V_k - B_{k-1} V_{k-1} with
V_k holding one column per target and A_k, B_k diagonal over the targets.  The
targets' recursions therefore stay independent; only the matrix H multiplying
them is shared.  With the four-orbital block seed each target contributes a
4-column block and A_k, B_k become block diagonal with 4x4 blocks.

Readings (the paper states neither):
* the shared H of a group is the Hamiltonian of the union of its targets'
  clusters, so each target's spectral record is the block Krylov space of its
  own four orbitals in that union cluster (with m = 1 this is the per-target
  method);
* the groups are spatially compact runs of a Morton (Z-order) curve: a grid of
  g x g x g cells, g the largest integer with m g^3 <= N (about m atoms per
  cell, g <= 1024); the cell of an atom is c = floor((x / L) * g) per
  component (each operation rounded separately, clamped to [0, g-1]); its
  Morton code puts bit b of c_x, c_y, c_z at bits 3b, 3b+1, 3b+2; the atoms are
  sorted by (code, index) and cut into consecutive groups of m (the last group
  holds the remainder).
"""
import numpy as np

MAX_GRID = 1024


def grid_cells(n, m):
    """Largest g >= 1 with m g^3 <= n (capped at 1024)."""
    g = 1
    while g < MAX_GRID and m * (g + 1) ** 3 <= n:
        g += 1
    return g


def morton(cx, cy, cz):
    """Bit interleave of three 10-bit cell coordinates (x in the lowest bit)."""
    code = 0
    for b in range(10):
        code |= ((cx >> b) & 1) << (3 * b)
        code |= ((cy >> b) & 1) << (3 * b + 1)
        code |= ((cz >> b) & 1) << (3 * b + 2)
    return code


def atom_cells(pos, L, g):
    c = np.floor((np.asarray(pos, dtype=np.float64) / L) * g).astype(np.int64)
    return np.clip(c, 0, g - 1)


def group_order(pos, L, m):
    """Atoms sorted by (Morton code of their cell, index)."""
    n = len(pos)
    g = grid_cells(n, m)
    c = atom_cells(pos, L, g)
    codes = np.array([morton(int(x), int(y), int(z)) for x, y, z in c], dtype=np.int64)
    return np.lexsort((np.arange(n), codes))


def group_atoms(pos, L, m):
    """List of int arrays: consecutive runs of m atoms along the Morton order."""
    order = group_order(pos, L, m)
    return [order[q:q + m] for q in range(0, len(order), m)]


def union_lists(clists, groups):
    """Per group: the ascending union of its members' cluster lists."""
    return [np.unique(np.concatenate([np.asarray(clists[i]) for i in grp])) for grp in groups]


def krylov_lists(clists, groups):
    """Per target i: i first, then the rest of its group's union cluster ascending
    (the same convention as a per-target cluster list)."""
    out = [None] * len(clists)
    for grp, u in zip(groups, union_lists(clists, groups)):
        for i in grp:
            out[int(i)] = np.concatenate([[int(i)], u[u != i]]).astype(np.int64)
    return out
