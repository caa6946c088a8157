"""Neighbour and cluster lists by brute force over all atom pairs.

Sec. 2 (locality): each target atom's local problem contains only the atoms
within the cutoff radius of that atom.  Two lists are built in a periodic cubic
box of side L:

* the Hamiltonian list: j != i with |R_j - R_i| <= rm (the hopping cutoff,
  2.6 A for Xu's parameters, Sec. 5), ascending j;
* the cluster list: the target i first, then every j != i with
  |R_j - R_i| <= Rc, ascending j.

Distance test (the definition the lists must reproduce bit for bit):
d = R_j - R_i per component, then the nearest periodic image: d - L if
d > L/2, d + L if d < -L/2, else d (positions lie in [0, L), so one shift
suffices; a separation of exactly half a box keeps its sign);
r2 = (dx*dx + dy*dy) + dz*dz with every operation rounded separately (no fused
multiply-add); the pair is in iff r2 <= R*R.
"""
import numpy as np


def minimum_image(d, L):
    h = 0.5 * L
    return np.where(d > h, d - L, np.where(d < -h, d + L, d))


def pair_r2(pos, i, L):
    d = minimum_image(pos - pos[i], L)
    return (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]


def neighbor_lists(pos, L, R):
    """List of int arrays: for each i, ascending j != i with r_ij <= R."""
    pos = np.asarray(pos, dtype=np.float64)
    R2 = R * R
    out = []
    for i in range(len(pos)):
        r2 = pair_r2(pos, i, L)
        sel = np.nonzero(r2 <= R2)[0]
        out.append(sel[sel != i])
    return out


def cluster_lists(pos, L, Rc):
    """List of int arrays: for each i, [i] followed by ascending j != i, r_ij <= Rc."""
    return [np.concatenate([[i], nb]).astype(np.int64)
            for i, nb in enumerate(neighbor_lists(pos, L, Rc))]


def to_csr(lists):
    off = np.zeros(len(lists) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(x) for x in lists])
    idx = np.concatenate(lists) if len(lists) else np.zeros(0, np.int64)
    return off, idx.astype(np.int64)
