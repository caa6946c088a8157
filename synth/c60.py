"""Seeded synthetic structures: fcc C60 crystals, a linear chain and a dimer.

Geometry only.  Conventions:

* A C60 cage is a truncated icosahedron obtained by cutting every edge of an
  icosahedron of edge 4.30 A at a fraction t = 1.45/4.30 from each end.  The
  cut points are the 60 atoms; pentagon bonds are 1.45 A and hexagon-hexagon
  bonds 1.40 A; cage radius ~3.55 A.
* Cells are cubic, periodic, side L = ncell * a; positions are wrapped into
  [0, L).  Molecules sit on fcc sites (0,0,0), (0,1/2,1/2), (1/2,0,1/2),
  (1/2,1/2,0) * a of each cubic cell, cells ordered (ix, iy, iz) with iz
  fastest, then the four basis sites, then the 60 cage atoms.
* Random draws use numpy.random.default_rng(seed) in this order: one unit
  quaternion per molecule (4 normals, normalised), then N x 3 normal jitters,
  then the bridge choices, then (separately) velocities.
"""
import numpy as np

PHI = (1.0 + 5.0 ** 0.5) / 2.0
ICOSA_EDGE = 4.30            # A; gives 1.45 / 1.40 A bonds with the cut below
CUT = 1.45 / 4.30            # fraction of each icosahedron edge cut off per end


def _icosahedron(edge):
    v = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            v.append((0.0, s1, s2 * PHI))
            v.append((s1, s2 * PHI, 0.0))
            v.append((s2 * PHI, 0.0, s1))
    v = np.array(v) * (edge / 2.0)
    edges = []
    for a in range(12):
        for b in range(a + 1, 12):
            if abs(np.linalg.norm(v[a] - v[b]) - edge) < 1e-9:
                edges.append((a, b))
    assert len(edges) == 30
    return v, edges


def c60_cage():
    """60 x 3 cage coordinates centred at the origin (ideal truncated icosahedron)."""
    v, edges = _icosahedron(ICOSA_EDGE)
    atoms = []
    for a, b in edges:
        atoms.append(v[a] + CUT * (v[b] - v[a]))
        atoms.append(v[b] + CUT * (v[a] - v[b]))
    return np.array(atoms)


def _quat_to_rot(q):
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def wrap(pos, L):
    """Wrap coordinates into [0, L)."""
    y = np.mod(pos, L)
    y[y >= L] = 0.0
    return y


def _min_image(d, L):
    return d - L * np.rint(d / L)


def _add_bridges(pos, centers, L, frac, rng):
    """Push the closest atom pair of a random `frac` of nearest-neighbour
    molecule pairs to a U(1.55, 1.65) A separation (sp3-like inter-cage bonds)."""
    nmol = len(centers)
    dc = _min_image(centers[None, :, :] - centers[:, None, :], L)
    rc = np.sqrt((dc * dc).sum(-1))
    nn = rc[rc > 1e-6].min()
    pairs = [(m1, m2) for m1 in range(nmol) for m2 in range(m1 + 1, nmol)
             if abs(rc[m1, m2] - nn) < 1e-6]
    k = int(round(frac * len(pairs)))
    order = rng.permutation(len(pairs))[:k]
    targets = rng.uniform(1.55, 1.65, size=k)
    used = np.zeros(len(pos), dtype=bool)
    nbridges = 0
    for sel, dist in zip(order, targets):
        m1, m2 = pairs[sel]
        a = pos[60 * m1:60 * m1 + 60]
        b = pos[60 * m2:60 * m2 + 60]
        d = _min_image(b[None, :, :] - a[:, None, :], L)
        r = np.sqrt((d * d).sum(-1))
        ia, ib = np.unravel_index(np.argmin(r), r.shape)
        ga, gb = 60 * m1 + ia, 60 * m2 + ib
        if used[ga] or used[gb]:
            continue
        u = d[ia, ib] / r[ia, ib]
        mid = pos[ga] + 0.5 * d[ia, ib]
        pos[ga] = mid - 0.5 * dist * u
        pos[gb] = mid + 0.5 * dist * u
        used[ga] = used[gb] = True
        nbridges += 1
    return nbridges


def fcc_c60_crystal(ncell, a, jitter, seed, bridges=0.0):
    """Seeded fcc C60 supercell.  Returns (pos[N,3] float64, L, info dict)."""
    rng = np.random.default_rng(seed)
    cage = c60_cage()
    basis = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]]) * a
    centers = []
    for ix in range(ncell):
        for iy in range(ncell):
            for iz in range(ncell):
                for b in basis:
                    centers.append(np.array([ix, iy, iz]) * a + b)
    centers = np.array(centers)
    L = ncell * a
    quats = rng.standard_normal((len(centers), 4))
    mols = []
    for c, q in zip(centers, quats):
        q = q / np.linalg.norm(q)
        mols.append(cage @ _quat_to_rot(q).T + c)
    pos = np.concatenate(mols, axis=0)
    pos = pos + jitter * rng.standard_normal(pos.shape)
    pos = wrap(pos, L)
    nb = 0
    if bridges > 0.0:
        nb = _add_bridges(pos, centers, L, bridges, rng)
        pos = wrap(pos, L)
    return pos, L, dict(n_molecules=len(centers), bridges=nb, centers=centers)


def maxwell_boltzmann_velocities(n, T_kelvin, mass_amu, seed, kB=8.617333262e-5,
                                 acc_conv=9.648533e-3):
    """Velocities in A/fs from a Maxwell-Boltzmann draw at T; centre of mass at rest."""
    rng = np.random.default_rng(seed)
    sigma = np.sqrt(kB * T_kelvin / mass_amu * acc_conv)
    v = sigma * rng.standard_normal((n, 3))
    return v - v.mean(axis=0)


def linear_chain(n_atoms, spacing, box=None):
    """Atoms on a line along x with the given spacing; periodic ring of n_atoms
    along x inside a cubic box of side n_atoms * spacing (or `box`)."""
    L = n_atoms * spacing if box is None else box
    pos = np.zeros((n_atoms, 3))
    pos[:, 0] = (np.arange(n_atoms) + 0.5) * spacing
    pos[:, 1] = 0.5 * L
    pos[:, 2] = 0.5 * L
    return pos, L


def dimer(r, box=20.0, axis=(0.0, 0.0, 1.0)):
    """Two atoms separated by r along `axis`, centred in a cubic box."""
    u = np.asarray(axis, dtype=float)
    u = u / np.linalg.norm(u)
    c = np.full(3, 0.5 * box)
    pos = np.stack([c - 0.5 * r * u, c + 0.5 * r * u])
    return pos, box


def diamond_cell(ncell, a=3.567):
    """Cubic diamond supercell (8 atoms per cubic cell), side L = ncell * a."""
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    basis = np.concatenate([fcc, fcc + 0.25]) * a
    pos = []
    for ix in range(ncell):
        for iy in range(ncell):
            for iz in range(ncell):
                pos.append(basis + np.array([ix, iy, iz]) * a)
    L = ncell * a
    return wrap(np.concatenate(pos), L), L
