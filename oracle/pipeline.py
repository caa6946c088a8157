"""One complete oracle force evaluation: lists -> H -> per-target block Krylov
-> eigenpairs -> mu -> energies, density-matrix blocks and forces.

Targets are independent (Sec. 3: the procedure is repeated for each atom), so
the per-target stage may be spread over worker processes (spawned, never
forked); the arithmetic of each target is the same either way.
"""
import multiprocessing as mp
from dataclasses import dataclass, field

import numpy as np

from . import model
from .neighbors import neighbor_lists, cluster_lists
from .hamiltonian import BondTable, cluster_hamiltonian
from .krylov import block_lanczos, spectral_record
from .density import find_mu, band_terms, rho_blocks, forces
from .grouping import group_atoms, krylov_lists


@dataclass
class OracleResult:
    hlists: list
    clists: list
    klists: list = None                         # per target: the atoms its Krylov run spans
    groups: list = None                         # target groups (m-target form), or None
    lam: list = field(default_factory=list)     # per target (kdim,)
    S: list = field(default_factory=list)       # per target (4, kdim)
    P: list = field(default_factory=list)       # per target ((1+z)*4, kdim)
    kdim: np.ndarray = None
    mu: float = None
    n_electrons: float = None
    E_band: float = None
    E_entropy: float = None                     # -TS
    E_rep: float = None
    F: np.ndarray = None
    rho: list = None
    per_atom: dict = None

    @property
    def A(self):
        return self.E_band + self.E_entropy

    @property
    def E_total(self):
        return self.A + self.E_rep


def target_record(bonds, clist, hlist, r, defl_tol):
    """Spectral record (lam, S, P) of one target atom."""
    Hc = cluster_hamiltonian(bonds, clist)
    slot = {int(a): s for s, a in enumerate(clist)}
    nbr_slots = [0] + [slot[int(j)] for j in hlist]
    V, T, _ = block_lanczos(Hc, r, defl_tol)
    return spectral_record(V, T, nbr_slots)


_W = {}


def _init_worker(pos, L, p, hlists, clists):
    _W["bonds"] = BondTable(pos, L, hlists, p)
    _W["hl"], _W["cl"], _W["p"] = hlists, clists, p


def _records_of(targets):
    p = _W["p"]
    return [target_record(_W["bonds"], _W["cl"][i], _W["hl"][i], p["r"],
                          p["defl_tol"]) for i in targets]


def spectral_records(pos, L, p, hlists, clists, targets, bonds=None, workers=1):
    if workers <= 1:
        bonds = bonds if bonds is not None else BondTable(pos, L, hlists, p)
        return [target_record(bonds, clists[i], hlists[i], p["r"], p["defl_tol"])
                for i in targets]
    chunks = np.array_split(np.asarray(targets), workers * 4)
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers, initializer=_init_worker,
                  initargs=(pos, L, p, hlists, clists)) as pool:
        parts = pool.map(_records_of, [list(c) for c in chunks])
    return [rec for part in parts for rec in part]


def force_evaluation(pos, L, p, workers=1, with_forces=True, group_m=1, groups=None):
    """Full evaluation.  `p` needs the model constants plus kT, Rc, r, defl_tol
    and n_electrons_per_atom.  group_m > 1: the m-target form of Eq.
    (lanczos_blas3), each target's Krylov run on its group's union cluster, the
    groups from oracle.grouping.group_atoms unless `groups` (a partition of the
    atoms into lists) is given."""
    pos = np.asarray(pos, dtype=np.float64)
    n = len(pos)
    hl = neighbor_lists(pos, L, p["rm"])
    cl = cluster_lists(pos, L, p["Rc"])
    kl = cl
    if groups is None and group_m > 1:
        groups = group_atoms(pos, L, group_m)
    if groups is not None:
        kl = krylov_lists(cl, groups)
    bonds = BondTable(pos, L, hl, p)
    recs = spectral_records(pos, L, p, hl, kl, range(n), bonds=bonds,
                            workers=workers)
    res = OracleResult(hlists=hl, clists=cl, klists=kl, groups=groups)
    res.lam = [x[0] for x in recs]
    res.S = [x[1] for x in recs]
    res.P = [x[2] for x in recs]
    res.kdim = np.array([len(x) for x in res.lam])
    kT = p["kT"]
    lam_all = np.concatenate(res.lam)
    w_all = np.concatenate([np.sum(S * S, axis=0) for S in res.S])
    ne = p["n_electrons_per_atom"] * n
    res.mu = find_mu(lam_all, w_all, kT, ne)
    eb, ee, nel = band_terms(lam_all, w_all, res.mu, kT)
    res.E_band, res.E_entropy, res.n_electrons = eb, ee, nel
    per = [band_terms(lam, np.sum(S * S, axis=0), res.mu, kT)
           for lam, S in zip(res.lam, res.S)]
    res.per_atom = dict(E_band=np.array([x[0] for x in per]),
                        E_entropy=np.array([x[1] for x in per]),
                        n_el=np.array([x[2] for x in per]))
    r_b = np.sqrt(np.sum(bonds.d * bonds.d, axis=1))
    phi, dphi = model.pair_repulsion(r_b, p)
    res.E_rep = 0.5 * np.sum(phi)
    if with_forces:
        res.rho = [rho_blocks(S, P, lam, res.mu, kT)
                   for S, P, lam in zip(res.S, res.P, res.lam)]
        res.F = forces(bonds, res.rho, hl, dphi)
    res.bonds = bonds
    return res
