"""Pins of the oracle in the long-range regime (hoppings of Xu's functional
form reaching a 7.0 A cutoff: the dense-Hamiltonian case of Sec. 5, with the
synthetic constants of synth.TB_CONSTANTS_LONGRANGE): the scaling function's
values and its C1 tail with these constants, the lists against cKDTree at
7.0 A, Gauss-quadrature moment matching on the nearly dense cluster
Hamiltonians, the whole-molecule limit against exact diagonalisation (a 240 x
240 Hamiltonian in which almost every pair couples, the tail region populated),
the force as minus the gradient of the exact energy there, and the truncated
240-atom cell's conservation laws.  CPU only."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
from oracle import model, neighbors, hamiltonian, krylov, exact
from synth import LONGRANGE, TB_CONSTANTS_LONGRANGE, workload_params, fcc_c60_crystal, c60_cage


def lr_params(**kw):
    p = dict(TB_CONSTANTS_LONGRANGE)
    p.update(kT=0.1, Rc=7.0, r=8, defl_tol=1e-9, n_electrons_per_atom=4.0)
    p.update(kw)
    return p


@pytest.fixture(scope="module")
def lr240():
    cfg = LONGRANGE[0]
    pos, L, _ = fcc_c60_crystal(cfg["ncell"], cfg["a"], cfg["jitter"], cfg["seed"])
    return pos, L, workload_params(cfg, defl_tol=1e-9)


def test_longrange_scale_values_and_tail():
    p = lr_params()
    # (r0/r)^2 exp{2[-(r/4)^2 + (r0/4)^2]} with r0 = 1.536, evaluated by hand
    # (math.exp) outside the oracle
    hand = {2.5: 0.23210714215284692, 4.0: 0.02680107037790495,
            5.0: 0.005568661520660238, 6.0: 0.0009777625889285965}
    r = np.array(sorted(hand))
    s, _ = model.hopping_scale(r, p)
    assert np.allclose(s, [hand[x] for x in sorted(hand)], rtol=1e-12, atol=0)
    s0, _ = model.hopping_scale(np.array([p["r0"]]), p)
    assert s0[0] == 1.0
    e = 1e-9
    v, d = model.hopping_scale(np.array([6.5 - e, 6.5 + e, 7.0 - e, 7.0, 7.3]), p)
    # across r1 the value moves by |s'| * 2e ~ 1.5e-12 only: C1 continuity
    assert abs(v[0] - v[1]) < 1e-11 and abs(d[0] - d[1]) < 1e-9
    assert abs(v[2]) < 1e-15 and abs(d[2]) < 1e-9
    assert v[3] == 0.0 and v[4] == 0.0 and d[4] == 0.0
    # the tail decays monotonically from s(r1) to zero
    rt = np.linspace(6.5, 7.0, 101)
    vt, _ = model.hopping_scale(rt, p)
    assert np.all(np.diff(vt) <= 1e-18) and np.all(vt >= -1e-18)
    # the pair repulsion keeps its short range: zero long before the tail
    phi, dphi = model.pair_repulsion(np.array([4.0, 6.6]), p)
    assert phi[0] < 1e-30 and phi[1] == 0.0 and dphi[1] == 0.0


def test_longrange_lists_match_ckdtree(lr240):
    pos, L, p = lr240
    tree = cKDTree(pos, boxsize=L)
    ours = neighbors.neighbor_lists(pos, L, p["rm"])
    ref = tree.query_ball_point(pos, p["rm"])
    sizes = []
    for i in range(len(pos)):
        exp = np.array(sorted(j for j in ref[i] if j != i))
        assert np.array_equal(ours[i], exp)
        sizes.append(len(exp))
    assert 100 < min(sizes) and max(sizes) <= LONGRANGE[0]["max_hnbr"]


def test_longrange_moment_matching(lr240):
    """E_i^T H_c^q E_i = e_1^T T^q e_1 for q < 2r on clusters whose
    Hamiltonians couple most pairs (Gauss quadrature of the block Lanczos)."""
    pos, L, p = lr240
    hl = neighbors.neighbor_lists(pos, L, p["rm"])
    cl = neighbors.cluster_lists(pos, L, p["Rc"])
    bonds = hamiltonian.BondTable(pos, L, hl, p)
    for i in (0, 131):
        Hc = hamiltonian.cluster_hamiltonian(bonds, cl[i])
        dense = np.count_nonzero(np.abs(Hc) > 0) / Hc.size
        assert dense > 0.4
        r = 5
        V, T, _ = krylov.block_lanczos(Hc, r, 1e-9)
        Hp = np.eye(Hc.shape[0])[:, 0:4]
        Tp = np.eye(T.shape[0])[:, 0:4]
        for q in range(2 * r):
            mh, mt = Hp[0:4, :], Tp[0:4, :]
            assert np.allclose(mh, mt, rtol=1e-9, atol=1e-9 * np.abs(mh).max())
            Hp = Hc @ Hp
            Tp = T @ Tp


@pytest.fixture(scope="module")
def molecule_exact():
    pos = c60_cage() + 10.0
    L = 20.0
    p = lr_params(Rc=18.0, r=61)         # every cluster = the whole molecule; r >= 60
    return pos, L, p, oracle.force_evaluation(pos, L, p), exact.whole_cell(pos, L, p)


def test_longrange_whole_molecule_matches_exact_diagonalisation(molecule_exact):
    pos, L, p, res, ex = molecule_exact
    hl = neighbors.neighbor_lists(pos, L, p["rm"])
    d = np.linalg.norm(pos[:, None] - pos[None], axis=-1)
    assert sum(len(h) for h in hl) > 0.9 * 60 * 59          # nearly every pair couples
    assert np.any((d > 6.5) & (d < 7.0))                     # pairs inside the tail
    assert abs(res.n_electrons - 4 * len(pos)) < 1e-9
    assert abs(res.E_band - ex["E_band"]) < 1e-8 * abs(ex["E_band"])
    assert abs(res.E_entropy - ex["E_entropy"]) < 1e-9
    assert np.abs(res.F - ex["F"]).max() < 1e-9


def test_longrange_force_is_minus_gradient_in_exact_limit(molecule_exact):
    pos, L, p, res, ex = molecule_exact
    h = 1e-4

    def energy(x):
        e = exact.whole_cell(x, L, p)
        return e["E_band"] + e["E_entropy"] + e["E_rep"]
    for atom, k in ((0, 0), (29, 2)):
        xp, xm = pos.copy(), pos.copy()
        xp[atom, k] += h
        xm[atom, k] -= h
        fd = -(energy(xp) - energy(xm)) / (2 * h)
        assert abs(fd - res.F[atom, k]) < 2e-6


def test_longrange_cell_conservation(lr240):
    pos, L, p = lr240
    res = oracle.force_evaluation(pos, L, p, workers=4)
    assert abs(res.n_electrons - 4 * len(pos)) < 1e-9 * len(pos)
    assert np.abs(res.F.sum(axis=0)).max() < 1e-9 * len(pos)
    assert all(len(k) == len(c) for k, c in zip(res.klists, neighbors.cluster_lists(pos, L, p["Rc"])))
