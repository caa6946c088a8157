"""Pins of the oracle's m-target form (Sec. 3, Eq. (lanczos_blas3)): the
Morton grouping against hand-derived codes and orders, the union lists against
brute-force set unions, the per-target recursions on the union cluster against
the paper's Level-3 recursion run on all m targets at once, the dense
diagonalisation of the union Hamiltonian, and the whole-molecule limit where
one group's union is the molecule (exact diagonalisation).  CPU only."""
import numpy as np
import pytest

import oracle
from oracle import exact, grouping, hamiltonian, krylov, neighbors, density
from synth import CONFIGS, TB_CONSTANTS, c60_cage, fcc_c60_crystal, workload_params


def base_params(**kw):
    p = dict(TB_CONSTANTS)
    p.update(kT=0.1, Rc=5.0, r=8, defl_tol=1e-9, n_electrons_per_atom=4.0)
    p.update(kw)
    return p


def test_morton_codes_by_hand():
    # x bit b -> 3b, y bit b -> 3b+1, z bit b -> 3b+2
    assert grouping.morton(1, 0, 0) == 1
    assert grouping.morton(0, 1, 0) == 2
    assert grouping.morton(0, 0, 1) == 4
    assert grouping.morton(2, 0, 0) == 8
    assert grouping.morton(3, 3, 3) == 63
    assert grouping.morton(2, 1, 3) == 0b101110          # 46
    assert grouping.morton(1023, 0, 0) == int("001" * 10, 2)
    assert grouping.morton(0, 0, 1023) == int("100" * 10, 2)


def test_grid_cells_by_hand():
    assert grouping.grid_cells(1920, 4) == 7            # 4*343 <= 1920 < 4*512
    assert grouping.grid_cells(240, 4) == 3             # 108 <= 240 < 256
    assert grouping.grid_cells(240, 2) == 4             # 2*64 <= 240 < 2*125
    assert grouping.grid_cells(8, 1) == 2
    assert grouping.grid_cells(7, 1) == 1
    assert grouping.grid_cells(3, 4) == 1
    assert grouping.grid_cells(15360, 4) == 15          # 13500 <= 15360 < 16384


def test_group_order_one_atom_per_cell():
    """Eight atoms, one in each cell of a 2x2x2 grid, listed out of order:
    the Morton order of the cells is (0,0,0) (1,0,0) (0,1,0) (1,1,0) (0,0,1)
    (1,0,1) (0,1,1) (1,1,1)."""
    L = 10.0
    cells = [(1, 1, 1), (0, 0, 0), (1, 0, 1), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 0), (0, 1, 1)]
    pos = (np.array(cells, dtype=float) + 0.5) * (L / 2)
    assert list(grouping.group_order(pos, L, 1)) == [1, 6, 3, 5, 4, 2, 7, 0]
    # m = 2: 2 * 8 > 8, so one cell holds everything and the order is by index
    assert [list(g) for g in grouping.group_atoms(pos, L, 2)] == [[0, 1], [2, 3], [4, 5], [6, 7]]


def test_group_order_ties_and_cell_edges():
    L = 8.0
    # 16 atoms, m = 2 -> g = 2 (2*8 <= 16 < 2*27); cell edge at x = 4 exactly
    pos = np.full((16, 3), 1.0)
    pos[3] = [4.0, 1.0, 1.0]            # (4/8)*2 = 1 -> cell (1,0,0), code 1
    pos[9] = [3.9999999, 1.0, 1.0]      # cell (0,0,0)
    pos[12] = [7.9999999999, 7.9, 7.9]  # cell (1,1,1), code 7, last
    pos[5] = [1.0, 5.0, 1.0]            # cell (0,1,0), code 2
    order = list(grouping.group_order(pos, L, 2))
    rest = [i for i in range(16) if i not in (3, 12, 5)]
    assert order == rest + [3, 5, 12]


def test_groups_partition_the_atoms():
    rng = np.random.default_rng(4)
    L = 12.0
    pos = rng.uniform(0.0, L, size=(50, 3))
    groups = grouping.group_atoms(pos, L, 4)
    assert [len(g) for g in groups] == [4] * 12 + [2]
    allm = np.sort(np.concatenate(groups))
    assert np.array_equal(allm, np.arange(50))


def test_union_lists_brute_force(cfg_small):
    pos, L, p = cfg_small
    cl = neighbors.cluster_lists(pos, L, p["Rc"])
    groups = grouping.group_atoms(pos, L, 4)
    ul = grouping.union_lists(cl, groups)
    kl = grouping.krylov_lists(cl, groups)
    for grp, u in zip(groups, ul):
        s = set()
        for i in grp:
            s |= {int(x) for x in cl[i]}
        assert list(u) == sorted(s)
        for i in grp:
            assert kl[i][0] == i
            assert sorted(int(x) for x in kl[i]) == sorted(s)
            assert list(kl[i][1:]) == sorted(s - {int(i)})


@pytest.fixture(scope="module")
def cfg_small():
    cfg = CONFIGS[0]
    pos, L, _ = fcc_c60_crystal(cfg["ncell"], cfg["a"], cfg["jitter"], cfg["seed"])
    p = workload_params(cfg, defl_tol=1e-9, Rc=3.6, r=6)
    return pos, L, p


def test_m1_grouping_is_the_per_target_method(cfg_small):
    pos, L, p = cfg_small
    a = oracle.force_evaluation(pos, L, p)
    b = oracle.force_evaluation(pos, L, p, group_m=1)
    assert np.array_equal(a.F, b.F) and a.E_band == b.E_band


def level3_recursion(Hc, seeds, steps):
    """The paper's Level-3 recursion for m targets at once, in its block form:
    L_k = H V_k - V_k A_k - V_{k-1} B_{k-1}^T with A_k, B_k block diagonal over
    the targets (4x4 blocks); every target's new block is orthogonalised against
    all of its own earlier blocks (no deflation: the test stays below the
    minimal-polynomial degree).  Returns the per-target T = V^T H V."""
    m = len(seeds)
    D = Hc.shape[0]
    V = np.zeros((D, 4 * m))
    for t, s in enumerate(seeds):
        V[4 * s:4 * s + 4, 4 * t:4 * t + 4] = np.eye(4)
    hist = [V]
    for _ in range(steps - 1):
        Lk = Hc @ hist[-1]                   # one product for all m targets
        Vn = np.zeros_like(V)
        for t in range(m):
            cols = slice(4 * t, 4 * t + 4)
            w = Lk[:, cols]
            Q = np.concatenate([h[:, cols] for h in hist], axis=1)
            for _ in range(2):
                w = w - Q @ (Q.T @ w)
            q, r = np.linalg.qr(w)
            Vn[:, cols] = q * np.sign(np.diag(r))[None, :]
        hist.append(Vn)
    T = []
    for t in range(m):
        cols = slice(4 * t, 4 * t + 4)
        Vt = np.concatenate([h[:, cols] for h in hist], axis=1)
        T.append(Vt.T @ Hc @ Vt)
    return T


def test_per_target_runs_equal_the_level3_recursion(cfg_small):
    """Each target's block Lanczos on its group's union cluster spans the same
    space, with the same T up to the sign of each basis column, as the paper's
    m-target recursion on the shared union Hamiltonian."""
    pos, L, p = cfg_small
    hl = neighbors.neighbor_lists(pos, L, p["rm"])
    cl = neighbors.cluster_lists(pos, L, p["Rc"])
    bonds = hamiltonian.BondTable(pos, L, hl, p)
    groups = grouping.group_atoms(pos, L, 4)
    ul = grouping.union_lists(cl, groups)
    kl = grouping.krylov_lists(cl, groups)
    steps = 4
    for q in (0, 17, 41):
        grp, u = groups[q], ul[q]
        Hu = hamiltonian.cluster_hamiltonian(bonds, u)
        slot = {int(a): s for s, a in enumerate(u)}
        T3 = level3_recursion(Hu, [slot[int(i)] for i in grp], steps)
        for t, i in enumerate(grp):
            Hk = hamiltonian.cluster_hamiltonian(bonds, kl[i])
            V, T, widths = krylov.block_lanczos(Hk, steps, p["defl_tol"])
            assert widths == [4] * steps
            # same Krylov space: equal spectra of T (the bases differ by signs)
            assert np.allclose(np.linalg.eigvalsh(T), np.linalg.eigvalsh(T3[t]), atol=1e-10)


def test_dense_limit_of_the_union_cluster(cfg_small):
    """Once r reaches the union's minimal-polynomial degree, a target's density
    columns are those of the dense union Hamiltonian (not of its own cluster)."""
    pos, L, p = cfg_small
    hl = neighbors.neighbor_lists(pos, L, p["rm"])
    cl = neighbors.cluster_lists(pos, L, p["Rc"])
    bonds = hamiltonian.BondTable(pos, L, hl, p)
    groups = grouping.group_atoms(pos, L, 4)
    kl = grouping.krylov_lists(cl, groups)
    mu, kT = 4.5, p["kT"]
    for i in (int(groups[3][1]), int(groups[30][2])):
        assert len(kl[i]) > len(cl[i])
        Hc = hamiltonian.cluster_hamiltonian(bonds, kl[i])
        V, T, _ = krylov.block_lanczos(Hc, len(kl[i]) + 1, 1e-9)
        lam, U = np.linalg.eigh(T)
        f = density.fermi((lam - mu) / kT)
        cols = V @ ((U * f) @ U[0:4, :].T)
        ref, _ = exact.cluster_columns(bonds, kl[i], mu, kT)
        assert np.allclose(cols, ref, atol=1e-10)
        own, _ = exact.cluster_columns(bonds, cl[i], mu, kT)
        assert np.abs(cols[0:4] - own[0:4]).max() > 1e-6      # the target's on-site block


def test_one_group_spanning_the_molecule_is_exact():
    """Isolated C60 with a 3.0 A cluster cutoff (each cluster ~7 atoms): with
    m = 60 every target shares one group whose union is the whole molecule, so
    at r = 61 the result is the exact diagonalisation, which the per-target
    method at the same cutoff is far from."""
    pos = c60_cage() + 10.0
    L = 20.0
    p = base_params(Rc=3.0, r=61)
    res = oracle.force_evaluation(pos, L, p, group_m=60)
    assert len(res.groups) == 1 and all(len(k) == 60 for k in res.klists)
    ex = exact.whole_cell(pos, L, p)
    assert abs(res.E_band - ex["E_band"]) < 1e-8 * abs(ex["E_band"])
    assert abs(res.E_entropy - ex["E_entropy"]) < 1e-9
    assert np.abs(res.F - ex["F"]).max() < 1e-9
    per_target = oracle.force_evaluation(pos, L, base_params(Rc=3.0, r=8))
    assert np.abs(per_target.F - ex["F"]).max() > 1e-3
