"""Pins of the FP64 oracle against facts fixed outside the oracle itself:
textbook Slater-Koster limits, rotation covariance, finite differences,
the paper's uniform-chain closed form (Sec. 3), a dimer solved by symmetry,
exact diagonalisation limits (Sec. 2 / Sec. 3 minimal polynomial), Gauss
quadrature moment matching, library routines (expit, brentq, cKDTree), and
conservation laws.  CPU only.
"""
import os
from math import comb

import numpy as np
import pytest
from scipy.optimize import brentq
from scipy.special import expit
from scipy.spatial import cKDTree
from scipy.stats import special_ortho_group

import oracle
from oracle import model, neighbors, hamiltonian, krylov, density, exact
from synth import (CONFIGS, TB_CONSTANTS, workload_params, fcc_c60_crystal,
                   linear_chain, dimer, c60_cage, diamond_cell)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def base_params(**kw):
    p = dict(TB_CONSTANTS)
    p.update(kT=0.1, Rc=5.0, r=8, defl_tol=1e-9, n_electrons_per_atom=4.0)
    p.update(kw)
    return p


def chain_params(**kw):
    # four decoupled uniform chains with t = 1 (Sec. 3 example)
    return base_params(Es=0.0, Ep=0.0, Vss=1.0, Vsp=0.0, Vpps=1.0, Vppp=1.0, **kw)


@pytest.fixture(scope="module")
def cfg0():
    cfg = CONFIGS[0]
    pos, L, _ = fcc_c60_crystal(cfg["ncell"], cfg["a"], cfg["jitter"], cfg["seed"])
    p = workload_params(cfg, defl_tol=1e-9)
    return pos, L, p


@pytest.fixture(scope="module")
def cfg0_result(cfg0):
    pos, L, p = cfg0
    return oracle.force_evaluation(pos, L, p)


# ---------------------------------------------------------------- model (Eq. 1)

def test_scale_is_one_at_r0_and_c1_tail():
    p = base_params()
    s, _ = model.hopping_scale(np.array([p["r0"]]), p)
    assert s[0] == 1.0
    for fn in (model.hopping_scale, model.pair_repulsion):
        r1, rm = p["r1"], p["rm"]
        e = 1e-9
        v, d = fn(np.array([r1 - e, r1 + e, rm - e, rm, rm + 0.1]), p)
        assert abs(v[0] - v[1]) < 1e-7 and abs(d[0] - d[1]) < 1e-6
        assert abs(v[2]) < 1e-12 and abs(d[2]) < 1e-7
        assert v[3] == 0.0 and v[4] == 0.0 and d[4] == 0.0


def test_scale_power_law_limit():
    # rc -> infinity removes the exponential: s(r) -> (r0/r)^n exactly.
    p = base_params(rc=1e9, r1=10.0, rm=11.0)
    r = np.array([1.2, 1.536, 2.0, 2.5])
    s, ds = model.hopping_scale(r, p)
    assert np.allclose(s, (1.536 / r) ** 2, rtol=1e-12)
    assert np.allclose(ds, -2.0 * 1.536 ** 2 / r ** 3, rtol=1e-9)


@pytest.mark.parametrize("fn", [model.hopping_scale, model.pair_repulsion])
def test_scale_derivative_fd(fn):
    p = base_params()
    r = np.array([1.3, 1.45, 1.9, 2.3, 2.44, 2.47, 2.55])
    h = 1e-5
    v, d = fn(r, p)
    fd = (fn(r + h, p)[0] - fn(r - h, p)[0]) / (2 * h)
    assert np.allclose(d, fd, rtol=1e-7, atol=1e-9)


def test_sk_textbook_axis():
    p = base_params()
    r = 1.42
    s, _ = model.hopping_scale(np.array([r]), p)
    t = model.sk_block([0.0, 0.0, r], p) / s[0]
    expect = np.array([[p["Vss"], 0, 0, p["Vsp"]],
                       [0, p["Vppp"], 0, 0],
                       [0, 0, p["Vppp"], 0],
                       [-p["Vsp"], 0, 0, p["Vpps"]]])
    assert np.allclose(t, expect, atol=1e-14)


def test_sk_rotation_covariance_and_symmetry():
    p = base_params()
    rng = np.random.default_rng(7)
    d = np.array([0.9, -0.7, 0.8])
    t = model.sk_block(d, p)
    g = model.sk_block_grad(d, p)
    for _ in range(5):
        R = special_ortho_group.rvs(3, random_state=rng)
        D = np.eye(4)
        D[1:, 1:] = R
        assert np.allclose(model.sk_block(R @ d, p), D @ t @ D.T, atol=1e-13)
        gr = model.sk_block_grad(R @ d, p)
        grot = np.einsum('kl,lab->kab', R, np.einsum('ai,lij,bj->lab', D, g, D))
        assert np.allclose(gr, grot, atol=1e-12)
    # Hermiticity of the pair: t(-d) = t(d)^T
    assert np.allclose(model.sk_block(-d, p), t.T, atol=1e-15)


def test_sk_gradient_fd():
    p = base_params()
    for d in ([0.9, -0.7, 0.8], [1.5, 0.2, -0.1], [0.1, 2.1, 1.3]):
        d = np.array(d)
        g = model.sk_block_grad(d, p)
        h = 1e-6
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            fd = (model.sk_block(d + e, p) - model.sk_block(d - e, p)) / (2 * h)
            assert np.allclose(g[k], fd, atol=1e-8)


# ---------------------------------------------------------------- lists

def test_neighbor_lists_match_ckdtree(cfg0):
    pos, L, p = cfg0
    tree = cKDTree(pos, boxsize=L)
    for R in (p["rm"], p["Rc"]):
        ours = neighbors.neighbor_lists(pos, L, R)
        ref = tree.query_ball_point(pos, R)
        for i in range(len(pos)):
            exp = np.array(sorted(j for j in ref[i] if j != i))
            assert np.array_equal(ours[i], exp)
            assert np.all(np.diff(ours[i]) > 0)
    cl = neighbors.cluster_lists(pos, L, p["Rc"])
    assert all(c[0] == i for i, c in enumerate(cl))


# ---------------------------------------------------------------- Sec. 3 chain

def _chain_system(n=24, **kw):
    p = chain_params(**kw)
    pos, L = linear_chain(n, p["r0"])
    hl = neighbors.neighbor_lists(pos, L, p["rm"])
    bonds = hamiltonian.BondTable(pos, L, hl, p)
    return pos, L, p, hl, bonds


def test_chain_krylov_vectors_match_paper_binomials():
    pos, L, p, hl, bonds = _chain_system()
    H = hamiltonian.full_hamiltonian(bonds)
    n = len(pos)
    rows = np.loadtxt(os.path.join(GOLDEN, "chain_krylov_binomial.txt"))
    v = np.zeros(4 * n)
    v[0] = 1.0                                   # |0>, s orbital of atom 0
    vecs = [v]
    for _ in range(8):
        vecs.append(H @ vecs[-1])
    for r in range(9):
        expect = np.zeros(4 * n)
        for rr, site, c in rows:
            if int(rr) == r:
                expect[4 * (int(site) % n)] = c
        assert np.allclose(vecs[r], expect, atol=1e-12)


def test_chain_lanczos_coefficients_and_moments():
    pos, L, p, hl, bonds = _chain_system()
    cl = neighbors.cluster_lists(pos, L, 12.0)     # open chain of 15 sites
    Hc = hamiltonian.cluster_hamiltonian(bonds, cl[0])
    r = 6
    V, T, widths = krylov.block_lanczos(Hc, r, 1e-9)
    assert widths == [4] * r
    for k in range(r):
        A = T[4 * k:4 * k + 4, 4 * k:4 * k + 4]
        assert np.allclose(A, 0.0, atol=1e-13)
        if k + 1 < r:
            B = T[4 * k + 4:4 * k + 8, 4 * k:4 * k + 4]
            beta = np.sqrt(2.0) if k == 0 else 1.0
            assert np.allclose(B, beta * np.eye(4), atol=1e-13)
    # seed moments <0|H^2p|0> = C(2p, p) (the |0> coefficient of the chain
    # formula), odd moments zero, exact up to order 2r-1 (Gauss quadrature)
    Tp = np.eye(T.shape[0])
    for q in range(2 * r):
        m = Tp[0:4, 0:4]
        expect = comb(q, q // 2) if q % 2 == 0 else 0.0
        assert np.allclose(m, expect * np.eye(4), atol=1e-9 * max(1, expect))
        Tp = Tp @ T


def test_chain_half_filling_gives_mu_zero():
    pos, L, p, hl, bonds = _chain_system(n=24, Rc=8.0, r=5)
    res = oracle.force_evaluation(pos, L, p)
    assert abs(res.mu) < 1e-12
    assert np.allclose(res.per_atom["n_el"], 4.0, atol=1e-12)
    assert np.abs(res.F).max() < 1e-10


def test_chain_p_block_deflates():
    pos, L, p, hl, bonds = _chain_system()
    p = dict(p, Vpps=0.0, Vppp=0.0)
    bonds = hamiltonian.BondTable(pos, L, hl, p)
    cl = neighbors.cluster_lists(pos, L, 12.0)
    Hc = hamiltonian.cluster_hamiltonian(bonds, cl[0])
    V, T, widths = krylov.block_lanczos(Hc, 6, 1e-9)
    assert widths == [4, 1, 1, 1, 1, 1]
    assert np.allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-13)


# ---------------------------------------------------------------- dimer

def test_dimer_closed_form():
    p = base_params()
    r = 1.45
    pos, L = dimer(r)
    s = model.hopping_scale(np.array([r]), p)[0][0]
    Es, Ep = p["Es"], p["Ep"]
    ss, sp, pps, ppp = p["Vss"] * s, p["Vsp"] * s, p["Vpps"] * s, p["Vppp"] * s

    def two(a, d, b):
        m, h = 0.5 * (a + d), np.sqrt((0.5 * (a - d)) ** 2 + b * b)
        return [m - h, m + h]
    expect = sorted(two(Es + ss, Ep - pps, -sp) + two(Es - ss, Ep + pps, sp)
                    + [Ep - ppp, Ep - ppp, Ep + ppp, Ep + ppp])
    hl = neighbors.neighbor_lists(pos, L, p["rm"])
    bonds = hamiltonian.BondTable(pos, L, hl, p)
    eps = np.linalg.eigvalsh(hamiltonian.full_hamiltonian(bonds))
    assert np.allclose(eps, expect, atol=1e-12)
    cl = neighbors.cluster_lists(pos, L, 5.0)
    V, T, widths = krylov.block_lanczos(hamiltonian.cluster_hamiltonian(bonds, cl[0]), 3, 1e-9)
    assert widths == [4, 4]
    assert np.allclose(np.linalg.eigvalsh(T), expect, atol=1e-12)


# ---------------------------------------------------------------- Krylov exactness

def test_moment_matching_cfg0(cfg0):
    pos, L, p = cfg0
    hl = neighbors.neighbor_lists(pos, L, p["rm"])
    cl = neighbors.cluster_lists(pos, L, p["Rc"])
    bonds = hamiltonian.BondTable(pos, L, hl, p)
    for i in (0, 77, 239):
        Hc = hamiltonian.cluster_hamiltonian(bonds, cl[i])
        r = 5
        V, T, _ = krylov.block_lanczos(Hc, r, 1e-9)
        assert np.allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-12)
        Hp = np.eye(Hc.shape[0])[:, 0:4]
        Tp = np.eye(T.shape[0])[:, 0:4]
        for q in range(2 * r):
            mh = Hp[0:4, :]
            mt = Tp[0:4, :]
            assert np.allclose(mh, mt, rtol=1e-9, atol=1e-9 * np.abs(mh).max())
            Hp = Hc @ Hp
            Tp = T @ Tp


def test_dense_cluster_limit(cfg0):
    """At r >= minimal-polynomial degree the Krylov columns equal dense eigh."""
    pos, L, p = cfg0
    hl = neighbors.neighbor_lists(pos, L, p["rm"])
    cl = neighbors.cluster_lists(pos, L, p["Rc"])
    bonds = hamiltonian.BondTable(pos, L, hl, p)
    mu, kT = 4.5, p["kT"]
    for i in (3, 150):
        Hc = hamiltonian.cluster_hamiltonian(bonds, cl[i])
        V, T, widths = krylov.block_lanczos(Hc, len(cl[i]) + 1, 1e-9)
        lam, U = np.linalg.eigh(T)
        f = density.fermi((lam - mu) / kT)
        cols = V @ ((U * f) @ U[0:4, :].T)
        ref, terms = exact.cluster_columns(bonds, cl[i], mu, kT)
        assert np.allclose(cols, ref, atol=1e-10)
        w = np.sum(U[0:4, :] ** 2, axis=0)
        assert np.allclose(density.band_terms(lam, w, mu, kT), terms, atol=1e-10)


def _isolated_c60():
    pos = c60_cage() + 10.0
    return pos, 20.0


@pytest.fixture(scope="module")
def c60_exact_limit():
    pos, L = _isolated_c60()
    p = base_params(Rc=18.0, r=61)        # every cluster = whole molecule; r >= 60
    return pos, L, p, oracle.force_evaluation(pos, L, p), exact.whole_cell(pos, L, p)


def test_whole_molecule_limit_matches_exact_diagonalisation(c60_exact_limit):
    pos, L, p, res, ex = c60_exact_limit
    assert abs(res.mu - ex["mu"]) < 1e-6   # mu sits in the gap: compare counts instead
    assert abs(res.n_electrons - 4 * len(pos)) < 1e-9
    assert abs(res.E_band - ex["E_band"]) < 1e-8 * abs(ex["E_band"])
    assert abs(res.E_entropy - ex["E_entropy"]) < 1e-9
    assert np.abs(res.F - ex["F"]).max() < 1e-9


def test_whole_periodic_cell_limit_diamond():
    pos, L = diamond_cell(2)
    p = base_params(Rc=6.5, r=70)
    pos = pos + 0.03 * np.random.default_rng(3).standard_normal(pos.shape)
    pos = np.mod(pos, L)
    res = oracle.force_evaluation(pos, L, p)
    ex = exact.whole_cell(pos, L, p)
    assert abs(res.E_band - ex["E_band"]) < 1e-8 * abs(ex["E_band"])
    assert np.abs(res.F - ex["F"]).max() < 1e-9


def test_force_is_minus_gradient_in_exact_limit(c60_exact_limit):
    """Central differences of the Mermin free energy plus repulsion (mu
    re-solved at fixed N) equal the Hellmann-Feynman force."""
    pos, L, p, res, ex = c60_exact_limit
    h = 1e-4

    def energy(x):
        e = exact.whole_cell(x, L, p)
        return e["E_band"] + e["E_entropy"] + e["E_rep"]
    for atom, k in ((0, 0), (17, 1), (42, 2)):
        xp, xm = pos.copy(), pos.copy()
        xp[atom, k] += h
        xm[atom, k] -= h
        fd = -(energy(xp) - energy(xm)) / (2 * h)
        assert abs(fd - res.F[atom, k]) < 2e-6


# ---------------------------------------------------------------- truncated cfg0

def test_newton_third_law_and_count(cfg0_result, cfg0):
    pos, L, p = cfg0
    res = cfg0_result
    assert np.abs(res.F.sum(axis=0)).max() < 1e-11
    assert abs(res.n_electrons - 4 * len(pos)) < 1e-9 * len(pos)
    assert abs(res.per_atom["n_el"].sum() - 4 * len(pos)) < 1e-9 * len(pos)


def test_energy_identity_checks_neighbour_rows(cfg0_result, cfg0):
    """sum_m f lam w = sum_a (H rho)_{ia,ia}: the Krylov residual is orthogonal
    to the seed, so the neighbour rows P must reproduce the band energy."""
    pos, L, p = cfg0
    res = cfg0_result
    b = res.bonds
    for i in (0, 5, 100, 239):
        f = density.fermi((res.lam[i] - res.mu) / p["kT"])
        w = np.sum(res.S[i] ** 2, axis=0)
        lhs = np.sum(f * res.lam[i] * w)
        R = res.rho[i]
        rhs = np.trace(b.onsite @ R[0])
        for q, j in enumerate(res.hlists[i]):
            rhs += np.trace(b.t[b.off[i] + q] @ R[1 + q])
        assert abs(lhs - rhs) < 1e-11


def test_axis_and_index_permutation_covariance(cfg0_result, cfg0):
    pos, L, p = cfg0
    res = cfg0_result
    perm_axes = [1, 2, 0]
    r2 = oracle.force_evaluation(pos[:, perm_axes], L, p)
    assert np.abs(r2.F - res.F[:, perm_axes]).max() < 1e-9
    rng = np.random.default_rng(11)
    perm = rng.permutation(len(pos))
    r3 = oracle.force_evaluation(pos[perm], L, p)
    assert np.abs(r3.F - res.F[perm]).max() < 1e-9
    assert abs(r3.E_band - res.E_band) < 1e-9 * abs(res.E_band)


# ---------------------------------------------------------------- occupations

def test_fermi_and_entropy_against_library_and_grand_potential():
    x = np.linspace(-60, 60, 1201)
    assert np.allclose(density.fermi(x), expit(-x), rtol=1e-14, atol=1e-300)
    rng = np.random.default_rng(5)
    lam = rng.uniform(-10, 10, 200)
    w = rng.uniform(0, 1, 200)
    mu, kT = 0.3, 0.1
    eb, ee, ne = density.band_terms(lam, w, mu, kT)
    # Omega = E - TS - mu N = 2 sum w omega(lam), omega = -kT ln(1 + e^{-(lam-mu)/kT})
    omega = -kT * np.logaddexp(0.0, -(lam - mu) / kT)
    assert abs((eb + ee - mu * ne) - 2.0 * np.sum(w * omega)) < 1e-10


def test_mu_bisection_against_brentq():
    rng = np.random.default_rng(9)
    lam = rng.uniform(-12, 8, 400)
    w = rng.uniform(0, 1, 400)
    kT = 0.1
    ne = 0.6 * 2 * w.sum()
    mu = density.find_mu(lam, w, kT, ne)
    ref = brentq(lambda m: density.electron_count(m, lam, w, kT) - ne,
                 lam.min() - 5, lam.max() + 5, xtol=1e-15, rtol=1e-15)
    assert abs(mu - ref) < 1e-12
