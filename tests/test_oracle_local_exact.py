"""Pins of the oracle's exact local gradient (Daleckii-Krein form of the
truncated local free energy at r = r_min) against facts outside it: the
definition of a divided difference (numerical quadrature of the occupation),
central finite differences of the energy it differentiates, the exact
whole-system limit (where it must equal the Hellmann-Feynman force of exact
diagonalisation), the Krylov record at r = r_min, translation and rotation
invariance.  CPU only.
"""
import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import expit
from scipy.stats import special_ortho_group

import oracle
from oracle import exact, local_exact
from synth import TB_CONSTANTS, c60_cage, diamond_cell
from synth.c60 import wrap


def params(**kw):
    p = dict(TB_CONSTANTS)
    p.update(kT=0.1, Rc=2.8, r=20, defl_tol=1e-9, n_electrons_per_atom=4.0)
    p.update(kw)
    return p


def jittered_diamond(seed=7, amp=0.06):
    pos, L = diamond_cell(2)
    pos = pos + amp * np.random.default_rng(seed).standard_normal(pos.shape)
    return wrap(pos, L), L


@pytest.fixture(scope="module")
def diamond_truncated():
    pos, L = jittered_diamond()
    p = params()
    return pos, L, p, local_exact.local_evaluation(pos, L, p)


def test_omega_derivative_is_the_occupation():
    mu, kT = 0.3, 0.1
    x = np.linspace(-3.0, 3.0, 61)
    h = 1e-5
    d = (local_exact.omega(x + h, mu, kT) - local_exact.omega(x - h, mu, kT)) / (2 * h)
    assert np.abs(d - expit(-(x - mu) / kT)).max() < 1e-8
    # deep below mu, omega -> lam - mu; far above, -> 0
    assert abs(local_exact.omega(np.array([mu - 5.0]), mu, kT)[0] - (-5.0)) < 1e-20 + 1e-18
    assert abs(local_exact.omega(np.array([mu + 5.0]), mu, kT)[0]) < 1e-20


def test_loewner_is_the_mean_occupation_over_the_interval():
    mu, kT = -0.2, 0.1
    rng = np.random.default_rng(3)
    lam = np.concatenate([rng.uniform(-1.0, 0.6, 12),
                          [0.05, 0.05 + 3e-5, 0.05 - 2e-6, -0.2, -0.2 + 1e-9]])
    G = local_exact.loewner(lam, mu, kT)
    for m in range(len(lam)):
        for k in range(len(lam)):
            a, b = sorted((lam[m], lam[k]))
            if b - a < 1e-12:
                ref = expit(-(a - mu) / kT)
            else:
                ref = quad(lambda e: expit(-(e - mu) / kT), a, b, epsabs=1e-14,
                           epsrel=1e-13)[0] / (b - a)
            assert abs(G[m, k] - ref) < 1e-11, (m, k, G[m, k], ref)


def test_gradient_matches_central_differences_on_truncated_clusters(diamond_truncated):
    pos, L, p, res = diamond_truncated
    h = 1e-4

    def energy(x):
        return local_exact.local_evaluation(wrap(x, L), L, p, with_forces=False)["E_total"]
    for atom, k in ((0, 0), (9, 1), (33, 2), (50, 0)):
        xp, xm = pos.copy(), pos.copy()
        xp[atom, k] += h
        xm[atom, k] -= h
        fd = -(energy(xp) - energy(xm)) / (2 * h)
        assert abs(fd - res["F"][atom, k]) < 1e-6, (atom, k, fd, res["F"][atom, k])


def test_truncated_gradient_differs_from_hellmann_feynman(diamond_truncated):
    """The clusters really are truncated here: the Hellmann-Feynman force (both
    density-matrix columns of each bond, Krylov at r >= r_min) is not the
    gradient, so the finite-difference pin above discriminates."""
    pos, L, p, res = diamond_truncated
    hf = oracle.force_evaluation(pos, L, p)
    assert max(len(c) for c in res["clists"]) < len(pos)
    assert np.abs(hf.F - res["F"]).max() > 1e-2


def test_energy_equals_krylov_record_at_rmin(diamond_truncated):
    """Sec. 3: with r at the minimal-polynomial degree the Krylov record is the
    dense one, so the band energy and the count agree with the Krylov oracle."""
    pos, L, p, res = diamond_truncated
    kr = oracle.force_evaluation(pos, L, p, with_forces=False)
    assert abs(kr.E_band - res["E_band"]) < 1e-10 * abs(res["E_band"])
    assert abs(kr.E_entropy - res["E_entropy"]) < 1e-10
    assert abs(kr.mu - res["mu"]) < 1e-8


def test_translation_invariance(diamond_truncated):
    _, _, _, res = diamond_truncated
    assert np.abs(res["F"].sum(axis=0)).max() < 1e-10


def test_rotation_covariance_truncated_molecule():
    pos = c60_cage()
    R = special_ortho_group.rvs(3, random_state=11)
    jit = 0.04 * np.random.default_rng(2).standard_normal(pos.shape)
    p = params(Rc=3.0)
    a = local_exact.local_evaluation(pos + jit + 12.0, 24.0, p)
    b = local_exact.local_evaluation((pos + jit) @ R.T + 12.0, 24.0, p)
    assert np.abs(a["F"] @ R.T - b["F"]).max() < 1e-9
    assert abs(a["E_total"] - b["E_total"]) < 1e-9 * abs(a["E_total"])


def test_whole_molecule_limit_equals_exact_hellmann_feynman():
    """Every cluster holds the whole molecule: the seeds of all targets span the
    identity, so the summed Daleckii-Krein gradient is the exact force."""
    pos = c60_cage() + 10.0 + 0.03 * np.random.default_rng(4).standard_normal((60, 3))
    L = 20.0
    p = params(Rc=18.0)
    res = local_exact.local_evaluation(pos, L, p)
    ex = exact.whole_cell(pos, L, p)
    assert abs(res["E_band"] - ex["E_band"]) < 1e-9 * abs(ex["E_band"])
    assert np.abs(res["F"] - ex["F"]).max() < 1e-9


def test_force_restricted_to_touching_targets(diamond_truncated):
    pos, L, p, res = diamond_truncated
    atoms = [3, 40]
    tg = local_exact.targets_touching(res["clists"], atoms)
    part = local_exact.local_evaluation(pos, L, p, targets=tg)
    assert np.abs(part["F"][atoms] - res["F"][atoms]).max() < 1e-12
