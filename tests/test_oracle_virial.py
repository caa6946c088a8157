"""Pins of the oracle's virial and pressure against facts outside it: the
pressure is -dE/dV of the exact whole-cell energy under uniform scaling (central
differences); the repulsive pressure of a perfect diamond lattice has a closed
form over its two bonded shells; the pair form equals the atomic form
sum_k R_k (x) F_k for an isolated molecule; the exact-limit virial is
symmetric.  CPU only."""
import numpy as np
import pytest

import oracle
from oracle import exact, model, virial
from oracle.hamiltonian import BondTable
from oracle.neighbors import neighbor_lists
from synth import TB_CONSTANTS, c60_cage, diamond_cell
from synth.c60 import wrap


def params(**kw):
    p = dict(TB_CONSTANTS)
    p.update(kT=0.1, Rc=5.0, r=8, defl_tol=1e-9, n_electrons_per_atom=4.0)
    p.update(kw)
    return p


def jittered_diamond(a=3.567, seed=3, amp=0.03):
    pos, L = diamond_cell(2, a)
    pos = pos + amp * np.random.default_rng(seed).standard_normal(pos.shape)
    return wrap(pos, L), L


def exact_energy_and_virial(pos, L, p):
    ex = exact.whole_cell(pos, L, p)
    bonds = BondTable(pos, L, neighbor_lists(pos, L, p["rm"]), p)
    return ex["E_band"] + ex["E_entropy"] + ex["E_rep"], virial.exact_virial(ex, bonds, p)


@pytest.mark.parametrize("a", [3.45, 3.567, 3.70])
def test_pressure_is_minus_dE_dV_in_the_exact_limit(a):
    pos, L = jittered_diamond(a)
    p = params()
    _, W = exact_energy_and_virial(pos, L, p)
    P = virial.pressure(W, L)
    h = 1e-5
    Ep, _ = exact_energy_and_virial(pos * (1 + h), L * (1 + h), p)
    Em, _ = exact_energy_and_virial(pos * (1 - h), L * (1 - h), p)
    dV = (L * (1 + h)) ** 3 - (L * (1 - h)) ** 3
    assert abs(P - (-(Ep - Em) / dV)) <= 1e-7 + 1e-6 * abs(P), (a, P, -(Ep - Em) / dV)
    assert np.abs(W - W.T).max() <= 1e-9 * np.abs(W).max()


def test_krylov_virial_equals_exact_in_the_limit():
    pos, L = jittered_diamond()
    p = params(Rc=6.5, r=70)
    res = oracle.force_evaluation(pos, L, p)
    _, Wex = exact_energy_and_virial(pos, L, p)
    assert np.abs(virial.evaluation_virial(res, p) - Wex).max() <= 1e-9 * np.abs(Wex).max()


def test_repulsive_pressure_closed_form_perfect_diamond():
    a = 3.567
    pos, L = diamond_cell(2, a)
    p = params(Vss=0.0, Vsp=0.0, Vpps=0.0, Vppp=0.0, Rc=2.6, r=1)
    res = oracle.force_evaluation(pos, L, p)
    W = virial.evaluation_virial(res, p)
    d1, d2 = np.sqrt(3.0) * a / 4.0, a / np.sqrt(2.0)     # shells inside the 2.6 A cutoff
    _, g = model.pair_repulsion(np.array([d1, d2]), p)
    n = len(pos)
    trW = -n * (2.0 * d1 * g[0] + 6.0 * d2 * g[1])       # 2 and 6 pairs per atom
    assert abs(np.trace(W) - trW) <= 1e-10 * abs(trW)
    assert np.abs(W - np.trace(W) / 3.0 * np.eye(3)).max() <= 1e-10 * abs(trW)
    assert abs(virial.pressure(W, L) - trW / (3.0 * L ** 3)) <= 1e-12 * abs(trW) / L ** 3


def test_pair_form_equals_atomic_form_for_an_isolated_molecule():
    pos = c60_cage() + 12.0 + 0.04 * np.random.default_rng(5).standard_normal((60, 3))
    L = 24.0
    p = params(Rc=3.0, r=6)
    res = oracle.force_evaluation(pos, L, p)
    W = virial.evaluation_virial(res, p)
    Wat = np.einsum('ka,kb->ab', pos, res.F)
    assert np.abs(W - Wat).max() <= 1e-9 * np.abs(W).max()
