"""GPU parity at the settings of the MD and NPT workloads: Krylov block order
r = 16 (64 x 64 projected problems), cluster cutoff 6.5 A, clusters of up to
~150 atoms, on 1920-atom cells at a = 12.5 A (L/2 = 12.5 A > Rc), with both
the persistent Krylov + eigensolve queue and separate launches in the mixed
path; the bridged crystal of the uneven-cluster workload at r = 16; and three
mixed-precision velocity-Verlet steps against the oracle's.

Tolerances as in the other parity tests: forces 1e-6 (FP64) / 1e-3 (mixed)
eV/A, band energy 1e-8 / 1e-5 relative.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import density, md
from synth import CONFIGS, fcc_c60_crystal, maxwell_boltzmann_velocities, workload_params

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(F=1e-6, Eb=1e-8), "mixed": dict(F=1e-3, Eb=1e-5)}


@pytest.fixture(scope="module")
def tb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_0910_4497_gb300 as tb
    assert torch.cuda.is_available()
    return tb


def small_cell(k, **over):
    """Configuration k's lattice, cutoff and Krylov order on a 2x2x2 cell."""
    cfg = dict(CONFIGS[k])
    pos, L, _ = fcc_c60_crystal(2, cfg["a"], cfg["jitter"], cfg["seed"], cfg["bridges"])
    p = workload_params(cfg, defl_tol=1e-9)
    p.update(over)
    return pos, L, p


_REF = {}


def reference(key, pos, L, p):
    if key not in _REF:
        _REF[key] = oracle.force_evaluation(pos, L, p, workers=8)
    return _REF[key]


def check(tb, key, pos, L, p, prec, graph=True):
    ref = reference(key, pos, L, p)
    s = tb.TBSystem(len(pos), L, p, prec=prec)
    s.set_positions(pos)
    if graph:
        s.capture()
        s.replay()
    else:
        s.evaluate()
    torch.cuda.synchronize()
    s.check()
    F = s.F.cpu().numpy()
    e = s.energies.cpu().numpy()
    errF = np.abs(F - ref.F).max()
    assert errF <= TOL[prec]["F"], f"{key} {prec}: max |dF| {errF:.3e}"
    assert abs(e[0] - ref.E_band) <= TOL[prec]["Eb"] * abs(ref.E_band)
    lam_all = np.concatenate(ref.lam)
    w_all = np.concatenate([np.sum(S_ * S_, axis=0) for S_ in ref.S])
    n_at = density.electron_count(s.mu.item(), lam_all, w_all, p["kT"])
    assert abs(n_at - 4 * len(pos)) <= (1e-9 if prec == "fp64" else 1e-5) * len(pos)
    if prec == "fp64":
        assert np.array_equal(s.kdim.cpu().numpy(), np.asarray(ref.kdim))
    return s, ref, errF


@pytest.mark.parametrize("prec,schedule", [("fp64", "auto"), ("mixed", "persistent"),
                                           ("mixed", "separate")])
def test_md_settings_r16(tb, prec, schedule):
    pos, L, p = small_cell(4, schedule=schedule)
    s, _, _ = check(tb, "md_r16", pos, L, p, prec)
    sizes = np.diff(s.c_off.cpu().numpy())
    assert sizes.max() > 128 and sizes.max() <= p["max_cluster"]
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bridged_crystal_r16(tb, prec):
    pos, L, p = small_cell(2)
    s, _, _ = check(tb, "bridged_r16", pos, L, p, prec)
    s.close()


def test_mixed_verlet_steps_match_oracle(tb):
    cfg = CONFIGS[0]
    pos, L, _ = fcc_c60_crystal(cfg["ncell"], cfg["a"], cfg["jitter"], cfg["seed"])
    p = workload_params(cfg, defl_tol=1e-9)
    vel = maxwell_boltzmann_velocities(len(pos), 2000.0, 12.011, seed=5)
    s = tb.TBSystem(len(pos), L, p, prec="mixed")
    s.set_positions(pos)
    s.evaluate()
    s.vel.copy_(torch.as_tensor(vel))
    for _ in range(3):
        s.md_step(0.5, 12.011)
    torch.cuda.synchronize()
    s.check()

    def ffn(x):
        r = oracle.force_evaluation(x, L, p)
        return r.F, r.E_total
    x, v = pos.copy(), vel.copy()
    F, _ = ffn(x)
    for _ in range(3):
        x, v, F, epot = md.verlet_step(x, v, F, L, 0.5, 12.011, ffn)
    dx = s.pos.cpu().numpy() - x
    dx -= L * np.rint(dx / L)
    assert np.abs(dx).max() <= 1e-6
    assert np.abs(s.vel.cpu().numpy() - v).max() <= 1e-5
    assert np.abs(s.F.cpu().numpy() - F).max() <= 1e-3
    e = s.energies.cpu().numpy()
    assert abs(e[4] - epot) <= 1e-5 * abs(epot)
    assert abs(e[7] - md.kinetic_energy(v, 12.011)) <= 1e-6 * abs(e[7])
    s.close()
