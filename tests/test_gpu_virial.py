"""GPU parity of the virial and pressure (tb_virial) through the C ABI against
the oracle's pair-form virial, on the 240-atom C60 cell and on the 4x4x4
diamond supercell of the equation-of-state workload, and after an MD step
(the context's own lists)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import virial
from synth import CONFIGS, DIAMOND_EOS, TB_CONSTANTS, diamond_cell, fcc_c60_crystal, workload_params

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-8, "mixed": 1e-4}      # relative to max |W|


@pytest.fixture(scope="module")
def tb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_0910_4497_gb300 as tb
    assert torch.cuda.is_available()
    return tb


def gpu_virial(tb, pos, L, p, prec):
    s = tb.TBSystem(len(pos), L, p, prec=prec)
    s.set_positions(pos)
    s.evaluate(with_virial=True)
    torch.cuda.synchronize()
    s.check()
    W = s.W.view(3, 3).cpu().numpy()
    P = s.pressure.item()
    E = s.energies.cpu().numpy()
    s.close()
    return W, P, E


@pytest.fixture(scope="module")
def c60_ref():
    cfg = CONFIGS[0]
    pos, L, _ = fcc_c60_crystal(cfg["ncell"], cfg["a"], cfg["jitter"], cfg["seed"])
    p = workload_params(cfg, defl_tol=1e-9)
    res = oracle.force_evaluation(pos, L, p)
    return pos, L, p, virial.evaluation_virial(res, p)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_virial_c60_cell(tb, c60_ref, prec):
    pos, L, p, Wref = c60_ref
    W, P, _ = gpu_virial(tb, pos, L, p, prec)
    scale = np.abs(Wref).max()
    assert np.abs(W - Wref).max() <= TOL[prec] * scale, np.abs(W - Wref).max() / scale
    assert abs(P - virial.pressure(Wref, L)) <= TOL[prec] * scale / L ** 3


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pressure_diamond_eos_cell(tb, prec):
    a = 3.55
    pos, L = diamond_cell(DIAMOND_EOS["ncell"], a)
    p = dict(TB_CONSTANTS)
    p.update(kT=DIAMOND_EOS["kT"], Rc=DIAMOND_EOS["Rc_over_a"] * a, r=DIAMOND_EOS["r"],
             max_hnbr=DIAMOND_EOS["max_hnbr"], max_cluster=DIAMOND_EOS["max_cluster"],
             n_electrons_per_atom=4.0, defl_tol=1e-9)
    res = oracle.force_evaluation(pos, L, p)
    Wref = virial.evaluation_virial(res, p)
    W, P, E = gpu_virial(tb, pos, L, p, prec)
    scale = np.abs(Wref).max()
    assert np.abs(W - Wref).max() <= TOL[prec] * scale
    # perfect cubic lattice: isotropic virial
    assert np.abs(W - np.trace(W) / 3 * np.eye(3)).max() <= TOL[prec] * scale
    assert abs(E[4] - res.E_total) <= (1e-8 if prec == "fp64" else 1e-5) * abs(res.E_total)


def test_virial_after_md_step_uses_the_context_lists(tb):
    from synth import maxwell_boltzmann_velocities
    cfg = CONFIGS[0]
    pos, L, _ = fcc_c60_crystal(cfg["ncell"], cfg["a"], cfg["jitter"], cfg["seed"])
    p = workload_params(cfg, defl_tol=1e-9)
    s = tb.TBSystem(len(pos), L, p, prec="fp64")
    s.set_positions(pos)
    s.vel.copy_(torch.as_tensor(maxwell_boltzmann_velocities(len(pos), 2000.0, 12.011, 5)))
    s.evaluate()
    s.md_step(0.5, 12.011)
    W = torch.zeros(9, dtype=torch.float64, device="cuda")
    tb.binding.tb_virial(s.ctx, s.n, s.pos, s.L, None, None, W)
    torch.cuda.synchronize()
    s.check()
    W_md = W.view(3, 3).cpu().numpy()
    x = s.pos.cpu().numpy()
    s.close()
    W2, _, _ = gpu_virial(tb, x, L, p, "fp64")
    assert np.abs(W_md - W2).max() <= 1e-9 * np.abs(W2).max()
