"""Edge cases of the call sequence on the GPU.

* n = 0: the list, assembly, Krylov and force stages return without work and
  leave the status clear; the mu search refuses it (there are no electrons).
* A ragged atom count (the 240-atom cell without its first atom, n = 239:
  odd, and a multiple of none of the block or batch sizes), in both
  precisions and through the persistent Krylov + eigensolve queue, whose last
  eigensolve pair then holds one target: forces and energies against the
  oracle at the parity tolerances.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import CONFIGS, fcc_c60_crystal, workload_params

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(F=1e-6, Eb=1e-8), "mixed": dict(F=1e-3, Eb=1e-5)}


@pytest.fixture(scope="module")
def tb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_0910_4497_gb300 as tb
    assert torch.cuda.is_available()
    return tb


def cell0():
    cfg = CONFIGS[0]
    pos, L, _ = fcc_c60_crystal(cfg["ncell"], cfg["a"], cfg["jitter"], cfg["seed"])
    return pos, L, workload_params(cfg, defl_tol=1e-9)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_empty_input(tb, prec):
    pos, L, p = cell0()
    s = tb.TBSystem(len(pos), L, p, prec=prec)
    B = tb.binding
    B.tb_build_neighbors(s.ctx, 0, s.pos, L, s.h_off, s.h_idx, s.c_off, s.c_idx)
    B.tb_assemble_H(s.ctx, 0, s.pos, L, s.h_off, s.h_idx, s.Hblk, s.dHblk, s.Hsk)
    B.tb_krylov_density(s.ctx, 0, s.c_off, s.c_idx, s.h_off, s.h_idx, s.Hblk, s.Hsk, s.lam,
                        s.S, s.P, s.kdim)
    B.tb_forces(s.ctx, 0, s.pos, L, s.h_off, s.h_idx, s.dHblk, s.lam, s.S, s.P, s.kdim, s.mu,
                s.F, s.energies)
    with pytest.raises(B.TBError):
        B.tb_find_mu(s.ctx, 0, s.lam, s.S, s.kdim, 0.0, None, s.mu)
    torch.cuda.synchronize()
    assert tuple(s.status()) == (0, 0)
    s.close()


@pytest.fixture(scope="module")
def ragged():
    pos, L, p = cell0()
    pos = np.ascontiguousarray(pos[1:])
    return pos, L, p, oracle.force_evaluation(pos, L, p, workers=8)


@pytest.mark.parametrize("prec,schedule", [("fp64", "auto"), ("mixed", "persistent"),
                                           ("mixed", "separate")])
def test_ragged_atom_count(tb, ragged, prec, schedule):
    pos, L, p, ref = ragged
    assert len(pos) == 239
    s = tb.TBSystem(len(pos), L, dict(p, schedule=schedule), prec=prec)
    s.set_positions(pos)
    s.capture()
    s.replay()
    torch.cuda.synchronize()
    s.check()
    F = s.F.cpu().numpy()
    e = s.energies.cpu().numpy()
    tol = TOL[prec]
    assert np.abs(F - ref.F).max() <= tol["F"]
    assert abs(e[0] - ref.E_band) <= tol["Eb"] * abs(ref.E_band)
    assert abs(e[5] - 4 * s.n) <= 1e-9 * s.n
    assert np.abs(F.sum(axis=0)).max() <= 1e-9 * s.n
    s.close()
