"""Autograd over the force evaluation: gradient = -F from the force kernels,
checked against central finite differences of the energy in the limit where the
method is exact (every cluster holds the whole molecule, block order at the
minimal-polynomial degree), and against the oracle's force there."""
import numpy as np
import pytest
import torch

import oracle
from synth import TB_CONSTANTS, diamond_cell

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_0910_4497_gb300 as tb
    return tb


def small_molecule():
    # 8 atoms of a diamond cell in a large box: an isolated, distorted cluster
    pos, _ = diamond_cell(1)
    rng = np.random.default_rng(21)
    pos = pos[:8] + 6.0 + 0.05 * rng.standard_normal((8, 3))
    return pos, 16.0


def test_autograd_gradient_matches_fd_in_exact_limit(tb):
    pos, L = small_molecule()
    p = dict(TB_CONSTANTS, kT=0.1, Rc=7.9, r=8, defl_tol=1e-9, n_electrons_per_atom=4.0,
             max_cluster=16)
    s = tb.TBSystem(len(pos), L, p, prec="fp64")
    x = torch.tensor(pos, dtype=torch.float64, device="cuda", requires_grad=True)
    e = tb.energy(x, s)
    (g,) = torch.autograd.grad(e, x)
    s.check()
    ref = oracle.force_evaluation(pos, L, p)
    assert np.abs(-g.cpu().numpy() - ref.F).max() <= 1e-6
    h = 1e-4
    for atom, k in ((0, 0), (3, 1), (6, 2)):
        xp, xm = pos.copy(), pos.copy()
        xp[atom, k] += h
        xm[atom, k] -= h
        ep = tb.energy(torch.tensor(xp, device="cuda"), s).item()
        em = tb.energy(torch.tensor(xm, device="cuda"), s).item()
        fd = (ep - em) / (2 * h)
        assert abs(fd - g[atom, k].item()) <= 2e-6, (atom, k, fd, g[atom, k].item())
    s.close()


def test_autograd_energy_is_free_energy_plus_repulsion(tb):
    pos, L = small_molecule()
    p = dict(TB_CONSTANTS, kT=0.1, Rc=7.9, r=8, defl_tol=1e-9, n_electrons_per_atom=4.0,
             max_cluster=16)
    s = tb.TBSystem(len(pos), L, p, prec="fp64")
    e = tb.energy(torch.tensor(pos, device="cuda"), s).item()
    ref = oracle.force_evaluation(pos, L, p)
    assert abs(e - ref.E_total) <= 1e-9 * abs(ref.E_total)
    s.close()
