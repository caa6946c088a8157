"""Failure paths of the device status word, made to fire on purpose without
faulting the GPU: every device-side wait in the library is bounded by the
context's timeout_cycles and returns TB_ERR_TIMEOUT when it runs out; the mu
search reports TB_ERR_NO_CONVERGENCE when its pass budget is spent; a NaN
coordinate is refused as a position outside [0, L).  After each failure the
GPU and a fresh context still give the oracle's answer.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from synth import CONFIGS, fcc_c60_crystal, workload_params

pytestmark = pytest.mark.gpu

TB_ERR_INVALID_ARG, TB_ERR_NO_CONVERGENCE, TB_ERR_TIMEOUT = 1, 7, 8


@pytest.fixture(scope="module")
def tb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_0910_4497_gb300 as tb
    assert torch.cuda.is_available()
    return tb


@pytest.fixture(scope="module")
def cell():
    cfg = CONFIGS[0]
    pos, L, _ = fcc_c60_crystal(cfg["ncell"], cfg["a"], cfg["jitter"], cfg["seed"])
    p = workload_params(cfg, defl_tol=1e-9)
    return pos, L, p


@pytest.fixture(scope="module")
def reference(cell):
    pos, L, p = cell
    return oracle.force_evaluation(pos, L, p)


def healthy(tb, pos, L, p, ref, prec):
    """A fresh context on the same GPU evaluates the cell correctly."""
    s = tb.TBSystem(len(pos), L, p, prec=prec)
    s.set_positions(pos)
    s.evaluate()
    torch.cuda.synchronize()
    s.check()
    err = np.abs(s.F.cpu().numpy() - ref.F).max()
    s.close()
    assert err <= (1e-6 if prec == "fp64" else 1e-3)


def test_persistent_queue_wait_times_out(tb, cell, reference):
    """Mixed path, persistent Krylov + eigensolve queue: with 240 targets on
    hundreds of CTAs, most CTAs take an eigensolve item at once and wait for a
    block-Lanczos record that is still being built; a one-cycle budget makes
    every such wait give up."""
    pos, L, p = cell
    s = tb.TBSystem(len(pos), L, dict(p, timeout_cycles=1, schedule="persistent"), prec="mixed")
    s.set_positions(pos)
    s.neighbors()
    s.assemble()
    s.krylov()
    torch.cuda.synchronize()
    code, info = s.status()
    assert code == TB_ERR_TIMEOUT and 0 <= info < len(pos)
    s.close()
    healthy(tb, pos, L, p, reference, "mixed")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_mu_grid_barrier_times_out(tb, cell, reference, prec):
    """The cooperative mu search synchronises its blocks with a bounded
    grid barrier: with a one-cycle budget the first blocks to arrive give up."""
    pos, L, p = cell
    s = tb.TBSystem(len(pos), L, p, prec=prec)
    s.set_positions(pos)
    s.neighbors()
    s.assemble()
    s.krylov()
    torch.cuda.synchronize()
    s.check()
    t = tb.TBSystem(len(pos), L, dict(p, timeout_cycles=1), prec=prec)
    tb.binding.tb_find_mu(t.ctx, s.n, s.lam, s.S, s.kdim, 4.0 * s.n, None, t.mu, t.ncount)
    torch.cuda.synchronize()
    code, _ = t.status()
    assert code == TB_ERR_TIMEOUT
    t.close()
    s.close()
    healthy(tb, pos, L, p, reference, prec)


def test_mu_pass_budget_reports_no_convergence(tb, cell, reference):
    pos, L, p = cell
    s = tb.TBSystem(len(pos), L, dict(p, mu_max_iter=1), prec="fp64")
    s.set_positions(pos)
    s.evaluate()
    torch.cuda.synchronize()
    code, _ = s.status()
    assert code == TB_ERR_NO_CONVERGENCE
    mu = s.mu.item()
    assert math.isfinite(mu)                     # the best estimate is still returned
    s.close()
    healthy(tb, pos, L, p, reference, "fp64")


@pytest.mark.parametrize("ncell", [1, 2])
def test_nan_coordinate_is_refused(tb, ncell):
    """A NaN coordinate fails the [0, L) check (brute-force lists on the
    240-atom cell, cell lists on the 1920-atom one); the rest of the call
    sequence runs on the remaining atoms without touching memory it does not
    own, and the status names the atom."""
    cfg = CONFIGS[0 if ncell == 1 else 1]
    pos, L, _ = fcc_c60_crystal(ncell, cfg["a"], cfg["jitter"], cfg["seed"])
    p = workload_params(cfg, defl_tol=1e-9)
    pos = pos.copy()
    pos[37, 1] = float("nan")
    s = tb.TBSystem(len(pos), L, p, prec="mixed")
    s.set_positions(pos)
    s.evaluate()
    torch.cuda.synchronize()
    code, info = s.status()
    assert code == TB_ERR_INVALID_ARG and info == 37
    # no list holds the NaN atom, and it holds nobody
    hl, cl = s.lists()
    assert len(hl[37]) == 0 and list(cl[37]) == [37]
    assert all(37 not in x for k, x in enumerate(cl) if k != 37)
    s.close()
