"""Restart of an MD trajectory from a checkpoint: two velocity-Verlet steps,
a checkpoint, a fresh system restored from it and two more steps give the
trajectory of four uninterrupted steps (to the mu-search tolerance, since
the first step after the restart has no previous mu to start from)."""
import pytest
import torch

from synth import CONFIGS, fcc_c60_crystal, maxwell_boltzmann_velocities, workload_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_0910_4497_gb300 as tb
    assert torch.cuda.is_available()
    return tb


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_restart_continues_the_trajectory(tb, tmp_path, prec):
    cfg = CONFIGS[0]
    pos, L, _ = fcc_c60_crystal(cfg["ncell"], cfg["a"], cfg["jitter"], cfg["seed"])
    p = workload_params(cfg, defl_tol=1e-9)
    vel = maxwell_boltzmann_velocities(len(pos), 2000.0, 12.011, seed=9)

    def start():
        s = tb.TBSystem(len(pos), L, p, prec=prec)
        s.set_positions(pos)
        s.vel.copy_(torch.as_tensor(vel))
        s.evaluate()
        return s
    a = start()
    for _ in range(4):
        a.md_step(0.5, 12.011)
    b = start()
    for _ in range(2):
        b.md_step(0.5, 12.011)
    torch.cuda.synchronize()
    b.checkpoint(tmp_path / "md.npz", step=2, seed=9)
    b.close()
    c = tb.TBSystem(len(pos), L, p, prec=prec)
    step, seed = c.restore(tmp_path / "md.npz")
    assert (step, seed) == (2, 9)
    for _ in range(2):
        c.md_step(0.5, 12.011)
    torch.cuda.synchronize()
    a.check()
    c.check()
    assert (a.pos - c.pos).abs().max().item() <= 1e-8
    assert (a.vel - c.vel).abs().max().item() <= 1e-8
    a.close()
    c.close()
