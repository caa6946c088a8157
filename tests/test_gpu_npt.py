"""GPU parity of the weak-coupling NPT step through the C ABI: three
steps of the 240-atom cell at 25 GPa and 500 K (tb_md_step, tb_virial,
tb_npt_berendsen) against the oracle's Verlet step, virial and scaling on the
same seeded state, in both precisions; the host argument checks and the
device's refusal of a non-positive scale factor.

Tolerances: FP64 positions and velocities 1e-9, box 1e-12 relative; mixed
(forces within 1e-3 eV/A) positions 1e-5 A, velocities 1e-5 A/fs, box 1e-8
relative, pressure 1e-4 eV/A^3."""
import numpy as np
import pytest
import torch

import oracle
from oracle import md, virial
from synth import CONFIGS, NPT, fcc_c60_crystal, maxwell_boltzmann_velocities, workload_params
from synth.configs import GPA_PER_EV_A3, MASS_C_AMU

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(x=1e-9, v=1e-9, L=1e-12, P=1e-9),
       "mixed": dict(x=1e-5, v=1e-5, L=1e-8, P=1e-4)}
COUPLING = (NPT["T0_K"], NPT["P0_GPa"] / GPA_PER_EV_A3, NPT["tau_T_fs"], NPT["tau_P_fs"],
            GPA_PER_EV_A3 / NPT["B_GPa"])


@pytest.fixture(scope="module")
def tb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_0910_4497_gb300 as tb
    assert torch.cuda.is_available()
    return tb


def cell():
    cfg = CONFIGS[0]
    pos, L, _ = fcc_c60_crystal(cfg["ncell"], cfg["a"], cfg["jitter"], cfg["seed"])
    vel = maxwell_boltzmann_velocities(len(pos), NPT["T0_K"], MASS_C_AMU, 11)
    return pos, vel, L, workload_params(cfg, defl_tol=1e-9)


_REF = {}


def oracle_npt(steps=3):
    if "npt" not in _REF:
        pos, vel, L, p = cell()

        def evaluate(x, Lb):
            res = oracle.force_evaluation(x, Lb, p)
            return res.F, res.E_total, virial.evaluation_virial(res, p)
        F, _, _ = evaluate(pos, L)
        x, v, out = pos.copy(), vel.copy(), []
        for _ in range(steps):
            x, v, F, L, _, st = md.npt_step(x, v, F, L, NPT["dt_fs"], MASS_C_AMU, evaluate,
                                            *COUPLING)
            out.append((x.copy(), v.copy(), L, st))
        _REF["npt"] = out
    return _REF["npt"]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_npt_steps_match_oracle(tb, prec):
    pos, vel, L, p = cell()
    ref = oracle_npt()
    s = tb.TBSystem(len(pos), L, p, prec=prec)
    s.set_positions(pos)
    s.vel.copy_(torch.as_tensor(vel))
    s.evaluate()
    tol = TOL[prec]
    for x_r, v_r, L_r, (T_r, P_r, lam_r, mu_r) in ref:
        s.npt_step(NPT["dt_fs"], MASS_C_AMU, *COUPLING)
        s.check()
        T, P, lam, mu = s.npt_state.cpu().tolist()
        assert abs(s.L - L_r) <= tol["L"] * L_r
        assert abs(P - P_r) <= tol["P"]
        assert abs(T - T_r) <= 1e-6 * T_r
        dx = s.pos.cpu().numpy() - x_r
        dx -= s.L * np.rint(dx / s.L)
        assert np.abs(dx).max() <= tol["x"]
        assert np.abs(s.vel.cpu().numpy() - v_r).max() <= tol["v"]
        assert np.all(s.pos.cpu().numpy() < s.L) and np.all(s.pos.cpu().numpy() >= 0.0)
    # the box moves toward the target pressure: it grows iff P > P0
    assert (s.L > L) == (ref[0][3][1] > COUPLING[1])
    s.close()


def test_npt_argument_checks_and_device_refusal(tb):
    pos, vel, L, p = cell()
    s = tb.TBSystem(len(pos), L, p, prec="fp64")
    s.set_positions(pos)
    s.vel.copy_(torch.as_tensor(vel))
    s.evaluate()
    B = tb.binding
    T0, P0, tT, tP, beta = COUPLING
    for bad in (dict(tau_T=0.4), dict(tau_P=0.5), dict(beta=0.0), dict(T0=-1.0)):
        a = dict(T0=T0, tau_T=tT, tau_P=tP, beta=beta)
        a.update(bad)
        with pytest.raises(B.TBError):
            B.tb_npt_berendsen(s.ctx, s.n, s.pos, s.vel, s.L, s.W, s.energies, a["T0"], P0,
                               0.5, a["tau_T"], a["tau_P"], a["beta"], s.L_dev, s.npt_state)
    # a target pressure so far above P that mu^3 <= 0: refused on the device,
    # nothing scaled
    s.md_step(0.5, MASS_C_AMU)
    B.tb_virial(s.ctx, s.n, s.pos, s.L, None, None, s.W, s.pressure)
    x0, v0 = s.pos.clone(), s.vel.clone()
    B.tb_npt_berendsen(s.ctx, s.n, s.pos, s.vel, s.L, s.W, s.energies, T0, 1e3, 0.5, tT, tP,
                       beta, s.L_dev, s.npt_state)
    torch.cuda.synchronize()
    code, info = s.status()
    assert B.STATUS_NAMES[code] == "TB_ERR_INVALID_ARG" and info == 1     # mu^3 <= 0
    assert torch.equal(s.pos, x0) and torch.equal(s.vel, v0) and s.L_dev.item() == s.L
    s.close()
