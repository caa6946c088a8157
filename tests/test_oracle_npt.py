"""Pins of the oracle's weak-coupling NPT step (Berendsen thermostat and
isotropic barostat, the reading used since the paper names neither) against
what its definition fixes: no change at the target state, the rescaled
temperature T + (dt/tau_T)(T0 - T) recomputed from the rescaled velocities,
the relative volume change -beta (dt/tau_P)(P0 - P) from the new box,
unchanged fractional coordinates and total momentum, the pressure of a
force-free gas, and the direction of the relaxation along a short trajectory
of a compressed diamond cell.  CPU only."""
import numpy as np
import pytest

import oracle
from oracle import md, virial
from synth import TB_CONSTANTS, diamond_cell, maxwell_boltzmann_velocities

KB = md.KB_EV_PER_K
MASS = 12.011


def state(n=64, T=400.0, seed=3, L=10.0):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, L, size=(n, 3))
    vel = maxwell_boltzmann_velocities(n, T, MASS, seed)
    return pos, vel, L


def temperature(vel):
    return 2.0 * md.kinetic_energy(vel, MASS) / (KB * (3 * len(vel) - 3))


def test_identity_at_the_target_state():
    pos, vel, L = state()
    W = np.diag([1.5, -0.3, 0.7])
    ke = md.kinetic_energy(vel, MASS)
    T = temperature(vel)
    P = (np.trace(W) + 2 * ke) / (3 * L ** 3)
    x, v, Ln, (T1, P1, lam, mu) = md.berendsen_scale(pos, vel, L, W, ke, T, P, 0.5, 100.0,
                                                     500.0, 1.6)
    assert lam == 1.0 and mu == 1.0 and Ln == L
    assert np.array_equal(x, pos) and np.array_equal(v, vel)
    assert abs(T1 - T) < 1e-12 * T and abs(P1 - P) < 1e-15


@pytest.mark.parametrize("T0", [100.0, 500.0, 2500.0])
def test_thermostat_relaxes_linearly(T0):
    pos, vel, L = state(T=800.0)
    ke = md.kinetic_energy(vel, MASS)
    T = temperature(vel)
    dt, tau = 0.5, 100.0
    _, v, _, (T1, _, lam, _) = md.berendsen_scale(pos, vel, L, np.zeros((3, 3)), ke, T0, 0.0,
                                                  dt, tau, 500.0, 1.6)
    assert abs(T1 - T) < 1e-12 * T
    assert abs(temperature(v) - (T + dt / tau * (T0 - T))) < 1e-10 * T
    assert (lam > 1.0) == (T0 > T)


@pytest.mark.parametrize("P0", [-0.05, 0.0, 0.156])
def test_barostat_changes_volume_linearly(P0):
    pos, vel, L = state()
    W = np.diag([2.0, 1.0, 3.0])
    ke = md.kinetic_energy(vel, MASS)
    P = (6.0 + 2 * ke) / (3 * L ** 3)
    dt, tau, beta = 0.5, 500.0, 1.6
    x, _, Ln, (_, P1, _, mu) = md.berendsen_scale(pos, vel, L, W, ke, 500.0, P0, dt, 100.0,
                                                  tau, beta)
    assert abs(P1 - P) < 1e-15
    assert abs((Ln / L) ** 3 - 1.0 - (-beta * dt / tau * (P0 - P))) < 1e-14
    assert (Ln > L) == (P > P0)
    # fractional coordinates and the (zero) total momentum are unchanged
    assert np.allclose(x / Ln, pos / L, rtol=0, atol=1e-15)
    assert np.all((x >= 0.0) & (x < Ln))


def test_momentum_and_force_free_gas_pressure():
    pos, vel, L = state(n=100)
    vel = vel - vel.mean(axis=0)
    ke = md.kinetic_energy(vel, MASS)
    _, v, _, (T, P, _, _) = md.berendsen_scale(pos, vel, L, np.zeros((3, 3)), ke, 300.0, 0.0,
                                               0.5, 100.0, 500.0, 1.6)
    assert np.abs(v.sum(axis=0)).max() < 1e-12
    # ideal gas: P V = (2/3) KE = (dof/3) k_B T
    assert abs(P * L ** 3 - (3 * 100 - 3) / 3.0 * KB * T) < 1e-12 * P * L ** 3


def test_nonpositive_factor_is_refused():
    pos, vel, L = state()
    ke = md.kinetic_energy(vel, MASS)
    with pytest.raises(ValueError):
        md.berendsen_scale(pos, vel, L, np.zeros((3, 3)), ke, 500.0, 1e3, 0.5, 100.0, 500.0,
                           1.6)


def test_short_trajectory_relaxes_toward_the_target():
    """A diamond cell compressed 4% (positive pressure, here ~10^2 GPa) below
    its target temperature: the box grows and the velocities are scaled up at
    every step, and the trajectory is the Verlet step followed by the scaling."""
    pos, L = diamond_cell(2, a=3.567 * 0.96)
    p = dict(TB_CONSTANTS, kT=0.1, Rc=4.0, r=6, defl_tol=1e-9, n_electrons_per_atom=4.0)
    vel = maxwell_boltzmann_velocities(len(pos), 100.0, MASS, 7)
    vel -= vel.mean(axis=0)

    def evaluate(x, Lb):
        res = oracle.force_evaluation(x, Lb, p)
        return res.F, res.E_total, virial.evaluation_virial(res, p)
    F, _, _ = evaluate(pos, L)
    x, v = pos.copy(), vel.copy()
    for _ in range(3):
        L_old = L
        x, v, F, L, _, (T, P, lam, mu) = md.npt_step(x, v, F, L, 0.5, MASS, evaluate, 500.0,
                                                      0.0, 100.0, 500.0, 1.6)
        assert P > 0.0 and mu > 1.0 and L > L_old
        assert lam > 1.0 and T < 500.0
        assert abs(temperature(v) - (T + 0.5 / 100.0 * (500.0 - T))) < 1e-9 * T
    assert np.abs(v.sum(axis=0)).max() < 1e-9
