"""Velocity-Verlet step of the MD workload (the paper runs MD, Sec. 4, but does
not state its integrator; NVE velocity-Verlet is the reading used here).

    v <- v + (dt/2) F/m;  x <- wrap(x + dt v);  F <- F(x);  v <- v + (dt/2) F/m
Units: A, fs, eV, amu; 1 eV/(A amu) = 9.648533e-3 A/fs^2.
"""
import numpy as np

ACC = 9.648533e-3


def wrap(x, L):
    y = np.mod(x, L)
    y[y >= L] = 0.0
    return y


def verlet_step(pos, vel, F, L, dt, mass, force_fn):
    """One step; force_fn(pos) -> (F, E_pot).  Returns (pos, vel, F, E_pot)."""
    a = ACC / mass
    vel = vel + 0.5 * dt * a * F
    pos = wrap(pos + dt * vel, L)
    F, epot = force_fn(pos)
    vel = vel + 0.5 * dt * a * F
    return pos, vel, F, epot


def kinetic_energy(vel, mass):
    return 0.5 * mass * np.sum(vel * vel) / ACC


# ---------------------------------------------------------------- NPT
# The paper runs its C60 polymerisation at 25 GPa and 500 K (Sec. 4) without
# naming a thermostat or barostat.  The reading used here is weak coupling
# (Berendsen): after each velocity-Verlet step, with the step's kinetic energy
# KE and virial W,
#   T = 2 KE / (k_B (3n - 3)),   P = (tr W + 2 KE) / (3 L^3),
#   lambda^2 = 1 + (dt/tau_T)(T0/T - 1),   mu^3 = 1 - beta (dt/tau_P)(P0 - P),
#   v <- lambda v,  x <- mu x,  L <- mu L.

KB_EV_PER_K = 8.617333262e-5


def berendsen_scale(pos, vel, L, W, ke, T0, P0, dt, tau_T, tau_P, beta):
    """Returns (pos, vel, L, (T, P, lambda, mu)) after the scaling."""
    n = len(pos)
    dof = 3.0 * n - 3.0 if n > 1 else 3.0
    T = 2.0 * ke / (KB_EV_PER_K * dof)
    P = (np.trace(W) + 2.0 * ke) / (3.0 * L ** 3)
    lam2 = 1.0 + dt / tau_T * (T0 / T - 1.0) if T > 0.0 else 1.0
    mu3 = 1.0 - beta * dt / tau_P * (P0 - P)
    if not (lam2 > 0.0 and mu3 > 0.0):
        raise ValueError("weak-coupling factor is not positive")
    lam, mu = np.sqrt(lam2), np.cbrt(mu3)
    Ln = mu * L
    x = mu * pos
    x[x >= Ln] -= Ln
    return x, lam * vel, Ln, (T, P, lam, mu)


def npt_step(pos, vel, F, L, dt, mass, evaluate, T0, P0, tau_T, tau_P, beta):
    """One velocity-Verlet step at box L, then the weak-coupling scaling.
    evaluate(pos, L) -> (F, E_pot, W) of the force evaluation at pos.
    Returns (pos, vel, F, L, E_pot, (T, P, lambda, mu)); F is the force of the
    unscaled configuration, which the next step's first half kick uses."""
    out = {}

    def force_fn(x):
        F_, epot_, W_ = evaluate(x, L)
        out["W"] = W_
        return F_, epot_
    pos, vel, F, epot = verlet_step(pos, vel, F, L, dt, mass, force_fn)
    ke = kinetic_energy(vel, mass)
    pos, vel, L, state = berendsen_scale(pos, vel, L, out["W"], ke, T0, P0, dt, tau_T, tau_P,
                                         beta)
    return pos, vel, F, L, epot, state
