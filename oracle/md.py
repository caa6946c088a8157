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
