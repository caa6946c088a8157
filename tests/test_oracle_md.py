"""Pins of the oracle's velocity-Verlet step, kinetic energy and unit constant
against facts that do not come from the oracle itself:

* the acceleration unit 1 eV/(A amu) in A/fs^2, derived here from the SI
  values of the electron volt, the atomic mass unit, the angstrom and the
  femtosecond;
* the kinetic energy of a given velocity, converted to eV from SI units;
* the closed-form trajectory of the Stoermer-Verlet recurrence in a harmonic
  well, x_n = x_0 cos(n th) + (h v_0 / sin th) sin(n th) with
  cos th = 1 - (h w)^2 / 2, and v_n = (x_{n+1} - x_{n-1}) / (2h);
* exactness of the scheme for a constant force, on a particle that crosses
  the periodic boundary several times (wrapping of the positions);
* second-order energy error on the exact forces of an isolated C60 molecule
  (whole-molecule diagonalisation, where the force is the exact gradient of
  the Mermin free energy plus the repulsion): halving dt divides the largest
  deviation of the total energy over the same time window by about four.
CPU only."""
import numpy as np
import pytest

import oracle
from oracle import md
from synth import TB_CONSTANTS, c60_cage, maxwell_boltzmann_velocities

# SI values (exact by definition, except the atomic mass unit, CODATA 2018)
E_CHARGE = 1.602176634e-19        # J per eV
AMU = 1.66053906660e-27           # kg
ANGSTROM = 1e-10                  # m
FEMTOSECOND = 1e-15               # s

ACC_SI = (E_CHARGE / ANGSTROM) / AMU * FEMTOSECOND ** 2 / ANGSTROM   # A/fs^2 per eV/(A amu)


def test_acceleration_unit_from_si():
    assert abs(md.ACC - ACC_SI) <= 1e-7 * ACC_SI


def test_kinetic_energy_from_si_units():
    rng = np.random.default_rng(11)
    v = rng.standard_normal((5, 3)) * 0.05                       # A/fs
    m = 12.011
    ke_joule = 0.5 * m * AMU * np.sum((v * ANGSTROM / FEMTOSECOND) ** 2)
    assert abs(md.kinetic_energy(v, m) - ke_joule / E_CHARGE) <= 1e-7 * ke_joule / E_CHARGE


def harmonic_force(k, center):
    """F = -k (x - center) per component (eV/A), E = k/2 |x - center|^2."""
    def f(x):
        d = x - center
        return -k * d, 0.5 * k * np.sum(d * d)
    return f


@pytest.mark.parametrize("dt", [0.25, 1.0, 3.0])
def test_harmonic_well_matches_closed_form(dt):
    m, k, L = 12.011, 40.0, 30.0
    center = np.full(3, 0.5 * L)
    x0 = center + np.array([[0.3, -0.2, 0.1], [-0.05, 0.4, 0.25]])
    v0 = np.array([[0.01, 0.02, -0.015], [-0.02, 0.0, 0.03]])
    w = np.sqrt(k * ACC_SI / m)                                  # 1/fs
    th = np.arccos(1.0 - 0.5 * (dt * w) ** 2)
    ffn = harmonic_force(k, center)
    x, v = x0.copy(), v0.copy()
    F, _ = ffn(x)
    nsteps = 40
    for _ in range(nsteps):
        x, v, F, _ = md.verlet_step(x, v, F, L, dt, m, ffn)

    x_exact = center + (x0 - center) * np.cos(nsteps * th) + dt * v0 / np.sin(th) * np.sin(nsteps * th)
    v_exact = np.sin(th) / dt * (-(x0 - center) * np.sin(nsteps * th)
                                 + dt * v0 / np.sin(th) * np.cos(nsteps * th))
    # the oracle's constant carries 7 digits (2e-8 relative): phase error ~1e-8 A
    assert np.abs(x - x_exact).max() <= 1e-7
    assert np.abs(v - v_exact).max() <= 5e-8


def test_constant_force_across_the_boundary():
    m, L, dt = 12.011, 6.0, 0.5
    f0 = np.array([[0.8, -0.5, 0.2]])                           # eV/A
    x0 = np.array([[5.5, 0.3, 3.0]])
    v0 = np.array([[0.9, -0.45, 0.05]])                         # A/fs: several box crossings

    def ffn(x):
        return f0.copy(), 0.0
    x, v, F = x0.copy(), v0.copy(), f0.copy()
    nsteps = 60
    for _ in range(nsteps):
        x, v, F, _ = md.verlet_step(x, v, F, L, dt, m, ffn)
        assert np.all(x >= 0.0) and np.all(x < L)
    t = nsteps * dt
    a = f0 * ACC_SI / m
    assert np.abs(v - (v0 + a * t)).max() <= 1e-9
    unwrapped = x0 + v0 * t + 0.5 * a * t * t
    assert np.abs(unwrapped).max() > 3 * L                        # it did cross
    d = x - unwrapped
    d -= L * np.round(d / L)
    assert np.abs(d).max() <= 1e-8


def test_energy_error_is_second_order_in_dt():
    """Isolated C60 (box 40 A) at 2000 K on the exact whole-molecule forces:
    the largest |E(t) - E(0)| over 12 fs scales as dt^2."""
    L = 40.0
    p = dict(TB_CONSTANTS, kT=0.1, Rc=5.0, r=1, n_electrons_per_atom=4.0)
    pos0 = c60_cage() + 0.5 * L
    vel0 = maxwell_boltzmann_velocities(60, 2000.0, 12.011, seed=7)

    def ffn(x):
        ex = oracle.exact.whole_cell(x, L, p)
        A = ex["E_band"] + ex["E_entropy"] + ex["E_rep"]
        return ex["F"], A

    def max_dev(dt, t_end=12.0):
        x, v = pos0.copy(), vel0.copy()
        F, epot = ffn(x)
        e0 = epot + md.kinetic_energy(v, 12.011)
        dev = 0.0
        for _ in range(int(round(t_end / dt))):
            x, v, F, epot = md.verlet_step(x, v, F, L, dt, 12.011, ffn)
            dev = max(dev, abs(epot + md.kinetic_energy(v, 12.011) - e0))
        return dev
    d1, d2 = max_dev(0.5), max_dev(0.25)
    assert d1 > 1e-4                                               # measurable, not roundoff
    assert 3.0 <= d1 / d2 <= 5.0, (d1, d2)
