"""Tight-binding model of Eq. (1): sp3 Slater-Koster hoppings with Xu-type
(GSP) distance scaling, a C1 cubic tail to zero, and a pair repulsion of the
same form (Sec. 5: both parameter sets share these functional forms).

Readings (the paper prints no formulas for the model):
* distance scaling s(r) = (r0/r)^n exp{n[-(r/rc)^nc + (r0/rc)^nc]} for r < r1;
* on [r1, rm] the cubic p(x) = s(r1) + s'(r1) x + a x^2 + b x^3, x = r - r1,
  with p(rm - r1) = 0 and p'(rm - r1) = 0; zero for r >= rm;
* Slater-Koster two-centre table for s and p orbitals, direction cosines l of
  d = R_j - R_i;
* on-site block diag(Es, Ep, Ep, Ep);
* E_rep = sum over pairs of phi(r), phi of the same GSP form and tail.

Orbital order: s, px, py, pz.
"""
import numpy as np


def _gsp(r, A, r_ref, expo, r_cut, expo_c):
    """A (r_ref/r)^expo exp{expo[-(r/r_cut)^expo_c + (r_ref/r_cut)^expo_c]} and its
    derivative with respect to r."""
    val = A * (r_ref / r) ** expo * np.exp(
        expo * (-(r / r_cut) ** expo_c + (r_ref / r_cut) ** expo_c))
    der = val * (-expo / r - expo * expo_c * (r / r_cut) ** expo_c / r)
    return val, der


def _tail_coefficients(v1, d1, delta):
    """Cubic p(x) = v1 + d1 x + a x^2 + b x^3 with p(delta) = p'(delta) = 0."""
    a = -(3.0 * v1 + 2.0 * d1 * delta) / delta ** 2
    b = (2.0 * v1 + d1 * delta) / delta ** 3
    return a, b


def _scaled(r, p, A, r_ref, expo, r_cut, expo_c):
    r = np.asarray(r, dtype=np.float64)
    r1, rm = p["r1"], p["rm"]
    v1, d1 = _gsp(r1, A, r_ref, expo, r_cut, expo_c)
    a, b = _tail_coefficients(v1, d1, rm - r1)
    val = np.zeros_like(r)
    der = np.zeros_like(r)
    inner = r < r1
    if np.any(inner):
        v, d = _gsp(r[inner], A, r_ref, expo, r_cut, expo_c)
        val[inner] = v
        der[inner] = d
    tail = (r >= r1) & (r < rm)
    if np.any(tail):
        x = r[tail] - r1
        val[tail] = v1 + d1 * x + a * x ** 2 + b * x ** 3
        der[tail] = d1 + 2.0 * a * x + 3.0 * b * x ** 2
    return val, der


def hopping_scale(r, p):
    """s(r) and ds/dr for the hopping integrals (s(r0) = 1)."""
    return _scaled(r, p, 1.0, p["r0"], p["n"], p["rc"], p["nc"])


def pair_repulsion(r, p):
    """phi(r) and dphi/dr of the pair repulsion (eV, eV/A)."""
    return _scaled(r, p, p["phi0"], p["d0"], p["m"], p["dc"], p["mc"])


def sk_matrix(l, p):
    """Slater-Koster 4x4 table M(l) for unit vector l (from atom i to atom j):
    H_{i a, j b} = s(r) M_ab(l)."""
    Vss, Vsp, Vpps, Vppp = p["Vss"], p["Vsp"], p["Vpps"], p["Vppp"]
    M = np.empty((4, 4))
    M[0, 0] = Vss
    M[0, 1:] = l * Vsp
    M[1:, 0] = -l * Vsp
    M[1:, 1:] = np.outer(l, l) * (Vpps - Vppp) + np.eye(3) * Vppp
    return M


def sk_block(d, p):
    """Hopping block t(d) (4x4) for bond vector d = R_j - R_i."""
    d = np.asarray(d, dtype=np.float64)
    r = np.sqrt(d @ d)
    s, _ = hopping_scale(np.array([r]), p)
    return s[0] * sk_matrix(d / r, p)


def sk_block_grad(d, p):
    """dt_ab/dd_k for bond vector d = R_j - R_i, shape (3, 4, 4) [k, a, b].
    dt/dR_i = -dt/dd and dt/dR_j = +dt/dd."""
    d = np.asarray(d, dtype=np.float64)
    r = np.sqrt(d @ d)
    l = d / r
    s, ds = hopping_scale(np.array([r]), p)
    s, ds = s[0], ds[0]
    M = sk_matrix(l, p)
    Vsp, dpp = p["Vsp"], p["Vpps"] - p["Vppp"]
    G = np.zeros((3, 4, 4))
    for k in range(3):
        dl = (np.eye(3)[k] - l * l[k]) / r          # d l / d d_k
        dM = np.zeros((4, 4))
        dM[0, 1:] = dl * Vsp
        dM[1:, 0] = -dl * Vsp
        dM[1:, 1:] = (np.outer(dl, l) + np.outer(l, dl)) * dpp
        G[k] = ds * l[k] * M + s * dM
    return G


def onsite_block(p):
    return np.diag([p["Es"], p["Ep"], p["Ep"], p["Ep"]])
