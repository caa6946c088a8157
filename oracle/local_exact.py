"""Exact gradient of the truncated local free energy (the differentiable form of
the method), at Krylov order r = r_min.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2 gives each target atom i its cluster Hamiltonian H_c(i) (the atoms
within the cutoff radius) and Sec. 3 its Krylov space K_r(H_c, |i,a>); once r
reaches the minimal-polynomial degree (r_min) the space is invariant and the
projection is exact: the target's spectral record equals the one from the
dense eigen-decomposition of H_c(i).  This module takes that limit as its
definition:

  Omega_i(mu) = 2 sum_a <i a| omega(H_c(i)) |i a>,
  omega(e)    = -kT ln(1 + exp(-(e - mu)/kT))       (so omega' = f),
  A_i         = Omega_i + mu N_i,   N_i = 2 sum_a <i a| f(H_c(i)) |i a>,
  A_loc       = sum_i A_i,  with mu fixed by sum_i N_i = N_e.

At fixed N_e, d A_loc / dR = d(sum_i Omega_i)/dR at fixed mu (the mu terms
cancel because sum_i dOmega_i/dmu = -N_e).  With H_c = Z diag(lam) Z^T and the
seed rows S = Z[0:4, :], the gradient of Omega_i with respect to the entries of
H_c is (Daleckii-Krein)

  G_i = dOmega_i / dH_c = 2 Z (Gamma o (S^T S)) Z^T,
  Gamma_mn = (omega(lam_m) - omega(lam_n)) / (lam_m - lam_n),  Gamma_mm = f(lam_m),

and every Hamiltonian block inside the cluster depends on the bond vector
d = R_b - R_a of its two atoms, so

  dOmega_i/dR_k = sum over directed bonds (a -> b) with a, b in cluster(i) of
                  sum_{alpha,beta} G_i[a alpha, b beta] dH_ab/dd (delta_kb - delta_ka).

Forces F = -d(A_loc + E_rep)/dR.  When every cluster holds the whole system the
seeds of all targets together span the identity and the sum over i reduces to
the Hellmann-Feynman pair force; for truncated clusters the two differ (the
Hellmann-Feynman force is not the gradient of any truncated energy).

Library primitives used as single steps: numpy.linalg.eigh, matmul.
"""
import numpy as np

from . import model
from .neighbors import neighbor_lists, cluster_lists
from .hamiltonian import BondTable, cluster_hamiltonian
from .density import fermi, find_mu, band_terms


def omega(lam, mu, kT):
    """Grand potential per spin orbital, -kT ln(1 + e^{-x}), x = (lam - mu)/kT,
    without overflow: for x < 0 it is written as (lam - mu) - kT ln(1 + e^{x})."""
    x = (np.asarray(lam, dtype=np.float64) - mu) / kT
    out = np.empty_like(x)
    p = x >= 0
    out[p] = -kT * np.log1p(np.exp(-x[p]))
    out[~p] = kT * x[~p] - kT * np.log1p(np.exp(x[~p]))
    return out


def loewner(lam, mu, kT):
    """Gamma_mn, the divided differences of omega on the eigenvalues.

    For |lam_m - lam_n| <= 1e-3 kT the quotient loses digits, so there the
    divided difference (the mean of f over [lam_n, lam_m]) is expanded about
    the midpoint c: f(c) + f''(c) (lam_m - lam_n)^2 / 24, with
    f''(e) = f (1 - f)(1 - 2 f) / kT^2; the next term is below 1e-13 f."""
    lam = np.asarray(lam, dtype=np.float64)
    om = omega(lam, mu, kT)
    dl = lam[:, None] - lam[None, :]
    close = np.abs(dl) <= 1e-3 * kT
    with np.errstate(divide="ignore", invalid="ignore"):
        G = (om[:, None] - om[None, :]) / dl
    c = 0.5 * (lam[:, None] + lam[None, :])
    fc = fermi((c - mu) / kT)
    d2 = fc * (1.0 - fc) * (1.0 - 2.0 * fc) / (kT * kT)
    G[close] = (fc + d2 * dl * dl / 24.0)[close]
    return G


def target_spectrum(bonds, clist):
    """Dense eigen-decomposition of H_c of one target: (lam, Z)."""
    Hc = cluster_hamiltonian(bonds, clist)
    return np.linalg.eigh(Hc)


def target_gradient_matrix(lam, Z, mu, kT):
    """G_i = dOmega_i/dH_c = 2 Z (Gamma o S^T S) Z^T (dense, symmetric)."""
    S = Z[0:4, :]
    M = loewner(lam, mu, kT) * (S.T @ S)
    return 2.0 * (Z @ M) @ Z.T


def target_force_terms(bonds, clist, G, out):
    """Adds -dOmega_i/dR to `out` (n x 3) from the gradient matrix G of one
    target, over every directed bond with both atoms in the cluster."""
    slot = {int(a): s for s, a in enumerate(clist)}
    for s, a in enumerate(clist):
        a = int(a)
        for q, b in enumerate(bonds.hlists[a]):
            t = slot.get(int(b))
            if t is None:
                continue
            bi = bonds.off[a] + q
            blk = G[4 * s:4 * s + 4, 4 * t:4 * t + 4]
            c = np.einsum('ab,kab->k', blk, bonds.g[bi])   # dOmega_i / dd of this block
            out[int(b)] -= c
            out[a] += c


def local_evaluation(pos, L, p, with_forces=True, targets=None):
    """A_loc + E_rep, mu and (optionally) F = -d(A_loc + E_rep)/dR.

    targets: restrict the force sum to these targets' terms (all by default;
    used to compare a few atoms' forces, with the terms of the targets whose
    clusters contain them)."""
    pos = np.asarray(pos, dtype=np.float64)
    n = len(pos)
    kT = p["kT"]
    hl = neighbor_lists(pos, L, p["rm"])
    cl = cluster_lists(pos, L, p["Rc"])
    bonds = BondTable(pos, L, hl, p)
    spec = [target_spectrum(bonds, cl[i]) for i in range(n)]
    lam_all = np.concatenate([s[0] for s in spec])
    w_all = np.concatenate([np.sum(s[1][0:4, :] ** 2, axis=0) for s in spec])
    mu = find_mu(lam_all, w_all, kT, p["n_electrons_per_atom"] * n)
    eb, ts, ne = band_terms(lam_all, w_all, mu, kT)
    r_b = np.sqrt(np.sum(bonds.d * bonds.d, axis=1))
    phi, dphi = model.pair_repulsion(r_b, p)
    res = dict(mu=mu, E_band=eb, E_entropy=ts, A=eb + ts, n_electrons=ne,
               E_rep=0.5 * np.sum(phi), hlists=hl, clists=cl,
               lam=[s[0] for s in spec], w=[np.sum(s[1][0:4, :] ** 2, axis=0) for s in spec])
    res["E_total"] = res["A"] + res["E_rep"]
    if with_forces:
        F = np.zeros((n, 3))
        for i in (range(n) if targets is None else targets):
            lam, Z = spec[i]
            target_force_terms(bonds, cl[i], target_gradient_matrix(lam, Z, mu, kT), F)
        for k in range(n):
            for q in range(len(hl[k])):
                b = bonds.off[k] + q
                F[k] += dphi[b] * bonds.d[b] / r_b[b]
        res["F"] = F
    return res


def targets_touching(clists, atoms):
    """Targets whose clusters contain any of `atoms` (their force terms are the
    only ones that reach those atoms)."""
    s = set(int(a) for a in atoms)
    return [i for i, c in enumerate(clists) if s.intersection(int(x) for x in c)]
