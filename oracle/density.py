"""Occupations, chemical potential, energies, density-matrix blocks and forces.

Sec. 2: rho = sum_m |m> f(e_m) <m| and <F_i> = Tr[rho F_i] with the force
matrix F_i = -dH/dR_i.  Locally, the columns rho|i, a> of the target's own
orbitals come from its Krylov projection: rho|i,a> ~ V f(T) V^T |i,a>.

Readings (the paper does not state the occupation function, the spin factor, how
mu is fixed, or how the two column estimates of a bond are combined):
* f(x) = 1 / (1 + e^x), x = (lambda - mu) / kT, per spin orbital; spin factor 2;
* mu solves  2 sum_i sum_m w_im f((lambda_im - mu)/kT) = N_e  with
  w_im = sum_a S_im[a]^2 (weight of Ritz pair m on the seed block), by
  bisection on [min lambda - 40 kT, max lambda + 40 kT] until the bracket is
  narrower than 1e-14 eV (at most 200 halvings);
* E_band = 2 sum w f lambda;  -TS = 2 kT sum w [f ln f + (1-f) ln(1-f)];
  A (Mermin free energy) = E_band - TS;
* force on atom k: with G = dt(d)/dd for bond d = R_j - R_k,
  F_k = 2 sum_{j in H(k)} sum_{a,b} [rho^(k)_{j b, k a} + rho^(j)_{k a, j b}] G_ab
        - dE_rep/dR_k,
  taking each density-matrix column from its own atom's Krylov run (both
  endpoint columns of every bond); pairwise, so sum_k F_k = 0.
"""
import numpy as np


def fermi(x):
    """f(x) = 1/(1+e^x), evaluated as e^-x/(1+e^-x) for x > 0."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    pos = x > 0
    e = np.exp(-x[pos])
    out[pos] = e / (1.0 + e)
    out[~pos] = 1.0 / (1.0 + np.exp(x[~pos]))
    return out


def entropy_term(f):
    """f ln f + (1-f) ln(1-f), with 0 ln 0 = 0."""
    f = np.asarray(f, dtype=np.float64)
    out = np.zeros_like(f)
    a = f > 0
    out[a] += f[a] * np.log(f[a])
    b = f < 1
    out[b] += (1 - f[b]) * np.log(1 - f[b])
    return out


def electron_count(mu, lam, w, kT):
    return 2.0 * np.sum(w * fermi((lam - mu) / kT))


def find_mu(lam, w, kT, n_electrons, width=1e-14, max_iter=200):
    """Bisection for mu (lam, w: flat arrays of all targets' Ritz pairs)."""
    lo = lam.min() - 40.0 * kT
    hi = lam.max() + 40.0 * kT
    for _ in range(max_iter):
        if hi - lo < width:
            break
        mid = 0.5 * (lo + hi)
        n = electron_count(mid, lam, w, kT)
        if n == n_electrons:
            return mid
        if n < n_electrons:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def band_terms(lam, w, mu, kT):
    """(E_band, -TS, N_e) of one target's (or all targets') Ritz pairs."""
    f = fermi((lam - mu) / kT)
    return (2.0 * np.sum(w * f * lam),
            2.0 * kT * np.sum(w * entropy_term(f)),
            2.0 * np.sum(w * f))


def rho_blocks(S, P, lam, mu, kT):
    """rho^(i) blocks: R[q, b, a] = rho_{(q-th row atom) b, (target) a}."""
    f = fermi((lam - mu) / kT)
    nq = P.shape[0] // 4
    return ((P * f[None, :]) @ S.T).reshape(nq, 4, 4)


def forces(bonds, rho, hlists, rep_der):
    """Hellmann-Feynman pair forces plus the repulsion (rep_der[b] = phi'(r_b))."""
    n = bonds.n
    F = np.zeros((n, 3))
    for k in range(n):
        for q, j in enumerate(hlists[k]):
            b = bonds.off[k] + q
            rq = int(np.searchsorted(hlists[j], k))
            R_sum = rho[k][1 + q] + rho[j][1 + rq].T       # [b, a]
            G = bonds.g[b]                                  # [kappa, a, b]
            F[k] += 2.0 * np.einsum('ba,kab->k', R_sum, G)
            r = np.sqrt(bonds.d[b] @ bonds.d[b])
            F[k] += rep_der[b] * bonds.d[b] / r
    return F
