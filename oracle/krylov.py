"""Block Krylov subspace of one target atom and its projected eigenproblem.

Sec. 3, Eq. (Krylov): K_r(H, phi) = span{phi, H phi, ..., H^{r-1} phi}, with the
seed phi the target atom's own atomic orbitals (not a random vector).  With the
four sp3 orbitals as a block seed E_i this is the block Krylov space
span{E_i, H_c E_i, ..., H_c^{r-1} E_i} of dimension <= 4r.

Eqs. (lanczos) / (lanczos_blas3) in block form: with V_0 = 0 and V_1 = E_i,
    W_k = H_c V_k - V_{k-1} B_{k-1}^T,  A_k = V_k^T W_k,  W_k <- W_k - V_k A_k,
    W_k = V_{k+1} B_k  (orthonormal V_{k+1}, B_k upper triangular).
T = V^T H_c V (Sec. 3: the Lanczos transform of H), here formed explicitly from
the orthonormal basis; its eigenpairs (lambda_m, U) are taken with LAPACK's
symmetric eigensolver (Sec. 3 names LAPACK for this step).

Readings where the paper is silent (it states the scalar recursion only):
* full reorthogonalisation: after the three-term step, W is projected out of
  all previous blocks twice (classical Gram-Schmidt, two passes);
* in-block QR: modified Gram-Schmidt, two passes per column, columns taken in
  order; a column whose norm after orthogonalisation is below `defl_tol`
  (absolute, eV) is dropped (deflation), so later blocks may be narrower;
* the iteration stops after r blocks or when a block is empty (the Krylov space
  is invariant: r has reached the minimal-polynomial degree of Sec. 3).
"""
import numpy as np


def _inblock_qr(W, defl_tol):
    """W = Q R with orthonormal kept columns Q (D x b) and R (b x W.shape[1])."""
    D, m = W.shape
    kept = []
    coeffs = []            # per input column: dict kept-index -> coefficient
    for c in range(m):
        w = W[:, c].copy()
        co = np.zeros(m)
        for _ in range(2):
            for j, q in enumerate(kept):
                h = q @ w
                w = w - h * q
                co[j] += h
        nrm = np.sqrt(w @ w)
        if nrm > defl_tol:
            co[len(kept)] = nrm
            kept.append(w / nrm)
        coeffs.append(co)
    b = len(kept)
    Q = np.array(kept).T if b else np.zeros((D, 0))
    R = np.array(coeffs).T[:b, :] if b else np.zeros((0, m))
    return Q, R


def block_lanczos(Hc, r, defl_tol, seed_slot=0):
    """Orthonormal basis V (D x kdim) of the block Krylov space of order r seeded
    with the four orbitals of cluster slot `seed_slot`, and T = V^T Hc V."""
    D = Hc.shape[0]
    V1 = np.zeros((D, 4))
    V1[4 * seed_slot:4 * seed_slot + 4, :] = np.eye(4)
    blocks = [V1]
    V_prev, B_prev = np.zeros((D, 0)), np.zeros((4, 0))
    for k in range(r - 1):
        Vk = blocks[-1]
        W = Hc @ Vk - V_prev @ B_prev.T
        A = Vk.T @ W
        W = W - Vk @ A
        Q = np.concatenate(blocks, axis=1)
        for _ in range(2):
            W = W - Q @ (Q.T @ W)
        Vn, B = _inblock_qr(W, defl_tol)
        if Vn.shape[1] == 0:
            break
        V_prev, B_prev = Vk, B
        blocks.append(Vn)
    V = np.concatenate(blocks, axis=1)
    T = V.T @ Hc @ V
    T = 0.5 * (T + T.T)
    return V, T, [b.shape[1] for b in blocks]


def spectral_record(V, T, nbr_slots):
    """Eigenpairs of T and the pieces of the density-matrix columns.

    Returns lam (kdim), S = U[0:4, :] (the seed block's components of each
    eigenvector), P = V[rows of nbr_slots, :] @ U  ((len(nbr_slots)*4) x kdim).
    With f_m = f(lam_m), rho[j b, i a] = sum_m P[(j,b), m] f_m S[a, m].
    """
    lam, U = np.linalg.eigh(T)
    S = U[0:4, :]
    rows = np.concatenate([np.arange(4 * s, 4 * s + 4) for s in nbr_slots])
    P = V[rows, :] @ U
    return lam, S, P
