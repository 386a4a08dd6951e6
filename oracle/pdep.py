"""Projective dielectric eigendecomposition (PDEP) of chi0bar (oracle; test infrastructure).

Paper Sec. 2.1, Eq. (5): chi0bar is diagonalised iteratively; its eigenvalues lambda_a and
eigenvectors phibar_a (N_PDEP of them) give the low-rank form of chi-bar. Sec. 3.3 states that
PDEP and the BSE/TDDFT problems share one Davidson implementation. The paper fixes no Davidson
parameters; the reading used here:

* target: the ``neig`` algebraically lowest eigenvalues (chi0bar is negative semidefinite, so
  these are the largest screening eigenvalues 1 - lambda);
* start: an orthonormal block (given); expansion by the plain residuals of the unconverged Ritz
  pairs (no preconditioner: chi0bar has no cheap diagonal); two-pass classical Gram-Schmidt,
  vectors whose norm after projection is below ``drop`` are discarded; when the basis would
  exceed ``nbasis_max`` it restarts from the current ``neig`` Ritz vectors;
* converged when ||chi0bar x_a - lambda_a x_a|| <= tol for every a <= neig.

Vectors are half-sphere coefficient rows; the linear algebra runs on their real coordinates
(basis.half_to_real), where the Gamma-point inner product is the plain dot product.
"""

from __future__ import annotations

import numpy as np

from . import basis


def _orthonormalise_against(V: np.ndarray, X: np.ndarray, drop: float) -> np.ndarray:
    """Columns of X made orthonormal to V's columns and to each other (two-pass CGS)."""
    keep = []
    for j in range(X.shape[1]):
        x = X[:, j] / np.linalg.norm(X[:, j])
        basis_cols = [V] + ([np.stack(keep, axis=1)] if keep else [])
        B = np.concatenate(basis_cols, axis=1) if V.size or keep else np.zeros((X.shape[0], 0))
        for _pass in range(2):
            if B.shape[1]:
                x = x - B @ (B.T @ x)
        n = np.linalg.norm(x)
        if n >= drop:
            keep.append(x / n)
    return np.stack(keep, axis=1) if keep else np.zeros((X.shape[0], 0))


def davidson(apply_half, guess_half, neig, nbasis_max=None, maxiter=100, tol=1e-10, drop=1e-12):
    """Block Davidson for the lowest ``neig`` eigenpairs of the operator ``apply_half``.

    apply_half maps half-sphere rows (n, m) to half-sphere rows (n, m). Returns a dict with
    ``lam`` (neig ascending), ``vec`` (neig, m), ``iters``, ``napply`` (vectors applied) and
    ``resnorm`` (neig).
    """
    nbasis_max = nbasis_max or 4 * neig
    q0 = basis.half_to_real(np.atleast_2d(guess_half)).T  # (n, k)
    V = _orthonormalise_against(np.zeros((q0.shape[0], 0)), q0, drop)
    W = basis.half_to_real(apply_half(basis.real_to_half(V.T))).T
    napply = V.shape[1]
    lam = rn = X = None
    for it in range(1, maxiter + 1):
        hs = V.T @ W
        hs = 0.5 * (hs + hs.T)
        theta, Y = np.linalg.eigh(hs)
        lam = theta[:neig]
        X = V @ Y[:, :neig]
        AX = W @ Y[:, :neig]
        R = AX - X * lam[None, :]
        rn = np.linalg.norm(R, axis=0)
        conv = rn <= tol
        if conv.all():
            break
        if it == maxiter:
            break
        if V.shape[1] + int((~conv).sum()) > nbasis_max:
            V, W = X, AX
        new = _orthonormalise_against(V, R[:, ~conv], drop)
        if new.shape[1] == 0:
            break
        Wn = basis.half_to_real(apply_half(basis.real_to_half(new.T))).T
        napply += new.shape[1]
        V = np.concatenate([V, new], axis=1)
        W = np.concatenate([W, Wn], axis=1)
    return {"lam": lam, "vec": basis.real_to_half(X.T), "iters": it, "napply": napply, "resnorm": rn}


def dense_eigs(chi_real: np.ndarray, neig: int):
    """Lowest ``neig`` eigenvalues of an explicit real symmetric chi0bar matrix."""
    w = np.linalg.eigvalsh(chi_real)
    return w[:neig]


def chibar_lowrank(lam: np.ndarray, q: np.ndarray) -> np.ndarray:
    """chi-bar of Eq. (5) without Xi: sum_a q_a lam_a / (1 - lam_a) q_a^T (real coordinates).

    q: (neig, d) orthonormal rows (the PDEP eigenvectors in real coordinates). With orthonormal
    plane-wave coefficient vectors the 1/Omega of Eq. (5) is absorbed: it belongs to the paper's
    real-space normalisation of the eigenpotentials. RPA: chi = chi0 + chi0 chi, so with every
    eigenpair this equals (1 - chi0)^-1 chi0.
    """
    lam = np.asarray(lam, dtype=np.float64)
    return (q.T * (lam / (1.0 - lam))[None, :]) @ q


def wp_apply(lam: np.ndarray, phibar_half: np.ndarray, vhalf_half: np.ndarray, x_half: np.ndarray) -> np.ndarray:
    """W_p x = v^1/2 chi-bar v^1/2 x for half-sphere rows x, chi-bar from chibar_lowrank."""
    q = basis.half_to_real(np.atleast_2d(phibar_half))
    y = basis.half_to_real(vhalf_half[None, :] * np.atleast_2d(x_half))
    z = (chibar_lowrank(lam, q) @ y.T).T
    return vhalf_half[None, :] * basis.real_to_half(z)
