"""Kohn-Sham-like Hamiltonian of the model systems (oracle; test infrastructure).

H = -1/2 nabla^2 + V_loc + V_NL with V_NL = sum_j |beta_j> D_j <beta_j| (Kleinman-Bylander form),
acting on plane-wave coefficients. This is the single-particle operator of the ground state
(paper Sec. 2.1, Eq. (1)) whose occupied eigenpairs (psi_v, eps_v) the response calculation uses.

Two independent constructions:
  * ``apply``: the grid operator 1/2|G|^2 c + fft_n(V_loc * ifft_u(c)) + V_NL c;
  * ``dense``: the explicit matrix H[G, G'] = 1/2|G|^2 delta + Vhat(G - G') + sum_j beta_j(G) D_j
    conj(beta_j(G')) with Vhat = fft_n(V_loc) read at (G - G') mod N.
They agree exactly when the grid holds every difference G - G' without wrap-around.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse.linalg

from . import basis

DENSE_MAX = 6000  # largest real dimension diagonalised densely


class Hamiltonian:
    def __init__(self, system):
        self.system = system
        self.grid = tuple(system.grid)
        self.omega = system.omega
        self.m = system.npw_h
        self.miller_half = np.asarray(system.miller)
        self.miller = basis.full_miller(self.miller_half)
        bvec = 2.0 * np.pi * np.linalg.inv(np.asarray(system.cell)).T
        self.gvec = self.miller.astype(np.float64) @ bvec
        self.g2 = np.einsum("ij,ij->i", self.gvec, self.gvec)
        self.vloc = np.asarray(system.vloc_r, dtype=np.float64)
        self.beta = basis.expand(np.asarray(system.beta))  # (nproj, npw)
        self.dij = np.asarray(system.dij, dtype=np.float64)

    @property
    def npw(self) -> int:
        return self.miller.shape[0]

    def kinetic(self, c):
        return 0.5 * self.g2 * c

    def local(self, c):
        f = basis.ifft_u(basis.to_box(c, self.miller, self.grid))
        return basis.from_box(basis.fft_n(self.vloc * f), self.miller, self.grid)

    def nonlocal_(self, c):
        proj = np.conj(self.beta) @ np.atleast_2d(c).T  # (nproj, B): <beta_j|c>
        out = (self.beta.T @ (self.dij[:, None] * proj)).T
        return out.reshape(np.shape(c))

    def apply(self, c: np.ndarray) -> np.ndarray:
        """H c for full-sphere coefficient vectors c of shape (..., npw)."""
        return self.kinetic(c) + self.local(c) + self.nonlocal_(c)

    def dense(self) -> np.ndarray:
        """Explicit complex Hermitian matrix of H on the full sphere."""
        n1, n2, n3 = self.grid
        vhat = basis.fft_n(self.vloc.astype(np.complex128))
        d = self.miller[:, None, :] - self.miller[None, :, :]
        h = vhat[np.mod(d[..., 2], n3), np.mod(d[..., 1], n2), np.mod(d[..., 0], n1)]
        h = h + np.diag(0.5 * self.g2)
        h = h + (self.beta.T * self.dij[None, :]) @ np.conj(self.beta)
        return h

    def dense_real(self) -> np.ndarray:
        """Real symmetric matrix of H in the real orthonormal basis of real functions."""
        phi = basis.real_isometry(self.m)
        h = np.conj(phi.T) @ self.dense() @ phi
        return 0.5 * (h.real + h.real.T)

    def ground_state(self, nstates: int, tol: float = 1e-13):
        """Lowest ``nstates`` eigenpairs: (eps ascending, psi as half-sphere rows, real in r)."""
        n = 2 * self.m - 1
        if n <= DENSE_MAX:
            w, v = scipy.linalg.eigh(self.dense_real(), subset_by_index=[0, nstates - 1])
        else:

            def mv(q):
                q = np.asarray(q).reshape(-1)
                c = basis.expand(basis.real_to_half(q))
                return basis.half_to_real(basis.fold(self.apply(c)))

            op = scipy.sparse.linalg.LinearOperator((n, n), matvec=mv, dtype=np.float64)
            w, v = scipy.sparse.linalg.eigsh(op, k=nstates, which="SA", tol=tol, ncv=min(n, max(2 * nstates + 1, nstates + 64)))
            order = np.argsort(w)
            w, v = w[order], v[:, order]
        psi = basis.real_to_half(v.T)
        return w, psi

    def all_states(self):
        """Full spectrum (dense): eps ascending and every eigenvector as half-sphere rows."""
        w, v = scipy.linalg.eigh(self.dense_real())
        return w, basis.real_to_half(v.T)
