"""Density-functional perturbation theory for chi0bar (oracle; test infrastructure).

Paper Sec. 2.1: W_p = v^1/2 chi0bar v^1/2 ... chi0bar is the symmetrised irreducible response
v^1/2 chi0 v^1/2; the density response is evaluated within DFPT by solving the Sternheimer
equation, without empty states. Readings of details the paper does not spell out:

* Orbitals: closed shell, real in r (Gamma point), normalised sum_G |c_v(G)|^2 = 1 over the full
  sphere; psi_v(r) = Omega^-1/2 ifft_u(c_v)(r).
* Perturbation phi (orthonormal plane-wave coefficients, G = 0 entry zero). Coulomb factor
  v^1/2(G) = sqrt(4 pi)/|G| for G != 0 and 0 at G = 0. The potential is
  dV(r) = Omega^-1/2 ifft_u(v^1/2 phi)(r).
* Sternheimer equation for each occupied v: (H - eps_v) dpsi_v = -Q dV psi_v with
  Q = 1 - sum_v' |psi_v'><psi_v'|, whose unique solution in the range of Q equals the solution of
  the positive-definite system (H - eps_v + alpha P) dpsi_v = -Q dV psi_v, P = 1 - Q,
  alpha = eps_max - eps_min + 1 hartree. Solved by conjugate gradients preconditioned with the
  Teter-Payne-Allan (TPA) function of x = (1/2|G|^2) / T_v, T_v the kinetic energy of psi_v.
* Density response of the closed shell: drho(r) = 4 sum_v psi_v(r) dpsi_v(r) (factor 2 for spin
  and 2 for psi dpsi* + c.c. with real orbitals).
* Output chi0bar phi = v^1/2 drho(G) with drho(G) = <b_G|drho>.

With the Omega factors collected, for coefficient vectors (tilde: unnormalised transforms):
  b_v   = -Q fft_n(ifft_u(x) * ifft_u(c_v)),  x = v^1/2 phi
  d_v   = A_v^-1 b_v
  drho  = (4/Omega) fft_n(sum_v ifft_u(c_v) * ifft_u(d_v))
  out   = v^1/2 drho
"""

from __future__ import annotations

import numpy as np

from . import basis


TKIN_FLOOR = 1e-3  # hartree


def tpa(x: np.ndarray) -> np.ndarray:
    """Teter-Payne-Allan preconditioner K(x) = P(x) / (P(x) + 16 x^4), P = 27+18x+12x^2+8x^3.

    (Phys. Rev. B 40, 12255 (1989).) K(0) = 1 and K ~ 1/(2x) for large x.
    """
    p = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x))
    return p / (p + 16.0 * x ** 4)


class Response:
    """chi0bar of one system, given its occupied ground state (eps_v, c_v)."""

    def __init__(self, ham, eps: np.ndarray, psi_half: np.ndarray, alpha: float | None = None):
        self.H = ham
        self.eps = np.asarray(eps, dtype=np.float64)
        self.nocc = len(self.eps)
        self.psi = basis.expand(np.asarray(psi_half))  # (nocc, npw) full sphere
        self.psi_r = basis.to_real_space(self.psi, ham.miller, ham.grid)  # ifft_u(c_v), real
        self.alpha = float(self.eps.max() - self.eps.min() + 1.0) if alpha is None else float(alpha)
        # kinetic energy of each orbital, floored so that a constant orbital (T = 0) still
        # gets a finite preconditioner; the floor changes iteration counts, never the result
        self.tkin = np.maximum(np.real(np.sum(0.5 * ham.g2 * np.abs(self.psi) ** 2, axis=-1)), TKIN_FLOOR)
        g = np.sqrt(ham.g2)
        self.vhalf = np.zeros_like(g)
        self.vhalf[1:] = np.sqrt(4.0 * np.pi) / g[1:]  # G = 0 is entry 0 of the full sphere

    # -- operators on full-sphere vectors, batched over rows ------------------------------------
    def project_p(self, x):
        """P x = sum_v psi_v <psi_v|x>."""
        s = np.conj(self.psi) @ x.T  # (nocc, B)
        return (self.psi.T @ s).T

    def project_q(self, x):
        return x - self.project_p(x)

    def shifted(self, x, eps_rows):
        """A x = (H - eps_v) x + alpha P x, one eps per row."""
        return self.H.apply(x) - eps_rows[:, None] * x + self.alpha * self.project_p(x)

    def rhs(self, x_pert, vidx):
        """b_v = -Q fft_n(ifft_u(x) * ifft_u(c_v)) for rows (perturbation row, orbital index)."""
        dv_r = basis.to_real_space(x_pert, self.H.miller, self.H.grid)
        prod = dv_r * self.psi_r[vidx]
        return -self.project_q(basis.to_sphere(prod, self.H.miller, self.H.grid))

    def tpa_rows(self, vidx):
        """TPA preconditioner K(1/2 |G|^2 / T_v) for the orbital of each row (full sphere)."""
        return tpa(0.5 * self.H.g2[None, :] / self.tkin[np.asarray(vidx)][:, None])

    def sternheimer(self, b, vidx, tol=1e-13, maxiter=5000, precondition=True):
        """Solve A_v d = b row by row by preconditioned CG (FP64).

        ``precondition``: True for TPA, False for none, or an array of diagonal preconditioner
        values (rows x plane waves), e.g. a learned scale times TPA.

        Stops a row when the recursive residual satisfies ||r|| <= tol ||b||, then recomputes
        the true residual b - A d; rows whose true residual is still above tol restart from the
        current iterate. Returns (d, iterations per row, true relative residual per row).
        """
        b = np.asarray(b, dtype=np.complex128)
        nrow = b.shape[0]
        eps_rows = self.eps[vidx]
        if isinstance(precondition, np.ndarray):  # an explicit diagonal preconditioner per row
            kprec = np.broadcast_to(np.asarray(precondition, dtype=np.float64), b.shape)
        elif precondition:
            kprec = self.tpa_rows(vidx)
        else:
            kprec = np.ones((nrow, b.shape[1]))
        bnorm = np.sqrt(np.real(basis.dot(b, b)))
        bnorm = np.where(bnorm > 0, bnorm, 1.0)
        d = np.zeros_like(b)
        iters = np.zeros(nrow, dtype=np.int64)
        done = np.zeros(nrow, dtype=bool)
        true_rel = np.full(nrow, np.inf)
        for _restart in range(8):
            act = np.nonzero(~done)[0]
            if act.size == 0:
                break
            r = b[act] - (self.shifted(d[act], eps_rows[act]) if np.any(d[act]) else 0.0)
            z = kprec[act] * r
            p = z.copy()
            rz = np.real(basis.dot(r, z))
            live = np.ones(act.size, dtype=bool)
            for _ in range(maxiter):
                if not live.any():
                    break
                li = np.nonzero(live)[0]
                rows = act[li]
                ap = self.shifted(p[li], eps_rows[rows])
                pap = np.real(basis.dot(p[li], ap))
                a = rz[li] / pap
                d[rows] += a[:, None] * p[li]
                r[li] -= a[:, None] * ap
                iters[rows] += 1
                rn = np.sqrt(np.real(basis.dot(r[li], r[li])))
                stop = rn <= tol * bnorm[rows]
                z_new = kprec[rows] * r[li]
                rz_new = np.real(basis.dot(r[li], z_new))
                beta = rz_new / rz[li]
                p[li] = z_new + beta[:, None] * p[li]
                rz[li] = rz_new
                live[li[stop]] = False
                if iters[rows].max() >= maxiter:
                    break
            res = b[act] - self.shifted(d[act], eps_rows[act])
            true_rel[act] = np.sqrt(np.real(basis.dot(res, res))) / bnorm[act]
            done[act] = true_rel[act] <= tol
            if iters.max() >= maxiter:
                break
        return d, iters, true_rel

    def vhalf_times(self, phi_half):
        return self.vhalf * basis.expand(np.asarray(phi_half, dtype=np.complex128))

    def density(self, d, vidx, npert, pidx):
        """drho(G) = (4/Omega) fft_n(sum_v ifft_u(c_v) ifft_u(d_v)), per perturbation (full sphere)."""
        d_r = basis.to_real_space(d, self.H.miller, self.H.grid)
        acc = np.zeros((npert,) + d_r.shape[1:])
        for k in range(d.shape[0]):
            acc[pidx[k]] += self.psi_r[vidx[k]] * d_r[k]
        return (4.0 / self.H.omega) * basis.to_sphere(acc, self.H.miller, self.H.grid)

    def apply(self, phi_half, tol=1e-13, maxiter=5000, precondition=True, solver="cg"):
        """chi0bar phi for half-sphere rows phi (npert, m).

        Returns dict with ``out`` (npert, m) = v^1/2 drho, ``drho`` (npert, m), and per-solve
        ``iters`` / ``residual`` (rows ordered perturbation-major, orbital-minor).
        """
        phi_half = np.atleast_2d(phi_half)
        npert = phi_half.shape[0]
        x = self.vhalf_times(phi_half)
        pidx = np.repeat(np.arange(npert), self.nocc)
        vidx = np.tile(np.arange(self.nocc), npert)
        b = self.rhs(x[pidx], vidx)
        if solver == "cg":
            d, iters, res = self.sternheimer(b, vidx, tol=tol, maxiter=maxiter, precondition=precondition)
        else:
            d, iters, res = solver(b, vidx), np.zeros(len(vidx), dtype=np.int64), np.zeros(len(vidx))
        drho = self.density(d, vidx, npert, pidx)
        out = self.vhalf * drho
        return {
            "out": basis.fold(out),
            "drho": basis.fold(drho),
            "iters": iters,
            "residual": res,
            "dpsi": d,
        }


def sos_solver(resp: Response, eps_all: np.ndarray, psi_all_half: np.ndarray):
    """Sum over states: d_v = sum_{c > nocc} psi_c <psi_c|b> / (eps_c - eps_v) (dense spectrum).

    For b in the range of Q this is the exact solution of the Sternheimer equation, i.e. the
    Adler-Wiser sum over empty states that DFPT avoids (paper Sec. 2.1).
    """
    psi_c = basis.expand(np.asarray(psi_all_half)[resp.nocc:])
    eps_c = np.asarray(eps_all)[resp.nocc:]

    def solve(b, vidx):
        coef = np.conj(psi_c) @ b.T  # (nc, B)
        coef = coef / (eps_c[:, None] - resp.eps[vidx][None, :])
        return (psi_c.T @ coef).T

    return solve


def adler_wiser_chi0bar(ham, eps_all: np.ndarray, psi_all_half: np.ndarray, nocc: int) -> np.ndarray:
    """Explicit real symmetric matrix of chi0bar on the real basis of G != 0 (dimension npw - 1).

    chi0(G, G') = 4 sum_{v <= nocc < c} M_vc(G) conj(M_vc(G')) / (eps_v - eps_c) with the pair
    matrix elements M_vc(G) = <b_G|psi_v psi_c> = Omega^-1/2 fft_n(ifft_u(c_v) ifft_u(c_c))(G);
    chi0bar = v^1/2 chi0 v^1/2, restricted to G != 0 and expressed in the real coordinates.
    """
    psi_all = basis.expand(np.asarray(psi_all_half))
    psi_r = basis.to_real_space(psi_all, ham.miller, ham.grid)
    g = np.sqrt(ham.g2)
    vhalf = np.zeros_like(g)
    vhalf[1:] = np.sqrt(4.0 * np.pi) / g[1:]
    npw = ham.npw
    chi = np.zeros((npw, npw), dtype=np.complex128)
    for v in range(nocc):
        mv = basis.to_sphere(psi_r[v][None] * psi_r[nocc:], ham.miller, ham.grid) / np.sqrt(ham.omega)
        w = 4.0 / (eps_all[v] - eps_all[nocc:])
        chi += (mv.T * w[None, :]) @ np.conj(mv)
    chi = vhalf[:, None] * chi * vhalf[None, :]
    phi = basis.real_isometry(ham.m)
    cr = np.conj(phi.T) @ chi @ phi
    cr = 0.5 * (cr.real + cr.real.T)
    return cr[1:, 1:]  # drop the G = 0 coordinate (v^1/2 vanishes there)
