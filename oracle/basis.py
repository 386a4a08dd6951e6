"""Plane-wave basis helpers of the oracle (test infrastructure; see the package docstring).

Basis: orthonormal plane waves b_G(r) = Omega^-1/2 exp(i G.r) on the sphere |G|^2 <= ecut. A
real function has coefficients with c(-G) = conj(c(G)). The interface stores only the half sphere
(G = 0 first); here vectors are expanded to the full sphere, ordered [half..., -(half[1:])...].

Grid transforms (numpy shape (n3, n2, n1); the frequency n sits at index n mod N):
  ifft_u(c)(r) = sum_G c(G) exp(i G.r)               (unnormalised, G -> r)
  fft_n(f)(G)  = (1/N^3) sum_r f(r) exp(-i G.r)       (normalised, r -> G)
so fft_n(ifft_u(c)) = c, and the matrix element of a local potential is
<b_G|V|b_G'> = fft_n(V)(G - G').
"""

from __future__ import annotations

import os

import numpy as np
import scipy.fft

# FFT threads: every core the process may use, unless ORACLE_FFT_WORKERS says otherwise (a pool of
# oracle processes gives each a share)
_WORKERS = int(os.environ.get("ORACLE_FFT_WORKERS", "0")) or max(
    1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


def full_miller(miller_half: np.ndarray) -> np.ndarray:
    """Full-sphere Miller indices: the half sphere followed by the mirrors of its G != 0."""
    return np.concatenate([miller_half, -miller_half[1:]], axis=0)


def expand(c_half: np.ndarray) -> np.ndarray:
    """Half-sphere coefficients (..., m) -> full sphere (..., 2m-1) of a real function."""
    return np.concatenate([c_half, np.conj(c_half[..., 1:])], axis=-1)


def fold(c_full: np.ndarray) -> np.ndarray:
    """Full-sphere coefficients (..., 2m-1) -> the half-sphere part (..., m)."""
    m = (c_full.shape[-1] + 1) // 2
    return c_full[..., :m].copy()


def box_index(miller_full: np.ndarray, grid) -> tuple:
    """Flat (i3, i2, i1) positions of the sphere's frequencies in a (n3, n2, n1) box."""
    n1, n2, n3 = grid
    return (np.mod(miller_full[:, 2], n3), np.mod(miller_full[:, 1], n2), np.mod(miller_full[:, 0], n1))


def to_box(c_full: np.ndarray, miller_full: np.ndarray, grid) -> np.ndarray:
    """Scatter full-sphere coefficients (..., npw) into zero boxes (..., n3, n2, n1)."""
    n1, n2, n3 = grid
    box = np.zeros(c_full.shape[:-1] + (n3, n2, n1), dtype=np.complex128)
    i3, i2, i1 = box_index(miller_full, grid)
    box[..., i3, i2, i1] = c_full
    return box


def from_box(box: np.ndarray, miller_full: np.ndarray, grid) -> np.ndarray:
    """Gather the sphere's frequencies from boxes (..., n3, n2, n1)."""
    i3, i2, i1 = box_index(miller_full, grid)
    return box[..., i3, i2, i1]


def ifft_u(box: np.ndarray) -> np.ndarray:
    """sum_G c(G) exp(iG.r) on the grid (numpy's inverse FFT times the number of points)."""
    n = box.shape[-1] * box.shape[-2] * box.shape[-3]
    return scipy.fft.ifftn(box, axes=(-3, -2, -1), workers=_WORKERS) * n


def fft_n(f: np.ndarray) -> np.ndarray:
    """(1/N^3) sum_r f(r) exp(-iG.r) on the grid (numpy's forward FFT over the point count)."""
    n = f.shape[-1] * f.shape[-2] * f.shape[-3]
    return scipy.fft.fftn(f, axes=(-3, -2, -1), workers=_WORKERS) / n


def to_real_space(c_full: np.ndarray, miller_full: np.ndarray, grid) -> np.ndarray:
    """Real function on the grid from full-sphere coefficients (imaginary rounding dropped)."""
    return ifft_u(to_box(c_full, miller_full, grid)).real


def to_sphere(f: np.ndarray, miller_full: np.ndarray, grid) -> np.ndarray:
    """Full-sphere coefficients of the normalised transform of grid data."""
    return from_box(fft_n(f), miller_full, grid)


def dot(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """<a|b> = sum_G conj(a(G)) b(G) over the full sphere, batched over leading axes."""
    return np.sum(np.conj(a) * b, axis=-1)


def real_isometry(m: int) -> np.ndarray:
    """Matrix Phi (2m-1 x 2m-1 complex) mapping real coordinates q to full-sphere coefficients.

    q = [c(0), sqrt2 Re c(G_1..), sqrt2 Im c(G_1..)] for the half-sphere G != 0. Phi is an isometry
    onto the real-in-r functions, so Phi^dagger A Phi is the real symmetric matrix of any
    Hermitian operator A that maps real functions to real functions.
    """
    n = 2 * m - 1
    phi = np.zeros((n, n), dtype=np.complex128)
    phi[0, 0] = 1.0
    s = 1.0 / np.sqrt(2.0)
    k = np.arange(1, m)
    # coordinate Re: c(G) = q/sqrt2, c(-G) = q/sqrt2 ; coordinate Im: c(G) = i q/sqrt2, c(-G) = -i q/sqrt2
    phi[k, k] = s
    phi[k + m - 1, k] = s
    phi[k, k + m - 1] = 1j * s
    phi[k + m - 1, k + m - 1] = -1j * s
    return phi


def half_to_real(c_half: np.ndarray) -> np.ndarray:
    """Half-sphere coefficients -> real coordinates q (see real_isometry)."""
    return np.concatenate(
        [c_half[..., :1].real, np.sqrt(2.0) * c_half[..., 1:].real, np.sqrt(2.0) * c_half[..., 1:].imag], axis=-1
    )


def real_to_half(q: np.ndarray) -> np.ndarray:
    """Real coordinates q -> half-sphere coefficients."""
    m = (q.shape[-1] + 1) // 2
    out = np.empty(q.shape[:-1] + (m,), dtype=np.complex128)
    out[..., 0] = q[..., 0]
    out[..., 1:] = (q[..., 1:m] + 1j * q[..., m:]) / np.sqrt(2.0)
    return out
