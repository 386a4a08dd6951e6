"""Brute-force discrete Fourier sums (test infrastructure; pins the oracle's FFT convention).

Direct O(N^6) evaluation of the two grid transforms used throughout the oracle:
  G -> r:  f(r_i) = sum_G c(G) exp(+2 pi i sum_j n_j i_j / N_j)
  r -> G:  c(G)   = (1/N1 N2 N3) sum_i f(r_i) exp(-2 pi i sum_j n_j i_j / N_j)
Only for tiny grids.
"""

from __future__ import annotations

import numpy as np


def g_to_r(c_full: np.ndarray, miller_full: np.ndarray, grid) -> np.ndarray:
    n1, n2, n3 = grid
    i3, i2, i1 = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    out = np.zeros((n3, n2, n1), dtype=np.complex128)
    for c, (a, b, d) in zip(c_full, miller_full):
        out += c * np.exp(2j * np.pi * (a * i1 / n1 + b * i2 / n2 + d * i3 / n3))
    return out


def r_to_g(f: np.ndarray, miller_full: np.ndarray, grid) -> np.ndarray:
    n1, n2, n3 = grid
    i3, i2, i1 = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    out = np.empty(len(miller_full), dtype=np.complex128)
    for k, (a, b, d) in enumerate(miller_full):
        out[k] = np.sum(f * np.exp(-2j * np.pi * (a * i1 / n1 + b * i2 / n2 + d * i3 / n3)))
    return out / (n1 * n2 * n3)
