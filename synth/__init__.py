"""Seeded synthetic model systems and perturbations.

This module only *describes* inputs: a periodic cell, its plane-wave sphere, a local potential
sampled on the FFT grid, Kleinman-Bylander projector values and random perturbation vectors. It
holds none of the arithmetic of the response calculation (no Hamiltonian application, no FFT, no
eigensolver, no Sternheimer solve, no density response). Both the FP64 oracle and the GPU library
consume the arrays made here; neither shares any other code with the other.

Model (the paper's workloads are real materials computed with pwscf ground states; these seeded
Gaussian-well systems stand in for them):

* Cubic cell of side L (bohr), FFT grid n1 x n2 x n3, plane-wave set {G : |G|^2 <= ecut}
  (ecut in bohr^-2, i.e. the kinetic energy 0.5|G|^2 of the largest wave is ecut/2 hartree).
* Local potential V_loc(r) = -A sum_I sum_T exp(-|r - R_I - T|^2 / (2 sigma^2)), a sum over
  atoms I and lattice images T, sampled at r = (i1/n1, i2/n2, i3/n3) L.
* Kleinman-Bylander projectors with a Gaussian radial form of width sigma_beta: per atom one s
  projector and optionally a p triplet. In reciprocal space
  beta_s(G) ~ exp(-|G|^2 sigma_beta^2 / 2) exp(-i G.R) and
  beta_p,a(G) ~ -i G_a exp(-|G|^2 sigma_beta^2 / 2) exp(-i G.R), each normalised over the full
  sphere. The strengths D are diagonal: D_s for s, D_p for p.
* Perturbations: Gaussian random coefficients on the half sphere without G = 0, orthonormalised
  in the Gamma-point inner product.

Storage conventions (shared interface of oracle and library):

* Half sphere ("Gamma storage"): G = (n1, n2, n3) with n3 > 0, or n3 = 0 and n2 > 0, or
  n3 = n2 = 0 and n1 >= 0. Sorted by (|n|^2, n1, n2, n3); G = 0 is first. A real function f has
  f(-G) = conj(f(G)), so the half sphere determines it.
* Grid arrays have numpy shape (n3, n2, n1) in C order: element [i3, i2, i1] sits at
  r = (i1/n1, i2/n2, i3/n3) L, so the first axis of the cell is the fastest in memory.
* Complex arrays are numpy complex128 (interleaved re, im).

Random numbers come from splitmix64 (Steele, Lea and Flood, OOPSLA 2014), which gives identical
streams on every platform and numpy version; normals come from the Box-Muller transform.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

__all__ = [
    "SystemSpec",
    "System",
    "SPECS",
    "BATCH_GRIDS",
    "batch_family",
    "GRID_SIZES",
    "grid_probe",
    "learned_family",
    "spec",
    "make_system",
    "make_perturbations",
    "make_guess",
    "half_sphere",
    "splitmix64",
    "uniform01",
    "normal",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """``count`` outputs of splitmix64 for state ``seed`` (with a stream offset), as uint64.

    Output i is the finaliser applied to seed + (stream * 2^32 + i + 1) * golden, which is
    the i-th output of the sequential generator started at that state.
    """
    idx = np.arange(count, dtype=np.uint64) + np.uint64(1) + np.uint64(stream) * np.uint64(1 << 32)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """Uniform doubles in (0, 1] from the top 53 bits of splitmix64."""
    z = splitmix64(seed, count, stream)
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def normal(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """Standard normal doubles by Box-Muller on pairs of uniforms."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m, stream)
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    t = 2.0 * np.pi * u[1::2]
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(t)
    out[1::2] = r * np.sin(t)
    return out[:count]


@dataclasses.dataclass(frozen=True)
class SystemSpec:
    """Parameters of one seeded model system (lengths in bohr, energies in hartree)."""

    name: str
    L: float
    grid: tuple
    ecut: float
    natom: int
    nocc: int
    well_depth: float = 4.0
    sigma: float = 1.0
    beta_sigma: float = 0.8
    d_s: float = 2.0
    d_p: Optional[float] = None  # None: s projectors only
    min_dist: float = 3.0
    seed: int = 0


# Named workloads. The first three follow the tiny / medium / precision configurations of the
# benchmark description; "small" and "ragged" are parity cases that finish in seconds on the CPU
# while spanning several GPU tiles with ragged tails (ragged: a 30^3 grid, radices 2, 3 and 5).
# Two occupied orbitals per atom (valence charge 4) sit inside the p / d manifold of a Gaussian
# well unless the levels are rearranged. The medium and precision systems therefore use deeper
# wells (12 hartree), an attractive s projector (D_s = -2), a repulsive p projector (D_p = +5) and
# atoms at least 5 bohr (4.5 in the denser precision cell) apart: 1s and 2s form narrow bands
# below the d-like levels, and the oracle finds a HOMO-LUMO gap of 0.47 hartree for the medium
# system (at least 0.1 hartree is required). The tiny system keeps the literal parameters
# (4 hartree wells, one s projector with D = +2, 3 bohr); its gap is 0.0069 hartree.
SPECS = {
    "tiny": SystemSpec("tiny", 10.0, (24, 24, 24), 10.0, 2, 4, 4.0, 1.0, 0.8, 2.0, None, 3.0, 0),
    "small": SystemSpec("small", 10.0, (24, 24, 24), 14.0, 2, 4, 8.0, 1.0, 0.8, -2.0, 5.0, 3.0, 1),
    "ragged": SystemSpec("ragged", 11.0, (30, 30, 30), 16.0, 3, 6, 8.0, 1.0, 0.8, -2.0, 5.0, 3.0, 2),
    "medium": SystemSpec("medium", 20.0, (64, 64, 64), 25.0, 32, 64, 12.0, 1.0, 0.8, -2.0, 5.0, 5.0, 0),
    "precision": SystemSpec("precision", 28.0, (96, 96, 96), 25.0, 128, 256, 12.0, 1.0, 0.8, -2.0, 5.0, 4.5, 0),
    # the precision system's cell, grid, cutoff and plane-wave layout (23,149 stored waves, the
    # same compile-time kernels) with 8 atoms and 16 orbitals, so that the oracle finishes in
    # about a minute
    "precision_reduced": SystemSpec("precision_reduced", 28.0, (96, 96, 96), 25.0, 8, 16, 12.0, 1.0, 0.8, -2.0, 5.0, 4.5, 0),
}


# The batching workload: systems of uneven size on 2,3,5-smooth grids from 32^3 to 80^3, the cell
# growing with the grid at the spacing of the precision system (L = 28 n / 96 bohr, same cutoff)
# and one atom per 171 bohr^3 as there, two occupied orbitals per atom, the precision system's
# wells and projectors. Sizes: 5 atoms / 10 orbitals (32^3) to 74 atoms / 148 orbitals (80^3).
BATCH_GRIDS = (32, 36, 40, 45, 48, 50, 54, 60, 64, 72, 75, 80, 40, 48, 60, 64)


def batch_family(count: int = 16, seed: int = 0) -> list:
    """Specs of ``count`` systems of the batching workload (deterministic in ``seed``)."""
    out = []
    for k in range(count):
        n = BATCH_GRIDS[k % len(BATCH_GRIDS)]
        L = n * 28.0 / 96.0
        natom = max(4, int(round(L ** 3 / 171.0)))
        out.append(SystemSpec(f"batch{k}", L, (n, n, n), 25.0, natom, 2 * natom, 12.0, 1.0, 0.8, -2.0, 5.0, 4.5,
                              1000 * seed + k))
    return out


# Every FFT grid size the library has compile-time kernels for (n3 transforms and plane kernels);
# grid_probe(n) is a cheap system on each: the precision family's spacing, cutoff, wells and
# projectors (L = 28 n / 96 bohr, |G|^2 <= 25), two atoms and four occupied orbitals.
GRID_SIZES = (24, 30, 32, 36, 40, 45, 48, 50, 54, 60, 64, 72, 75, 80, 96)


def grid_probe(n: int, seed: int = 7) -> SystemSpec:
    """Spec of the two-atom system on an n^3 grid (deterministic in ``seed``)."""
    return SystemSpec(f"grid{n}", n * 28.0 / 96.0, (n, n, n), 25.0, 2, 4, 12.0, 1.0, 0.8, -2.0, 5.0, 4.5, seed)


def learned_family(seed: int, n: int = 96) -> SystemSpec:
    """A member of the learned-preconditioner family: the precision system's spacing, cutoff,
    wells and projectors on an n^3 grid (L = 28 n / 96 bohr; the benchmark uses n = 96 and 108),
    at the reduced precision system's density of 8 atoms per (28 bohr)^3 (two occupied orbitals
    per atom)."""
    L = n * 28.0 / 96.0
    natom = max(2, int(round(8 * (n / 96.0) ** 3)))
    return SystemSpec(f"learned{n}_{seed}", L, (n, n, n), 25.0, natom, 2 * natom, 12.0, 1.0, 0.8, -2.0, 5.0, 4.5, seed)


def spec(name: str) -> SystemSpec:
    """The named spec."""
    return SPECS[name]


@dataclasses.dataclass
class System:
    """Arrays of one model system (see the module docstring for the conventions)."""

    spec: SystemSpec
    cell: np.ndarray  # (3, 3) lattice vectors as rows, bohr
    grid: tuple  # (n1, n2, n3)
    atoms: np.ndarray  # (natom, 3) Cartesian positions, bohr
    miller: np.ndarray  # (npw_h, 3) int32, half sphere, G = 0 first
    gvec: np.ndarray  # (npw_h, 3) Cartesian G, bohr^-1
    vloc_r: np.ndarray  # (n3, n2, n1) float64, hartree
    beta: np.ndarray  # (nproj, npw_h) complex128, half-sphere coefficients
    dij: np.ndarray  # (nproj,) float64, hartree
    nocc: int

    @property
    def omega(self) -> float:
        return float(abs(np.linalg.det(self.cell)))

    @property
    def npw_h(self) -> int:
        return int(self.miller.shape[0])

    @property
    def npw(self) -> int:
        return 2 * self.npw_h - 1

    @property
    def nproj(self) -> int:
        return int(self.beta.shape[0])


def half_sphere(L: float, ecut: float) -> np.ndarray:
    """Miller indices of {G : |G|^2 <= ecut} in a cubic cell, Gamma half, canonical order."""
    t = ecut * (L / (2.0 * np.pi)) ** 2
    tmax = int(math.floor(t + 1e-9))
    nmax = int(math.isqrt(tmax))
    r = np.arange(-nmax, nmax + 1)
    n1, n2, n3 = np.meshgrid(r, r, r, indexing="ij")
    n1, n2, n3 = n1.ravel(), n2.ravel(), n3.ravel()
    nn = n1 * n1 + n2 * n2 + n3 * n3
    keep = (nn <= tmax) & ((n3 > 0) | ((n3 == 0) & (n2 > 0)) | ((n3 == 0) & (n2 == 0) & (n1 >= 0)))
    n1, n2, n3, nn = n1[keep], n2[keep], n3[keep], nn[keep]
    order = np.lexsort((n3, n2, n1, nn))
    return np.stack([n1[order], n2[order], n3[order]], axis=1).astype(np.int32)


def _place_atoms(sp: SystemSpec) -> np.ndarray:
    """Uniform positions in [0, L)^3, rejecting any closer than min_dist (minimum image)."""
    pos = []
    k = 0
    block = 3 * 4096
    u = uniform01(sp.seed, block, stream=1)
    while len(pos) < sp.natom:
        if 3 * (k + 1) > u.size:
            u = np.concatenate([u, uniform01(sp.seed, block, stream=1 + u.size // block)])
        cand = u[3 * k: 3 * k + 3] * sp.L
        k += 1
        ok = True
        for p in pos:
            d = cand - p
            d -= sp.L * np.round(d / sp.L)
            if np.sqrt(d @ d) < sp.min_dist:
                ok = False
                break
        if ok:
            pos.append(cand)
        if k > 1_000_000:
            raise RuntimeError("could not place atoms at the requested minimum distance")
    return np.array(pos)


def _vloc(sp: SystemSpec, atoms: np.ndarray) -> np.ndarray:
    n1, n2, n3 = sp.grid
    L = sp.L
    # images T with |component| up to m*L: the Gaussian is below 1e-30 beyond 12 sigma
    m = int(math.ceil((12.0 * sp.sigma + 0.5 * L) / L))
    x1 = np.arange(n1) * (L / n1)
    x2 = np.arange(n2) * (L / n2)
    x3 = np.arange(n3) * (L / n3)
    v = np.zeros((n3, n2, n1))
    inv = 1.0 / (2.0 * sp.sigma ** 2)
    for R in atoms:
        # separable Gaussian: exp(-(dx^2+dy^2+dz^2)/2s^2) = g(dx) g(dy) g(dz)
        def g1(x, c):
            d = x[:, None] - c + L * np.arange(-m, m + 1)[None, :]
            return np.exp(-d * d * inv).sum(axis=1)

        gx, gy, gz = g1(x1, R[0]), g1(x2, R[1]), g1(x3, R[2])
        v -= sp.well_depth * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return v


def _projectors(sp: SystemSpec, gvec: np.ndarray, atoms: np.ndarray):
    g2 = np.einsum("ij,ij->i", gvec, gvec)
    radial = np.exp(-0.5 * g2 * sp.beta_sigma ** 2)
    rows, dij = [], []
    for R in atoms:
        sf = np.exp(-1j * (gvec @ R))
        cols = [radial * sf]
        ds = [sp.d_s]
        if sp.d_p is not None:
            for a in range(3):
                cols.append(-1j * gvec[:, a] * radial * sf)
                ds.append(sp.d_p)
        for c, d in zip(cols, ds):
            # norm over the full sphere: |c(0)|^2 + 2 sum_{G != 0} |c(G)|^2
            nrm2 = abs(c[0]) ** 2 + 2.0 * np.sum(np.abs(c[1:]) ** 2)
            rows.append(c / np.sqrt(nrm2))
            dij.append(d)
    return np.array(rows, dtype=np.complex128), np.array(dij, dtype=np.float64)


def make_system(sp: SystemSpec | str) -> System:
    """Build the arrays of a model system from its spec (deterministic in ``sp.seed``)."""
    if isinstance(sp, str):
        sp = spec(sp)
    miller = half_sphere(sp.L, sp.ecut)
    nmax = int(np.abs(miller).max())
    if min(sp.grid) < 2 * nmax + 1:
        raise ValueError(f"grid {sp.grid} too small for the sphere (|n| <= {nmax})")
    cell = np.eye(3) * sp.L
    bvec = 2.0 * np.pi * np.linalg.inv(cell).T  # rows b_i with a_i . b_j = 2 pi delta_ij
    gvec = miller.astype(np.float64) @ bvec
    atoms = _place_atoms(sp)
    beta, dij = _projectors(sp, gvec, atoms)
    return System(
        spec=sp,
        cell=cell,
        grid=tuple(sp.grid),
        atoms=atoms,
        miller=miller,
        gvec=gvec,
        vloc_r=_vloc(sp, atoms),
        beta=beta,
        dij=dij,
        nocc=sp.nocc,
    )


def _gamma_orthonormal(c: np.ndarray) -> np.ndarray:
    """Orthonormalise rows of half-sphere vectors in <a,b> = a0 b0 + 2 Re sum_{G!=0} conj(a) b.

    Uses the isometry q = [Re c0, sqrt2 Re c_G, sqrt2 Im c_G] to a real vector and a QR
    factorisation there (rows stay in the same span and order, like Gram-Schmidt).
    """
    n, m = c.shape
    q = np.concatenate([c[:, :1].real, np.sqrt(2.0) * c[:, 1:].real, np.sqrt(2.0) * c[:, 1:].imag], axis=1)
    Q, R = np.linalg.qr(q.T)
    Q = Q * np.sign(np.diag(R))[None, :]
    Q = Q.T
    out = np.empty_like(c)
    out[:, 0] = Q[:, 0]
    out[:, 1:] = (Q[:, 1:m] + 1j * Q[:, m:]) / np.sqrt(2.0)
    return out


def make_perturbations(system: System, npert: int, seed: int = 0) -> np.ndarray:
    """``npert`` orthonormal perturbation vectors on the half sphere with a zero G = 0 entry."""
    m = system.npw_h
    z = normal(seed, 2 * npert * (m - 1), stream=7).reshape(npert, 2, m - 1)
    c = np.zeros((npert, m), dtype=np.complex128)
    c[:, 1:] = z[:, 0] + 1j * z[:, 1]
    out = _gamma_orthonormal(c)
    out[:, 0] = 0.0  # exactly zero (the factorisation leaves rounding noise there)
    return out


def make_guess(system: System, nvec: int, seed: int = 0) -> np.ndarray:
    """Random starting block for an iterative eigensolver (orthonormal, G = 0 entry kept)."""
    m = system.npw_h
    z = normal(seed, 2 * nvec * m, stream=11).reshape(nvec, 2, m)
    c = z[:, 0] + 1j * z[:, 1]
    c[:, 0] = z[:, 0, 0]
    return _gamma_orthonormal(c)
