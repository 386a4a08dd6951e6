"""FP64 CPU oracle for the DFPT screening hot path. TEST INFRASTRUCTURE ONLY.

This package is the slow, plain reference against which the GPU library is checked. Only the
test suite, the smoke check and the CPU-baseline leg of the benchmark may import it; the library
never does, and the oracle never imports the library. The two share nothing but the seeded
inputs of the ``synth`` module.

What it computes (paper: "The WEST code for large-scale excited-state materials simulations",
Sec. 2.1): the symmetrised independent-particle response chi0bar = v^1/2 chi0 v^1/2 applied to
perturbations by density-functional perturbation theory, i.e. one Sternheimer solve per occupied
orbital and perturbation with no empty states, and the projective eigendecomposition (PDEP) of
chi0bar whose eigenpairs enter the low-rank form of Eq. (5).

Every routine works on the FULL plane-wave sphere with plain complex arithmetic (no Gamma-point
pairing trick); the half-sphere storage of the interface is expanded on entry and folded on exit.
Library primitives serve as steps: numpy/scipy FFTs, dense LAPACK eigensolvers, matrix products.

Modules:
  basis        plane-wave sphere, grid transforms, inner products, real-basis isometry
  dft          brute-force discrete Fourier sums (pins the FFT convention)
  hamiltonian  H = -1/2 nabla^2 + V_loc + sum beta D beta^dagger, grid and dense forms, ground state
  dfpt         Sternheimer PCG, chi0bar application, sum-over-states and Adler-Wiser forms
  pdep         block Davidson for the lowest eigenpairs of chi0bar; dense reference

Pins (tests marked "not gpu"): direct DFT, dense-vs-grid Hamiltonian, sum over states,
Adler-Wiser matrix, the free-electron closed form lambda_G = -32 pi / (Omega |G|^4),
symmetry, negative semidefiniteness, charge neutrality of the response, invariance under
occupied-orbital rotations, Davidson vs dense eigenvalues. No function is parity unpinned.
"""

from . import basis, dft, hamiltonian, dfpt, pdep  # noqa: F401
