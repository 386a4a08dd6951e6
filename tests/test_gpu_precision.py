"""Precision form on the large configuration (L = 28 bohr, 96^3 grid, 23,149 stored plane waves,
128 atoms, 512 projectors, 256 occupied orbitals) through the C ABI.

The FP64 oracle would need hours here, so the per-result errors of the reduced-precision forms
are measured against the plain FP64 GPU form (itself held to the oracle at 1e-8 on the tiny,
small and ragged systems), on the same orbitals and perturbations, and the FP64 result is checked
for properties of chi0bar that hold at any size: symmetry and negative semidefiniteness of
<phi_a, chi0bar phi_b>, and a density response without G = 0 component.
Bar: 1e-8 relative (largest deviation over the largest magnitude) at cg_tol 1e-10, the same as
the mixed forms' parity bar against the oracle.
"""

import numpy as np
import pytest

import synth
from oracle import basis

pytestmark = pytest.mark.gpu

wdf = pytest.importorskip("paper_2607_14025_gb300.wdf")


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


@pytest.fixture(scope="module")
def state():
    from paper_2607_14025_gb300 import build

    build.build()
    s = synth.make_system("precision")
    with wdf.Context(s, precision="fp64", cg_tol=1e-10) as c:
        eps, psi = c.orbitals()
    return s, eps, psi


def test_precision_system_forms_agree_and_chi0_properties(state):
    s, eps, psi = state
    assert psi.shape == (256, 23149)
    phi = synth.make_perturbations(s, 4, 31)
    res = {}
    for prec in ("fp64", "mixed_df", "mixed"):
        with wdf.Context(s, psi=psi, eps=eps, precision=prec, cg_tol=1e-10) as c:
            out, drho, st = c.apply_chi0(phi, want_drho=True)
        assert st.converged == 1 and st.max_residual <= 1e-10, prec
        assert st.nsolve == 4 * 256
        res[prec] = (out, drho)
    out64, drho64 = res["fp64"]
    for prec in ("mixed_df", "mixed"):
        assert rel(res[prec][1], drho64) <= 1e-8, prec
        assert rel(res[prec][0], out64) <= 1e-8, prec
    # chi0bar properties on the FP64 result
    q = basis.half_to_real(phi)
    m = q @ basis.half_to_real(out64).T
    scale = np.abs(m).max()
    assert np.abs(m - m.T).max() <= 1e-9 * scale
    assert np.linalg.eigvalsh(0.5 * (m + m.T)).max() <= 1e-9 * scale
    # drho(G = 0) = (4 / Omega) sum_v <psi_v | dpsi_v>: zero up to the solves' tolerance
    assert np.abs(drho64[:, 0]).max() <= 1e-10 * np.abs(drho64).max()
