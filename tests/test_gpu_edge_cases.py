"""Edge and degenerate cases of chi0bar through the C ABI.

* Free electrons (V_loc = 0, projector strengths 0, one occupied orbital: the constant function
  with eps = 0): chi0bar is diagonal in plane waves with eigenvalue -32 pi / (Omega |G|^4) at
  G != 0 (the closed form the oracle is pinned to), in every precision form.
* An empty block of perturbations returns at once with no solves; a zero perturbation gives a zero
  response up to the rounding of its Gamma partner (its right-hand sides are zero and its solves
  are skipped); a single perturbation (a Gamma pair with a phantom partner) equals the same
  perturbation applied inside a larger block.
"""

import dataclasses

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

wdf = pytest.importorskip("paper_2607_14025_gb300.wdf")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_14025_gb300 import build

    build.build()
    wdf.load()


@pytest.mark.parametrize("prec,cg_tol,bar", [("fp64", 1e-12, 1e-10), ("mixed", 1e-10, 1e-8), ("mixed_df", 1e-10, 1e-8)])
def test_free_electron_closed_form(prec, cg_tol, bar):
    sp = dataclasses.replace(synth.spec("tiny"), well_depth=0.0, d_s=0.0, nocc=1)
    s = synth.make_system(sp)
    g2 = np.einsum("ij,ij->i", s.gvec, s.gvec)
    lam = np.zeros_like(g2)
    lam[1:] = -32.0 * np.pi / (s.omega * g2[1:] ** 2)
    phi = synth.make_perturbations(s, 3, 0)
    with wdf.Context(s, precision=prec, cg_tol=cg_tol) as c:
        eps, _ = c.orbitals()
        out, _, st = c.apply_chi0(phi)
    assert abs(eps[0]) < 1e-10
    assert st.converged == 1
    ref = lam * phi
    assert np.abs(out - ref).max() <= bar * np.abs(ref).max()


def test_empty_zero_and_single_perturbations():
    s = synth.make_system("small")
    phi = synth.make_perturbations(s, 5, 21)
    with wdf.Context(s, precision="mixed_df", cg_tol=1e-10) as c:
        out0, _, st0 = c.apply_chi0(np.zeros((0, s.npw_h), dtype=np.complex128))
        assert out0.shape == (0, s.npw_h) and st0.nsolve == 0
        block = phi.copy()
        block[2] = 0.0
        out, _, st = c.apply_chi0(block)
        assert st.converged == 1
        # zero up to the rounding of its Gamma partner's transforms (they share complex FFTs)
        assert np.abs(out[2]).max() <= 1e-12 * np.abs(out).max()
        one, _, st1 = c.apply_chi0(phi[4:5])
        assert st1.converged == 1 and st1.nsolve == s.nocc
    assert np.abs(one[0] - out[4]).max() <= 1e-8 * np.abs(out[4]).max()
