"""GPU checks of the smaller entry points: the context's G vectors, error reset on a healthy
context, and PDEP from a library-drawn start block against the dense eigenvalues of the explicit
chi0bar of the tiny system (1e-8 relative, the plain-FP64 bar)."""

import numpy as np
import pytest

import synth
from oracle import dfpt, hamiltonian, pdep

pytestmark = pytest.mark.gpu

wdf = pytest.importorskip("paper_2607_14025_gb300.wdf")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_14025_gb300 import build

    build.build()


def test_gvectors_and_reset_error():
    s = synth.make_system("small")
    with wdf.Context(s, precision="fp64") as c:
        assert np.array_equal(c.gvectors(), s.miller)
        c.reset_error()  # nothing to clear: WDF_OK
        assert np.array_equal(wdf.half_sphere(s.cell, s.spec.ecut), s.miller)


def test_pdep_from_a_seeded_start_matches_dense_eigenvalues():
    s = synth.make_system("tiny")
    H = hamiltonian.Hamiltonian(s)
    wa, pa = H.all_states()
    chi = dfpt.adler_wiser_chi0bar(H, wa, pa, s.nocc)
    neig = 6
    ref = pdep.dense_eigs(chi, neig)
    with wdf.Context(s, precision="fp64", cg_tol=1e-12, gs_tol=1e-11) as c:
        lam, vec, st = c.pdep_seeded(neig, seed=7, maxiter=80, tol=1e-9)
    assert st.converged == 1
    assert np.abs(lam - ref).max() <= 1e-8 * np.abs(ref).max()


def test_low_rank_wp_matches_oracle():
    # eigenpairs from the oracle's explicit chi0bar feed both sides (no input from the GPU path)
    from oracle import basis

    s = synth.make_system("tiny")
    H = hamiltonian.Hamiltonian(s)
    wa, pa = H.all_states()
    R = dfpt.Response(H, wa[: s.nocc], pa[: s.nocc])
    chi = dfpt.adler_wiser_chi0bar(H, wa, pa, s.nocc)
    w, V = np.linalg.eigh(chi)
    neig = 10
    lam = w[:neig]
    phib = basis.real_to_half(np.concatenate([np.zeros((neig, 1)), V[:, :neig].T], axis=1))
    x = synth.make_perturbations(s, 5, 12)
    ref = pdep.wp_apply(lam, phib, R.vhalf[: s.npw_h], x)
    with wdf.Context(s, precision="fp64") as c:
        got = c.apply_wp(lam, phib, x)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
