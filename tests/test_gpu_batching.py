"""Batching form through the C ABI: several systems of uneven size in one wdf_apply_chi0_multi
call give exactly what wdf_apply_chi0 gives for each of them (same contexts, so the same kernels
and reduction orders: bit for bit), and the smallest system of the family matches the FP64
oracle at the mixed form's bar (1e-8 relative at cg_tol 1e-10)."""

import numpy as np
import pytest

import synth
from oracle import dfpt, hamiltonian

pytestmark = pytest.mark.gpu

wdf = pytest.importorskip("paper_2607_14025_gb300.wdf")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_14025_gb300 import build

    build.build()


def test_multi_equals_single_applies():
    specs = synth.batch_family(4, seed=0)  # grids 32, 36, 40, 45; 10 to 26 orbitals
    systems = [synth.make_system(sp) for sp in specs]
    ctxs = [wdf.Context(s, precision="mixed_df", cg_tol=1e-10) for s in systems]
    phis = [synth.make_perturbations(s, 6 + k, 40 + k) for k, s in enumerate(systems)]
    try:
        single = [c.apply_chi0(p) for c, p in zip(ctxs, phis)]
        outs, stats = wdf.apply_chi0_multi(ctxs, phis)
    finally:
        for c in ctxs:
            c.close()
    for k, (o, st) in enumerate(zip(outs, stats)):
        assert np.array_equal(o, single[k][0]), k
        assert st.nsolve == single[k][2].nsolve == phis[k].shape[0] * systems[k].nocc
        assert st.cg_iters == single[k][2].cg_iters
        assert st.converged == 1


def test_smallest_batch_system_matches_oracle():
    s = synth.make_system(synth.batch_family(1, seed=0)[0])
    H = hamiltonian.Hamiltonian(s)
    w, psi = H.ground_state(s.nocc)
    R = dfpt.Response(H, w, psi)
    phi = synth.make_perturbations(s, 4, 3)
    ref = R.apply(phi, tol=1e-13)
    c2 = wdf.Context(synth.make_system(synth.batch_family(1, seed=0)[0]), psi=psi, eps=w, precision="mixed_df",
                     cg_tol=1e-10)
    other = wdf.Context(synth.make_system(synth.batch_family(2, seed=0)[1]), precision="mixed_df", cg_tol=1e-10)
    try:
        outs, stats = wdf.apply_chi0_multi([c2, other], [phi, synth.make_perturbations(other, 3, 1)])
    finally:
        c2.close()
        other.close()
    assert np.abs(outs[0] - ref["out"]).max() <= 1e-8 * np.abs(ref["out"]).max()


@pytest.mark.parametrize("index", [1, 3])  # grids 36 (radices 4 3 3) and 45 (5 3 3)
def test_batch_system_on_further_compile_time_sizes_matches_oracle(index, monkeypatch):
    # the compile-time Stockham plane kernels and n3 transforms of the further sizes (float inner
    # iterations, double-float residuals) against the FP64 oracle, each side with its own ground state
    spec = synth.batch_family(index + 1, seed=0)[index]
    s = synth.make_system(spec)
    assert s.grid[0] in (36, 45)
    H = hamiltonian.Hamiltonian(s)
    w, psi = H.ground_state(s.nocc)
    R = dfpt.Response(H, w, psi)
    phi = synth.make_perturbations(s, 3, 7)
    ref = R.apply(phi, tol=1e-13)
    monkeypatch.setenv("WDF_PLANE_VARIANT", "2")  # the compile-time Stockham kernels, whatever the timing
    with wdf.Context(s, precision="mixed_df", cg_tol=1e-10) as c:
        assert c.plane_variant(32) == 2 and c.plane_variant(48) == 2
        out, drho, st = c.apply_chi0(phi, want_drho=True)
    assert st.converged == 1 and st.max_residual <= 1e-10
    assert np.abs(drho - ref["drho"]).max() <= 1e-8 * np.abs(ref["drho"]).max()
    assert np.abs(out - ref["out"]).max() <= 1e-8 * np.abs(ref["out"]).max()


def test_multi_rejects_a_repeated_context():
    s = synth.make_system("tiny")
    with wdf.Context(s) as c:
        phi = synth.make_perturbations(s, 2, 1)
        with pytest.raises(wdf.WdfError) as e:
            wdf.apply_chi0_multi([c, c], [phi, phi])
    assert e.value.code == wdf.WDF_EINVAL


def test_contexts_of_different_grids_coexist():
    # kernel shared-memory limits are per function: a smaller grid set up later must not lower
    # them below what the larger context's launches need
    big = synth.make_system("medium")
    small = synth.make_system("tiny")
    phi = synth.make_perturbations(big, 2, 8)
    with wdf.Context(big, precision="mixed_df", cg_tol=1e-8) as cb:
        ref, _, _ = cb.apply_chi0(phi)
        with wdf.Context(small, precision="mixed_df", cg_tol=1e-8) as cs:
            cs.apply_chi0(synth.make_perturbations(small, 2, 8))
            out, _, st = cb.apply_chi0(phi)
    assert st.converged == 1
    assert np.array_equal(out, ref)
