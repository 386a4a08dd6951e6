"""The library's block Davidson on a caller's operator (wdf_davidson).

The paper's Sec. 3.3 has one Davidson solver serve PDEP and the BSE and TDDFT eigenproblems; here
the engine that runs PDEP takes any operator the caller applies through a callback.
* A diagonal operator in plane waves, A c(G) = d(G) c(G) with d = |G|^2 plus a seeded split of
  each shell by up to 0.01: its spectrum is known in closed form (d(0) once, every other d(G)
  twice: the cosine and the sine of the real functions), with and without the G = 0 component.
* chi0bar itself, applied by a second context through the callback: the eigenvalues must equal
  those of wdf_pdep_davidson on the same start block.
"""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

wdf = pytest.importorskip("paper_2607_14025_gb300.wdf")


@pytest.fixture(scope="module")
def tiny():
    from paper_2607_14025_gb300 import build

    build.build()
    return synth.make_system("tiny")


# neig covers whole degenerate pairs: the first shell (3 half-sphere waves, 6 real functions),
# plus G = 0 when it is in the space
@pytest.mark.parametrize("zero_g0,neig", [(True, 6), (False, 7)])
def test_diagonal_operator_spectrum(tiny, zero_g0, neig):
    import torch

    s = tiny
    g2 = np.einsum("ij,ij->i", s.gvec, s.gvec)
    d = g2 + 0.01 * synth.uniform01(1234, s.npw_h)  # shells split by less than their spacing
    d[0] = 0.2  # G = 0: the lowest when it is in the space
    dt = torch.from_numpy(d).to(torch.complex128).cuda()
    calls = []

    def apply(x, out):
        calls.append(x.shape[0])
        out.copy_(dt[None, :] * x)

    guess = synth.make_guess(s, neig + 3, 9)
    with wdf.Context(s, precision="mixed", cg_tol=1e-10) as c:
        try:
            lam, vec, st = c.davidson(apply, neig, guess, maxiter=400, tol=1e-9, zero_g0=zero_g0)
        except wdf.NotConverged as e:
            pytest.fail(f"not converged: {e.result[2].as_dict()}")
    assert st.converged == 1 and sum(calls) == st.napply
    spec = np.sort(np.concatenate([d[1:], d[1:]] + ([] if zero_g0 else [d[:1]])))
    assert np.abs(lam - spec[:neig]).max() < 1e-12
    # eigenvector residuals with the operator applied on the host
    r = d[None, :] * vec - lam[:, None] * vec
    assert np.abs(r).max() < 1e-8
    if zero_g0:
        assert np.abs(vec[:, 0]).max() == 0.0


def test_chi0_through_callback_matches_pdep(tiny):
    import torch

    s = tiny
    neig = 4
    guess = synth.make_perturbations(s, neig + 2, 3)
    with wdf.Context(s, precision="mixed", cg_tol=1e-11) as op, wdf.Context(s, precision="mixed", cg_tol=1e-11) as c:
        def apply(x, out):
            y, _, _ = op.apply_chi0(x)
            out.copy_(y)

        lam_cb, vec_cb, st_cb = c.davidson(apply, neig, guess, maxiter=60, tol=1e-9, zero_g0=True)
        lam_pd, vec_pd, st_pd = c.pdep(neig, guess, maxiter=60, tol=1e-9)
    assert st_cb.converged == 1 and st_pd.converged == 1
    assert np.abs(lam_cb - lam_pd).max() <= 1e-9 * np.abs(lam_pd).max()
    assert torch.cuda.is_available()
