"""Iterative refinement of the FP32 inner forms: the solutions returned meet the tolerance when
their residual is recomputed from scratch (Sec. 2.1).

With wdf_options.residual_update set, after the first refinement the library may take the residual
of x + d as r - A d with A d in FP32 and an error bound eps_A ||d|| (eps_A measured on the batch)
added to the stopping test. Here, in that mode and in the default one, the
returned x is put through the residual operator in the residuals' precision
(wdf_apply_sternheimer_operator: double-float or FP64), b - A x is formed in FP64, and every solve
must satisfy ||b - A x|| <= cg_tol ||b||, within the reported max_residual, on the small, medium and
reduced-precision (96^3) systems with right-hand sides -Q fft(dV psi_v) from the oracle. The trace
shows which refinements took the update; at cg_tol 1e-8 (the metric's) every case must take it,
at 1e-10 the bound may send the last refinement to the full residual. The default mode (every
refinement recomputes the residual) and the update mode agree on the solutions to what the
tolerance allows.
"""

import numpy as np
import pytest

import synth
from oracle import basis, dfpt, hamiltonian

pytestmark = pytest.mark.gpu

wdf = pytest.importorskip("paper_2607_14025_gb300.wdf")

@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_14025_gb300 import build

    build.build()
    wdf.load()


_cache = {}


def problem(name, npert):
    key = (name, npert)
    if key not in _cache:
        s = synth.make_system(name)
        with wdf.Context(s, precision="fp64") as c:
            eps, psi = c.orbitals()
        R = dfpt.Response(hamiltonian.Hamiltonian(s), eps, psi)
        phi = synth.make_perturbations(s, npert, 3)
        vidx = np.tile(np.arange(s.nocc), npert).astype(np.int32)
        pidx = np.repeat(np.arange(npert), s.nocc)
        b = basis.fold(R.rhs(basis.expand(phi)[pidx], vidx))
        _cache[key] = (s, eps, psi, vidx, b)
    return _cache[key]


def rel_res(b, Ax):
    r = basis.expand(b - Ax)
    bf = basis.expand(b)
    return np.linalg.norm(r, axis=1) / np.linalg.norm(bf, axis=1)


@pytest.mark.parametrize("update", [True, False])
@pytest.mark.parametrize(
    "name,npert,prec,tol",
    [("small", 4, "mixed_df", 1e-8), ("medium", 2, "mixed_df", 1e-8), ("medium", 2, "mixed", 1e-10),
     ("precision_reduced", 1, "mixed_df", 1e-8)],
)
def test_refined_solutions_meet_tolerance(name, npert, prec, tol, update, capfd, monkeypatch):
    s, eps, psi, vidx, b = problem(name, npert)
    monkeypatch.setenv("WDF_TRACE", "1")
    with wdf.Context(s, psi=psi, eps=eps, precision=prec, cg_tol=tol, residual_update=update) as c:
        x, st = c.sternheimer(vidx, b)
        Ax = c.apply_sternheimer_operator(vidx, x)
    res = rel_res(b, Ax)
    trace = capfd.readouterr().err
    print(f"{name} {prec} {tol}: true max {res.max():.3e}, reported {st.max_residual:.3e}")
    print("\n".join(l for l in trace.splitlines() if "residual (eps_A" in l))
    assert res.max() <= tol
    assert res.max() <= st.max_residual * (1 + 1e-6) + 1e-14
    if update and tol >= 1e-8:  # at the benchmark's tolerance the correction is small enough
        assert "updated residual" in trace
    if not update:
        assert "updated residual" not in trace


def test_update_and_full_residuals_agree():
    s, eps, psi, vidx, b = problem("medium", 2)
    xs = []
    with wdf.Context(s, psi=psi, eps=eps, precision="mixed_df", cg_tol=1e-8) as c:
        for on in (True, False):
            c.set_residual_update(on)
            x, st = c.sternheimer(vidx, b)
            xs.append(x)
    xa, xb = xs
    # both meet 1e-8 in the residual; the solutions agree to the error that allows (kappa x tol)
    assert np.abs(xa - xb).max() <= 1e-5 * np.abs(xb).max()
