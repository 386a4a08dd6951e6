"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test ties one oracle routine to something fixed by mathematics or by an independent
construction: a published generator test vector, brute-force Fourier sums, the explicit matrix of
the Hamiltonian, the sum over empty states (the Adler-Wiser route that DFPT avoids, paper
Sec. 2.1), the free-electron closed form, and the invariants of chi0bar. The planted-mistake
tests at the end show that plausible slips (a dropped factor, a wrong sign, a missing conjugate)
break at least one pin.
"""

import dataclasses

import numpy as np
import pytest

import synth
from oracle import basis, dfpt, dft, hamiltonian, pdep


# ---------------------------------------------------------------------------------------------
# fixtures


@pytest.fixture(scope="module")
def tiny():
    s = synth.make_system("tiny")
    H = hamiltonian.Hamiltonian(s)
    eps_all, psi_all = H.all_states()
    R = dfpt.Response(H, eps_all[: s.nocc], psi_all[: s.nocc])
    return s, H, eps_all, psi_all, R


@pytest.fixture(scope="module")
def small():
    s = synth.make_system("small")
    H = hamiltonian.Hamiltonian(s)
    eps_all, psi_all = H.all_states()
    R = dfpt.Response(H, eps_all[: s.nocc], psi_all[: s.nocc])
    return s, H, eps_all, psi_all, R


def gdot(a, b):
    """Gamma inner product of half-sphere rows: a0 b0 + 2 Re sum_{G != 0} conj(a) b."""
    return np.real(np.conj(a[..., 0]) * b[..., 0]) + 2.0 * np.real(np.sum(np.conj(a[..., 1:]) * b[..., 1:], axis=-1))


# ---------------------------------------------------------------------------------------------
# inputs


def test_splitmix64_published_vectors():
    # first outputs of splitmix64 from state 0 (Vigna's reference implementation)
    z = synth.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_half_sphere_brute_force():
    L, ecut = 10.0, 10.0
    m = synth.half_sphere(L, ecut)
    assert tuple(m[0]) == (0, 0, 0)
    full = basis.full_miller(m)
    # brute force: every integer point with |G|^2 <= ecut appears exactly once in the full set
    pts = set()
    for a in range(-8, 9):
        for b in range(-8, 9):
            for c in range(-8, 9):
                if (2 * np.pi / L) ** 2 * (a * a + b * b + c * c) <= ecut:
                    pts.add((a, b, c))
    assert len(pts) == full.shape[0] == 515
    assert set(map(tuple, full)) == pts
    # no G together with -G in the half set, and the half-space rule
    hs = set(map(tuple, m))
    for a, b, c in m[1:]:
        assert (-a, -b, -c) not in hs
        assert c > 0 or (c == 0 and b > 0) or (c == 0 and b == 0 and a > 0)
    nn = (m.astype(int) ** 2).sum(1)
    assert np.all(np.diff(nn) >= 0)


def test_perturbations_orthonormal(tiny):
    s = tiny[0]
    phi = synth.make_perturbations(s, 8, 0)
    g = gdot(phi[:, None, :], phi[None, :, :])
    assert np.abs(g - np.eye(8)).max() < 1e-13
    assert np.all(phi[:, 0] == 0)


# ---------------------------------------------------------------------------------------------
# basis and transforms


def test_fft_matches_direct_sums():
    grid = (6, 5, 4)  # odd, even and non-cubic sizes
    rng = np.random.default_rng(1)
    half = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [2, -1, 0], [1, 2, 1], [-2, 0, 1], [0, -2, 1]], dtype=np.int32)
    full = basis.full_miller(half)
    c = rng.normal(size=len(full)) + 1j * rng.normal(size=len(full))
    f = basis.ifft_u(basis.to_box(c, full, grid))
    assert np.abs(f - dft.g_to_r(c, full, grid)).max() < 1e-12
    g = rng.normal(size=(4, 5, 6)) + 1j * rng.normal(size=(4, 5, 6))
    assert np.abs(basis.from_box(basis.fft_n(g), full, grid) - dft.r_to_g(g, full, grid)).max() < 1e-13


def test_gamma_pair_identity_and_isometry():
    rng = np.random.default_rng(2)
    m = 17
    a = rng.normal(size=m) + 1j * rng.normal(size=m)
    b = rng.normal(size=m) + 1j * rng.normal(size=m)
    a[0], b[0] = a[0].real, b[0].real
    full = np.real(basis.dot(basis.expand(a), basis.expand(b)))
    assert abs(full - gdot(a, b)) < 1e-12
    q = basis.half_to_real(a)
    assert abs(q @ basis.half_to_real(b) - gdot(a, b)) < 1e-12
    phi = basis.real_isometry(m)
    assert np.abs(phi @ q - basis.expand(a)).max() < 1e-14
    assert np.abs(np.conj(phi.T) @ phi - np.eye(2 * m - 1)).max() < 1e-14
    assert np.abs(basis.real_to_half(q) - a).max() < 1e-14


# ---------------------------------------------------------------------------------------------
# Hamiltonian and ground state


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_hamiltonian_grid_equals_dense(name):
    s = synth.make_system(name)
    H = hamiltonian.Hamiltonian(s)
    hd = H.dense()
    assert np.abs(hd - np.conj(hd.T)).max() < 1e-13
    c = basis.expand(synth.make_guess(s, 3, 5))
    assert np.abs(hd @ c.T - H.apply(c).T).max() < 1e-12
    hr = H.dense_real()
    assert np.abs(hr - hr.T).max() == 0.0


def test_ground_state(tiny):
    s, H, eps_all, psi_all, R = tiny
    c = basis.expand(psi_all[: s.nocc + 2])
    res = H.apply(c) - eps_all[: s.nocc + 2, None] * c
    assert np.abs(res).max() < 1e-11
    ov = np.real(np.conj(c) @ c.T)
    assert np.abs(ov - np.eye(len(c))).max() < 1e-12
    f = basis.ifft_u(basis.to_box(c, H.miller, H.grid))
    assert np.abs(f.imag).max() < 1e-12 * np.abs(f.real).max()
    assert eps_all[s.nocc] - eps_all[s.nocc - 1] > 1e-3  # gap of the seeded tiny system
    w2, _ = H.ground_state(s.nocc)
    assert np.abs(w2 - eps_all[: s.nocc]).max() < 1e-12


# ---------------------------------------------------------------------------------------------
# chi0bar by DFPT against independent routes


@pytest.mark.parametrize("fx", ["tiny", "small"])
def test_dfpt_equals_sum_over_states(fx, request):
    s, H, eps_all, psi_all, R = request.getfixturevalue(fx)
    phi = synth.make_perturbations(s, 4, 1)
    o = R.apply(phi, tol=1e-13)
    assert o["residual"].max() <= 1e-13
    o2 = R.apply(phi, solver=dfpt.sos_solver(R, eps_all, psi_all))
    rel = np.abs(o["out"] - o2["out"]).max() / np.abs(o2["out"]).max()
    assert rel < 1e-11
    rel = np.abs(o["drho"] - o2["drho"]).max() / np.abs(o2["drho"]).max()
    assert rel < 1e-11


def test_dfpt_equals_adler_wiser_matrix(tiny):
    s, H, eps_all, psi_all, R = tiny
    chi = dfpt.adler_wiser_chi0bar(H, eps_all, psi_all, s.nocc)
    phi = synth.make_perturbations(s, 5, 2)
    o = R.apply(phi, tol=1e-13)
    y = (chi @ basis.half_to_real(phi)[:, 1:].T).T
    yr = basis.half_to_real(o["out"])[:, 1:]
    assert np.abs(y - yr).max() / np.abs(y).max() < 1e-11
    w = np.linalg.eigvalsh(chi)
    assert w.max() <= 1e-12  # negative semidefinite
    assert np.abs(chi - chi.T).max() < 1e-12


def test_free_electron_closed_form():
    sp = dataclasses.replace(synth.spec("tiny"), well_depth=0.0, d_s=0.0, nocc=1)
    s = synth.make_system(sp)
    H = hamiltonian.Hamiltonian(s)
    w, psi = H.ground_state(2)
    assert abs(w[0]) < 1e-14 and abs(w[1] - 0.5 * (2 * np.pi / s.spec.L) ** 2) < 1e-12
    R = dfpt.Response(H, w[:1], psi[:1])
    phi = synth.make_perturbations(s, 3, 0)
    o = R.apply(phi, tol=1e-14)
    g2 = H.g2[: s.npw_h]
    lam = np.zeros_like(g2)
    lam[1:] = -32.0 * np.pi / (s.omega * g2[1:] ** 2)
    assert np.abs(o["out"] - lam * phi).max() / np.abs(lam * phi).max() < 1e-12


def test_symmetry_linearity_neutrality(small):
    s, H, eps_all, psi_all, R = small
    phi = synth.make_perturbations(s, 4, 3)
    o = R.apply(phi, tol=1e-13)["out"]
    # <a, chi b> = <chi a, b>
    g = gdot(phi[:, None, :], o[None, :, :])
    assert np.abs(g - g.T).max() < 1e-11 * np.abs(g).max()
    # negative semidefinite compression
    assert np.linalg.eigvalsh(0.5 * (g + g.T)).max() < 0
    # linearity
    comb = 0.7 * phi[0] - 1.3 * phi[1]
    oc = R.apply(comb[None], tol=1e-13)["out"][0]
    assert np.abs(oc - (0.7 * o[0] - 1.3 * o[1])).max() < 1e-11 * np.abs(oc).max()
    # the response density integrates to zero (charge conservation)
    d = R.apply(phi[:1], tol=1e-13)["drho"]
    assert abs(d[0, 0]) < 1e-13 * np.abs(d).max()


def test_invariant_under_orbital_signs_and_order(small):
    s, H, eps_all, psi_all, R = small
    phi = synth.make_perturbations(s, 2, 4)
    o = R.apply(phi, tol=1e-13)["out"]
    perm = np.arange(s.nocc)[::-1]
    sign = np.where(np.arange(s.nocc) % 2 == 0, -1.0, 1.0)
    R2 = dfpt.Response(H, eps_all[: s.nocc][perm], sign[:, None] * psi_all[: s.nocc][perm])
    o2 = R2.apply(phi, tol=1e-13)["out"]
    assert np.abs(o - o2).max() < 1e-11 * np.abs(o).max()


def test_result_independent_of_preconditioner(tiny):
    s, H, eps_all, psi_all, R = tiny
    phi = synth.make_perturbations(s, 2, 5)
    a = R.apply(phi, tol=1e-13, precondition=True)
    b = R.apply(phi, tol=1e-13, precondition=False)
    assert np.abs(a["out"] - b["out"]).max() < 1e-11 * np.abs(a["out"]).max()
    assert a["iters"].mean() < b["iters"].mean()


def test_tpa_limits():
    x = np.array([0.0, 1e-3, 1e5])
    k = dfpt.tpa(x)
    assert k[0] == 1.0 and abs(k[1] - 1.0) < 1e-3
    assert abs(k[2] * 2 * x[2] - 1.0) < 2e-5  # K = (1 + 1/x + ...) / (2x)


def test_tpa_interior_values_by_hand():
    # Teter, Payne and Allan's polynomial P = 27 + 18x + 12x^2 + 8x^3 evaluated by hand:
    # x = 1/2: P = 27 + 9 + 3 + 1 = 40, 16 x^4 = 1   -> K = 40/41
    # x = 1:   P = 27 + 18 + 12 + 8 = 65, 16 x^4 = 16 -> K = 65/81
    # x = 2:   P = 27 + 36 + 48 + 64 = 175, 16 x^4 = 256 -> K = 175/431
    # (each coefficient enters at a different weight, so a wrong one fails at least one value)
    k = dfpt.tpa(np.array([0.5, 1.0, 2.0]))
    assert np.abs(k - np.array([40 / 41, 65 / 81, 175 / 431])).max() < 1e-15


# ---------------------------------------------------------------------------------------------
# PDEP


def test_davidson_equals_dense_eigenvalues(tiny):
    s, H, eps_all, psi_all, R = tiny
    chi = dfpt.adler_wiser_chi0bar(H, eps_all, psi_all, s.nocc)
    neig = 6
    res = pdep.davidson(lambda x: R.apply(x, tol=1e-13)["out"], synth.make_perturbations(s, neig, 3), neig, maxiter=60, tol=1e-10)
    ref = pdep.dense_eigs(chi, neig)
    assert np.abs(res["lam"] - ref).max() < 1e-10 * np.abs(ref).max()
    assert np.all(np.diff(res["lam"]) >= 0)
    # eigenvectors: orthonormal and true eigenvectors of the explicit matrix
    q = basis.half_to_real(res["vec"])[:, 1:]
    assert np.abs(q @ q.T - np.eye(neig)).max() < 1e-10
    assert np.abs(chi @ q.T - q.T * res["lam"][None, :]).max() < 1e-8


# ---------------------------------------------------------------------------------------------
# planted mistakes: each must be caught by a pin above


def test_planted_density_factor_is_caught(monkeypatch, tiny):
    s, H, eps_all, psi_all, R = tiny
    phi = synth.make_perturbations(s, 2, 1)
    ref = R.apply(phi, solver=dfpt.sos_solver(R, eps_all, psi_all))["out"]
    chi = dfpt.adler_wiser_chi0bar(H, eps_all, psi_all, s.nocc)
    good = (chi @ basis.half_to_real(phi)[:, 1:].T).T
    assert np.abs(basis.half_to_real(ref)[:, 1:] - good).max() < 1e-10 * np.abs(good).max()
    orig = dfpt.Response.density

    def half_density(self, d, vidx, npert, pidx):
        return 0.5 * orig(self, d, vidx, npert, pidx)  # spin factor dropped

    monkeypatch.setattr(dfpt.Response, "density", half_density)
    bad = R.apply(phi, solver=dfpt.sos_solver(R, eps_all, psi_all))["out"]
    assert np.abs(basis.half_to_real(bad)[:, 1:] - good).max() > 1e-3 * np.abs(good).max()


def test_planted_rhs_sign_is_caught(monkeypatch, tiny):
    s, H, eps_all, psi_all, R = tiny
    phi = synth.make_perturbations(s, 3, 1)
    orig = dfpt.Response.rhs
    monkeypatch.setattr(dfpt.Response, "rhs", lambda self, x, v: -orig(self, x, v))
    o = R.apply(phi, tol=1e-12)["out"]
    g = gdot(phi[:, None, :], o[None, :, :])
    # a flipped Sternheimer right-hand side makes chi0bar positive: the NSD pin fails
    assert np.linalg.eigvalsh(0.5 * (g + g.T)).max() > 0


def test_planted_missing_conjugate_is_caught(monkeypatch):
    # a projection without the conjugate breaks the Hermiticity / dense-vs-grid pin
    s = synth.make_system("tiny")
    H = hamiltonian.Hamiltonian(s)
    hd = H.dense()
    c = basis.expand(synth.make_guess(s, 2, 5))
    monkeypatch.setattr(
        hamiltonian.Hamiltonian,
        "nonlocal_",
        lambda self, c: ((self.beta.T @ (self.dij[:, None] * (self.beta @ np.atleast_2d(c).T))).T).reshape(np.shape(c)),
    )
    assert np.abs(hd @ c.T - H.apply(c).T).max() > 1e-6


def test_medium_system_has_the_required_gap():
    # the medium workload needs a HOMO-LUMO gap of at least 0.1 hartree; the oracle's iterative
    # eigensolver (about a minute on 8 cores) finds 0.473 hartree for the seeded system
    s = synth.make_system("medium")
    assert (s.npw, s.npw_h, s.nproj) == (16879, 8440, 128)
    H = hamiltonian.Hamiltonian(s)
    w, _ = H.ground_state(s.nocc + 1, tol=1e-8)
    assert w[s.nocc] - w[s.nocc - 1] > 0.1


def test_lowrank_chibar_with_every_eigenpair_is_the_rpa_inverse(tiny):
    # Eq. (5) without Xi: with all eigenpairs of chi0bar the low-rank sum is exact, and RPA
    # (chi = chi0 + chi0 chi) fixes it as (1 - chi0)^-1 chi0
    s, H, eps_all, psi_all, R = tiny
    chi0 = dfpt.adler_wiser_chi0bar(H, eps_all, psi_all, s.nocc)
    w, V = np.linalg.eigh(chi0)
    full = pdep.chibar_lowrank(w, V.T)
    rpa = np.linalg.solve(np.eye(len(w)) - chi0, chi0)
    assert np.abs(full - rpa).max() <= 1e-12 * np.abs(rpa).max()
    # W_p = v^1/2 chi v^1/2 through the half-sphere interface, against the matrix (G != 0 block)
    m = s.npw_h
    vh = R.vhalf[:m]
    x = synth.make_perturbations(s, 3, 4)
    phib = basis.real_to_half(np.concatenate([np.zeros((len(w), 1)), V.T], axis=1))
    got = basis.half_to_real(pdep.wp_apply(w, phib, vh, x))[:, 1:]
    vreal = np.concatenate([vh[1:], vh[1:]])  # real coordinates: sqrt(2) Re c_G, then sqrt(2) Im c_G
    want = ((vreal[:, None] * rpa * vreal[None, :]) @ basis.half_to_real(x)[:, 1:].T).T
    assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max()


def test_planted_wrong_screening_factor_is_caught(monkeypatch, tiny):
    s, H, eps_all, psi_all, R = tiny
    chi0 = dfpt.adler_wiser_chi0bar(H, eps_all, psi_all, s.nocc)
    w, V = np.linalg.eigh(chi0)
    rpa = np.linalg.solve(np.eye(len(w)) - chi0, chi0)
    bad = (V * w[None, :]) @ V.T  # lambda instead of lambda / (1 - lambda): chi0 itself
    assert np.abs(bad - rpa).max() > 1e-2 * np.abs(rpa).max()
