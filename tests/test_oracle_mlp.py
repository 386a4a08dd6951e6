"""Pins of the learned-preconditioner oracle (features, targets, MLP, Adam).

The paper defines no learned preconditioner, so these pins come from mathematics alone: central
finite differences of the loss, closed forms of a zero network and of the first Adam steps, and
the targets of a diagonal operator, for which the solution of A d = b is known exactly. The
last pin trains the model on a few seeded systems and checks that it lowers the CG iteration
count on a held-out system without changing the solution.
"""

import dataclasses

import numpy as np
import pytest

import synth
from oracle import basis, dfpt, hamiltonian, mlp


def random_model(seed, wscale=0.5):
    flat = wscale * synth.normal(seed, mlp.NMODEL, stream=3)
    flat[mlp.NPARAM:mlp.NPARAM + mlp.NIN] = synth.normal(seed, mlp.NIN, stream=4)
    flat[mlp.NPARAM + mlp.NIN:] = 0.5 + synth.uniform01(seed, mlp.NIN, stream=5)
    return flat


def random_samples(seed, n):
    F = 2.0 * synth.normal(seed, n * mlp.NIN, stream=6).reshape(n, mlp.NIN)
    T = synth.normal(seed, n * 2, stream=7).reshape(n, 2)
    W = synth.uniform01(seed, n * 2, stream=8).reshape(n, 2)
    return F, T, W


def fd_gradient(flat, F, T, W, h=1e-5):
    g = np.zeros(mlp.NPARAM)
    for j in range(mlp.NPARAM):
        fp = flat.copy()
        fm = flat.copy()
        fp[j] += h
        fm[j] -= h
        g[j] = (mlp.loss(fp, F, T, W) - mlp.loss(fm, F, T, W)) / (2 * h)
    return g


def test_gradient_matches_central_differences():
    flat = random_model(1)
    F, T, W = random_samples(2, 40)
    L, g = mlp.loss_grad(flat, F, T, W)
    assert abs(L - mlp.loss(flat, F, T, W)) <= 1e-14 * abs(L)
    gfd = fd_gradient(flat, F, T, W)
    # central differences: truncation ~h^2 |f'''|, rounding ~eps |L| / h
    assert np.abs(g - gfd).max() <= 1e-7 * np.abs(g).max()
    # every block of parameters takes part
    o = 0
    for name, shape in mlp.SHAPES:
        n = int(np.prod(shape))
        assert np.abs(g[o:o + n]).max() > 0, name
        o += n


def test_zero_network_closed_form():
    flat = np.zeros(mlp.NMODEL)
    flat[mlp.NPARAM + mlp.NIN:] = 1.0  # sd
    b3 = np.array([0.3, -1.2])
    flat[mlp.NPARAM - 2:mlp.NPARAM] = b3
    F, T, W = random_samples(3, 25)
    L, g = mlp.loss_grad(flat, F, T, W)
    assert np.isclose(L, np.sum(W * (b3[None, :] - T) ** 2), rtol=1e-14)
    # hidden activations are tanh(0) = 0: only the output bias has a gradient
    assert np.allclose(g[-2:], 2.0 * np.sum(W * (b3[None, :] - T), axis=0), rtol=1e-13)
    assert np.abs(g[:-2]).max() == 0.0
    o = mlp.forward(flat, F)[3]
    assert np.allclose(o, b3[None, :])
    assert np.allclose(mlp.scale(flat, F), np.exp(b3[0]))


def test_first_adam_steps_closed_form():
    flat = random_model(4)
    g1 = synth.normal(5, mlp.NPARAM, stream=1)
    g2 = synth.normal(6, mlp.NPARAM, stream=1)
    lr = 1e-3
    m = np.zeros(mlp.NPARAM)
    v = np.zeros(mlp.NPARAM)
    f1, m, v = mlp.adam_step(flat, g1, m, v, 1, lr)
    # step 1: bias-corrected moments are g and g^2, so every parameter moves by lr g / (|g| + eps)
    assert np.allclose(f1[:mlp.NPARAM] - flat[:mlp.NPARAM], -lr * g1 / (np.abs(g1) + 1e-8), rtol=1e-12, atol=0)
    assert np.array_equal(f1[mlp.NPARAM:], flat[mlp.NPARAM:])  # mu, sd are not trained
    f2, m, v = mlp.adam_step(f1, g2, m, v, 2, lr)
    mh = (0.9 * 0.1 * g1 + 0.1 * g2) / (1 - 0.9 ** 2)
    vh = (0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2) / (1 - 0.999 ** 2)
    assert np.allclose(f2[:mlp.NPARAM] - f1[:mlp.NPARAM], -lr * mh / (np.sqrt(vh) + 1e-8), rtol=1e-10, atol=1e-18)


def test_targets_of_a_diagonal_operator():
    # A = diag(a): the solution is d = b / a exactly, whatever b is, so t0 = -log(a K), t1 = 1/(a K)
    nocc, ng, nsol = 3, 17, 12
    a = 0.5 + synth.uniform01(7, ng, stream=1)
    K = 0.1 + synth.uniform01(8, nocc * ng, stream=1).reshape(nocc, ng)
    vidx = np.arange(nsol) % nocc
    b = (synth.normal(9, nsol * ng, stream=1) + 1j * synth.normal(9, nsol * ng, stream=2)).reshape(nsol, ng)
    d = b / a[None, :]
    ex, ek, ck = mlp.solve_sums(b, d, K[vidx], vidx, nocc)
    T, W = mlp.targets(ex, ek, ck)
    ref0 = -np.log(a[None, :] * K).reshape(-1)
    ref1 = (1.0 / (a[None, :] * K)).reshape(-1)
    assert np.allclose(T[:, 0], ref0, rtol=1e-13, atol=1e-13)
    assert np.allclose(T[:, 1], ref1, rtol=1e-13)
    assert np.isclose(W[:, 0].sum(), 1.0) and np.isclose(W[:, 1].sum(), 1.0)
    assert (W >= 0).all()


def test_features_by_hand():
    g2 = np.array([0.0, 2.0, 8.0])
    tkin = np.array([0.5, 2.0])
    eps = np.array([-1.5, -0.25])
    psi = np.array([[1.0, 0.5j, 0.0], [0.0, 0.25, -0.5]])
    F = mlp.features(g2, tkin, eps, psi, nh=4)
    # f0 = log(1 + g2 / (2 T)): T = 0.5 -> log(1 + g2); T = 2 -> log(1 + g2 / 4)
    assert np.allclose(F[0, :, 0], np.log([1.0, 3.0, 9.0]))
    assert np.allclose(F[1, :, 0], np.log([1.0, 1.5, 3.0]))
    assert np.allclose(F[:, :, 1], [[-1.5] * 3, [-0.25] * 3])
    assert np.allclose(F[:, :, 2], [[0.5] * 3, [2.0] * 3])
    assert np.allclose(F[0, :, 3], np.log([4.0 + 1e-6, 1.0 + 1e-6, 1e-6]))
    assert np.allclose(F[1, :, 3], np.log([1e-6, 0.25 + 1e-6, 1.0 + 1e-6]))


def test_normalisation_weighted():
    F = np.array([[1.0, 0, 0, 0], [3.0, 0, 0, 0]])
    mu, sd = mlp.normalisation(F, np.array([1.0, 3.0]))
    assert np.isclose(mu[0], 2.5) and np.isclose(sd[0], np.sqrt(0.75))
    assert np.allclose(sd[1:], 1.0)  # constant features pass through


def collect(seed, npert=8):
    sp = dataclasses.replace(synth.spec("small"), seed=seed)
    s = synth.make_system(sp)
    H = hamiltonian.Hamiltonian(s)
    eps, psi = H.ground_state(s.nocc)
    R = dfpt.Response(H, eps, psi)
    phi = synth.make_perturbations(s, npert, seed + 100)
    x = R.vhalf_times(phi)
    pidx = np.repeat(np.arange(npert), s.nocc)
    vidx = np.tile(np.arange(s.nocc), npert)
    b = R.rhs(x[pidx], vidx)
    d, it, _ = R.sternheimer(b, vidx, tol=1e-8)
    ex, ek, ck = mlp.solve_sums(b, d, R.tpa_rows(vidx), vidx, s.nocc)
    F = mlp.features(H.g2, R.tkin, R.eps, R.psi, len(s.miller))
    return dict(R=R, b=b, vidx=vidx, it=it, d=d, F=F, sums=(ex, ek, ck), nocc=s.nocc)


def test_trained_model_lowers_iterations_on_held_out_system():
    train = [collect(k) for k in range(4)]
    held = collect(32)
    F = np.concatenate([t["F"].reshape(-1, mlp.NIN) for t in train])
    Ts, Ws = zip(*[mlp.targets(*t["sums"]) for t in train])
    T = np.concatenate(Ts)
    W = np.concatenate(Ws) / len(train)
    flat = random_model(11, wscale=0.0)
    flat[: mlp.NPARAM] = 0.3 * synth.normal(12, mlp.NPARAM, stream=1)
    mu, sd = mlp.normalisation(F)
    flat[mlp.NPARAM:mlp.NPARAM + mlp.NIN] = mu
    flat[mlp.NPARAM + mlp.NIN:] = sd
    flat, hist = mlp.train(flat, F, T, W, steps=1200, lr=3e-3)
    assert hist[-1] < 0.2 * hist[0]
    R, b, vidx = held["R"], held["b"], held["vidx"]
    s = mlp.scale(flat, held["F"].reshape(-1, mlp.NIN)).reshape(held["nocc"], -1)
    M = s[vidx] * R.tpa_rows(vidx)
    d, it, res = R.sternheimer(b, vidx, tol=1e-8, precondition=M)
    assert res.max() <= 1e-8
    assert it.mean() < 0.95 * held["it"].mean()
    # the preconditioner changes the path, not the solution
    assert np.abs(d - held["d"]).max() <= 1e-6 * np.abs(held["d"]).max()


def test_planted_missing_tanh_derivative_is_caught(monkeypatch):
    orig = mlp.loss_grad

    def bad(flat, F, T, W):
        P = mlp.unpack(flat)
        X, h1, h2, o = mlp.forward(flat, F)
        e = 2.0 * W * (o - T)
        d2 = e @ P["W3"].T  # (1 - h2^2) dropped
        d1 = (d2 @ P["W2"].T) * (1.0 - h1 ** 2)
        g = np.concatenate([a.reshape(-1) for a in (X.T @ d1, d1.sum(0), h1.T @ d2, d2.sum(0), h2.T @ e, e.sum(0))])
        return float(np.sum(W * (o - T) ** 2)), g

    flat = random_model(1)
    F, T, W = random_samples(2, 40)
    gfd = fd_gradient(flat, F, T, W)
    assert np.abs(orig(flat, F, T, W)[1] - gfd).max() <= 1e-7 * np.abs(gfd).max()
    assert np.abs(bad(flat, F, T, W)[1] - gfd).max() > 1e-3 * np.abs(gfd).max()
