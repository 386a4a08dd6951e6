"""GPU tests of the learned Sternheimer preconditioner (through the C ABI).

The library's forward/backward kernels are checked against the FP64 oracle MLP (loss and
gradient), its Adam kernel against the oracle's update with the same gradient, and its training
samples (features, targets, weights from converged solves) against the oracle's construction on
the same system and perturbations. Then a model trained on seeded systems must lower the CG
iteration count on held-out systems without changing chi0bar, a deliberately bad model must be
rescued by the TPA fallback, and the first-iterate option must reach the same result.

Tolerances: the kernels run the network in FP32 with FP64 sums, so outputs carry ~1e-6 relative
error and the gradient is held to 1e-4 of its largest entry; Adam is applied in FP64 and compared
after rounding to FP32 (1e-6 relative).
"""

import dataclasses

import numpy as np
import pytest

import synth
from oracle import basis, dfpt, hamiltonian, mlp

pytestmark = pytest.mark.gpu

wdf = pytest.importorskip("paper_2607_14025_gb300.wdf")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_14025_gb300 import build

    build.build()
    wdf.load()


def model_weights(seed, wscale=0.5):
    flat = wscale * synth.normal(seed, mlp.NMODEL, stream=3)
    flat[mlp.NPARAM:mlp.NPARAM + mlp.NIN] = synth.normal(seed, mlp.NIN, stream=4)
    flat[mlp.NPARAM + mlp.NIN:] = 0.5 + synth.uniform01(seed, mlp.NIN, stream=5)
    return flat.astype(np.float32)


def samples(seed, n):
    F = (2.0 * synth.normal(seed, n * 4, stream=6)).reshape(n, 4).astype(np.float32)
    T = synth.normal(seed, n * 2, stream=7).reshape(n, 2).astype(np.float32)
    W = synth.uniform01(seed, n * 2, stream=8).reshape(n, 2).astype(np.float32)
    return F, T, W


@pytest.mark.parametrize("n", [1, 1000, 152 * 128 * 2 + 77])
def test_loss_and_gradient_match_oracle(n):
    w = model_weights(1)
    F, T, W = samples(2, n)
    m = wdf.Model(seed=0)
    m.weights = w
    m.set_samples(F, T, W)
    assert m.num_samples == n
    f2, t2, w2 = m.samples()
    assert np.array_equal(f2, F) and np.array_equal(t2, T) and np.array_equal(w2, W)
    L, g = m.loss_grad()
    Lr, gr = mlp.loss_grad(w.astype(np.float64), F.astype(np.float64), T.astype(np.float64), W.astype(np.float64))
    assert abs(L - Lr) <= 1e-5 * abs(Lr)
    assert np.abs(g - gr).max() <= 1e-4 * np.abs(gr).max()
    out = m.predict(F[:257])
    ref = mlp.forward(w.astype(np.float64), F[:257].astype(np.float64))[3]
    assert np.abs(out - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


def test_adam_steps_match_oracle():
    w = model_weights(3)
    F, T, W = samples(4, 3000)
    m = wdf.Model(seed=0)
    m.weights = w
    m.set_samples(F, T, W)
    flat = w.astype(np.float64)
    mom = np.zeros(mlp.NPARAM)
    var = np.zeros(mlp.NPARAM)
    for t in (1, 2):
        _, g = m.loss_grad()  # the library's gradient at its current weights
        m.train(steps=1, lr=1e-3)
        flat, mom, var = mlp.adam_step(flat, g, mom, var, t, 1e-3)
        got = m.weights.astype(np.float64)
        assert np.abs(got - flat).max() <= 1e-6 * np.abs(flat).max()
        flat = got  # continue from the FP32-rounded weights, as the library does for its kernels


def test_training_samples_match_oracle():
    s = synth.make_system("small")
    H = hamiltonian.Hamiltonian(s)
    w, psi = H.ground_state(s.nocc)
    R = dfpt.Response(H, w, psi)
    npert = 4
    phi = synth.make_perturbations(s, npert, 21)
    # oracle: TPA solves, per-(v, G) sums on the full sphere, then the half sphere with counts
    x = R.vhalf_times(phi)
    pidx = np.repeat(np.arange(npert), s.nocc)
    vidx = np.tile(np.arange(s.nocc), npert)
    b = R.rhs(x[pidx], vidx)
    d, _, _ = R.sternheimer(b, vidx, tol=1e-13)
    ex, ek, ck = mlp.solve_sums(b, d, R.tpa_rows(vidx), vidx, s.nocc)
    m_h = len(s.miller)
    mult = np.r_[1.0, np.full(m_h - 1, 2.0)]
    T, Wt = mlp.targets(ex[:, :m_h], ek[:, :m_h], ck[:, :m_h], mult)
    F = mlp.features(H.g2[:m_h], R.tkin, R.eps, R.psi[:, :m_h], m_h).reshape(-1, 4)
    # library: the same orbitals, FP64 solves to 1e-12
    with wdf.Context(s, psi=psi, eps=w, precision="fp64", cg_tol=1e-12) as c:
        m = wdf.Model(seed=0)
        st = m.add_solves(c, phi)
        assert st.converged == 1 and st.nsolve == npert * s.nocc
    f, t, wt = m.samples()
    assert f.shape == (s.nocc * m_h, 4)
    assert np.abs(f - F).max() <= 1e-5 * np.abs(F).max()
    assert np.isclose(wt[:, 0].sum(), 1.0, rtol=1e-5) and np.isclose(wt[:, 1].sum(), 1.0, rtol=1e-5)
    assert np.abs(wt - Wt).sum() <= 1e-5
    # targets: weighted deviations (entries of negligible weight carry the solves' rounding)
    assert np.sqrt(np.sum(Wt[:, 0] * (t[:, 0] - T[:, 0]) ** 2)) <= 1e-5
    assert np.sqrt(np.sum(Wt[:, 1] * (t[:, 1] - T[:, 1]) ** 2)) <= 1e-5 * np.sqrt(np.sum(Wt[:, 1] * T[:, 1] ** 2))


def _family(seed):
    return synth.make_system(dataclasses.replace(synth.spec("small"), seed=seed))


def test_trained_model_lowers_iterations_on_held_out_systems():
    train = [wdf.Context(_family(k), precision="mixed_df", cg_tol=1e-10) for k in range(4)]
    model, ts = wdf.train_preconditioner(train, npert=8, steps=800, lr=3e-3, seed=5)
    assert ts.nsamples == sum(c.nocc * c.npw_h for c in train)
    assert ts.loss_last < 0.3 * ts.loss_first
    for c in train:
        c.close()
    it_tpa, it_ml = 0.0, 0.0
    for k in (32, 33):
        s = _family(k)
        phi = synth.make_perturbations(s, 8, 100 + k)
        with wdf.Context(s, precision="mixed_df", cg_tol=1e-10) as c:
            out0, dr0, st0 = c.apply_chi0(phi, want_drho=True)
            c.set_model(model)
            out1, dr1, st1 = c.apply_chi0(phi, want_drho=True)
        assert st1.converged == 1 and st1.max_residual <= 1e-10
        # the preconditioner changes the path, not chi0bar
        assert np.abs(dr1 - dr0).max() <= 1e-8 * np.abs(dr0).max()
        assert np.abs(out1 - out0).max() <= 1e-8 * np.abs(out0).max()
        it_tpa += st0.cg_iters / st0.nsolve
        it_ml += st1.cg_iters / st1.nsolve
    assert it_ml < 0.95 * it_tpa


def test_bad_model_falls_back_to_tpa():
    s = _family(7)
    phi = synth.make_perturbations(s, 4, 3)
    # a model whose scale jumps between e^-8 and e^8 with |c_v(G)|^2: CG stalls, then reverts
    wf = np.zeros(mlp.NMODEL)
    o = 0
    for name, shape in mlp.SHAPES:
        n = int(np.prod(shape))
        if name == "W1":
            blk = np.zeros(shape)
            blk[3, 0] = 40.0  # h1_0 = tanh(40 f3), a sign of the orbital weight at G
            blk[0, 1] = 40.0
            wf[o:o + n] = blk.reshape(-1)
        if name == "W2":
            blk = np.zeros(shape)
            blk[0, 0] = 3.0
            blk[1, 0] = -3.0
            wf[o:o + n] = blk.reshape(-1)
        if name == "W3":
            blk = np.zeros(shape)
            blk[0, 0] = 8.0
            wf[o:o + n] = blk.reshape(-1)
        o += n
    wf[mlp.NPARAM + mlp.NIN:] = 1.0  # mu 0, sd 1
    # the scale is 1 where N_h |c_v(G)|^2 > 1 and e^-8 elsewhere (G != 0)
    F = mlp.features(np.array([0.0, 1.0, 1.0]), np.array([1.0]), np.array([-1.0]), np.array([[0.0, 1.0, 1e-3]]), 4)[0]
    assert np.allclose(mlp.scale(wf, F)[1:], [1.0, np.exp(-8.0 * np.tanh(6.0))], rtol=1e-3)
    with wdf.Context(s, precision="mixed_df", cg_tol=1e-10) as c:
        out0, _, st0 = c.apply_chi0(phi)
        m = wdf.Model(seed=0)
        m.weights = wf.astype(np.float32)
        c.set_model(m)
        out1, _, st1 = c.apply_chi0(phi)
    assert st1.converged == 1
    assert st1.fallbacks > 0
    assert np.abs(out1 - out0).max() <= 1e-8 * np.abs(out0).max()


def test_first_iterate_option_reaches_the_same_result():
    train = [wdf.Context(_family(k), precision="mixed_df", cg_tol=1e-10) for k in range(2)]
    model, _ = wdf.train_preconditioner(train, npert=4, steps=300, seed=9)
    for c in train:
        c.close()
    s = _family(40)
    phi = synth.make_perturbations(s, 4, 5)
    with wdf.Context(s, precision="mixed_df", cg_tol=1e-10) as c:
        out0, _, _ = c.apply_chi0(phi)
    with wdf.Context(s, precision="mixed_df", cg_tol=1e-10, warm_start=True) as c:
        c.set_model(model)
        out1, _, st1 = c.apply_chi0(phi)
    assert st1.converged == 1
    assert np.abs(out1 - out0).max() <= 1e-8 * np.abs(out0).max()


def test_model_on_fp64_context_and_back_to_tpa():
    s = _family(41)
    phi = synth.make_perturbations(s, 2, 6)
    m = wdf.Model(seed=3)
    with wdf.Context(s, precision="fp64", cg_tol=1e-11) as c:
        out0, _, st0 = c.apply_chi0(phi)
        m.add_solves(c, phi)
        m.train(steps=50)
        c.set_model(m)
        out1, _, st1 = c.apply_chi0(phi)
        c.set_model(None)
        out2, _, st2 = c.apply_chi0(phi)
    assert np.abs(out1 - out0).max() <= 1e-9 * np.abs(out0).max()
    assert np.array_equal(out2, out0) and st2.cg_iters == st0.cg_iters  # TPA path is deterministic


def test_learned_family_96_held_out_gain():
    # the learned form's own family (96^3 grid, 23,149 stored plane waves, the precision system's
    # cell and cutoff at a reduced atom count): train on 6 seeds, test on 2 held-out seeds
    train = [wdf.Context(synth.make_system(synth.learned_family(k, 96)), precision="mixed_df", cg_tol=1e-8) for k in range(6)]
    model, ts = wdf.train_preconditioner(train, npert=8, steps=800, lr=3e-3, seed=11)
    for c in train:
        c.close()
    assert ts.loss_last < 0.5 * ts.loss_first
    it_tpa, it_ml = 0.0, 0.0
    for k in (32, 33):
        s = synth.make_system(synth.learned_family(k, 96))
        phi = synth.make_perturbations(s, 8, 700 + k)
        with wdf.Context(s, precision="mixed_df", cg_tol=1e-10) as c:
            out0, _, st0 = c.apply_chi0(phi)
            c.set_model(model)
            out1, _, st1 = c.apply_chi0(phi)
        assert st1.converged == 1 and st1.max_residual <= 1e-10
        assert np.abs(out1 - out0).max() <= 1e-8 * np.abs(out0).max()
        it_tpa += st0.cg_iters / st0.nsolve
        it_ml += st1.cg_iters / st1.nsolve
    assert it_ml < 0.95 * it_tpa
