"""Learned Sternheimer preconditioner: features, targets and the MLP (oracle; test infrastructure).

The paper has no learned preconditioner (it motivates machine-learning datasets built from the
code's outputs in its outlook). This module defines, in plain FP64 numpy, the model that the
library implements, so that the library's forward, backward and Adam kernels and its
training-sample construction can be checked against it:

* One sample per occupied orbital v and plane wave G. Features
      f0 = log(1 + x),  x = (1/2 |G|^2) / T_v     (the Teter-Payne-Allan variable)
      f1 = eps_v,   f2 = T_v,   f3 = log(N_h |c_v(G)|^2 + 1e-6)
  with T_v the (floored) kinetic energy of psi_v and N_h the number of half-sphere plane waves.
  The network sees (f - mu) / sd.
* Targets, from converged solves A_v d = b of the Sternheimer equation, summed over the solves
  that share the orbital v (K the TPA preconditioner of v):
      E_x(v,G) = sum |d(G)|^2,  E_k(v,G) = sum |K b(G)|^2,  C(v,G) = sum Re(conj(K b(G)) d(G))
      t0 = 1/2 log(E_x / E_k)   the log of the diagonal scale s = exp(o0): M = s K maps the
                                spectrum of K b onto that of the solution
      t1 = C / E_k              the least-squares gain of a first iterate d0 = o1 K b
  weighted by w0 = E_x + E_k and w1 = E_k, each normalised to unit sum over one system.
* Network 4 -> 64 -> 64 -> 2, tanh hidden layers, linear output:
      h1 = tanh(X W1 + b1), h2 = tanh(h1 W2 + b2), o = h2 W3 + b3.
  Loss = sum_i sum_k w_ik (o_ik - t_ik)^2 (full batch).
* Adam (Kingma and Ba, "Adam: a method for stochastic optimization", ICLR 2015, Algorithm 1):
      m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
      theta <- theta - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Flat parameter layout (shared with the library's interface): W1[4][64], b1[64], W2[64][64],
b2[64], W3[64][2], b3[2] (4610 trained values), then mu[4], sd[4] (8 fixed values).

Pins (tests marked "not gpu"): the gradient against central finite differences of the loss, the
zero-network closed form, the first Adam step (each parameter moves by lr sign(g)), the
targets of a diagonal operator (t0 = -log(a K), t1 = 1/(a K)), and a trained model that
lowers the CG iteration count on held-out systems.
"""

from __future__ import annotations

import numpy as np

NIN, NH, NOUT = 4, 64, 2
SHAPES = [("W1", (NIN, NH)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH, NOUT)), ("b3", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)  # 4610
NMODEL = NPARAM + 2 * NIN  # + mu, sd
S_CLAMP = 8.0  # |o0| is clamped before exp so the scale stays in [e^-8, e^8]


def unpack(flat: np.ndarray) -> dict:
    """Split a flat model vector (NMODEL values) into named arrays (views)."""
    flat = np.asarray(flat, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = flat[o:o + n].reshape(shape)
        o += n
    out["mu"] = flat[o:o + NIN]
    out["sd"] = flat[o + NIN:o + 2 * NIN]
    return out


def features(g2: np.ndarray, tkin: np.ndarray, eps: np.ndarray, psi: np.ndarray, nh: int) -> np.ndarray:
    """Raw features (nocc, nG, 4) for |G|^2 (nG), T_v and eps_v (nocc) and coefficients c_v(G)."""
    nocc, ng = psi.shape
    F = np.empty((nocc, ng, NIN))
    F[:, :, 0] = np.log1p(0.5 * g2[None, :] / tkin[:, None])
    F[:, :, 1] = eps[:, None]
    F[:, :, 2] = tkin[:, None]
    F[:, :, 3] = np.log(nh * np.abs(psi) ** 2 + 1e-6)
    return F


def solve_sums(b: np.ndarray, d: np.ndarray, K: np.ndarray, vidx: np.ndarray, nocc: int):
    """E_x, E_k, C per (v, G) from solves (rows of b, d; K the preconditioner rows of each solve)."""
    Kb = K * b
    ex = np.zeros((nocc, b.shape[1]))
    ek = np.zeros_like(ex)
    ck = np.zeros_like(ex)
    for v in range(nocc):
        rows = vidx == v
        ex[v] = np.sum(np.abs(d[rows]) ** 2, axis=0)
        ek[v] = np.sum(np.abs(Kb[rows]) ** 2, axis=0)
        ck[v] = np.sum(np.real(np.conj(Kb[rows]) * d[rows]), axis=0)
    return ex, ek, ck


def targets(ex: np.ndarray, ek: np.ndarray, ck: np.ndarray, mult: np.ndarray | None = None):
    """Targets (n, 2) and weights (n, 2) from the per-(v, G) sums (flattened v-major).

    ``mult`` (per G) counts how many plane waves a stored coefficient stands for (the half-sphere
    storage keeps one of G, -G); weights are normalised to unit sum per output. Entries with
    E_k = 0 get zero weight and zero targets.
    """
    ex, ek, ck = (np.asarray(a, dtype=np.float64) for a in (ex, ek, ck))
    m = np.ones(ex.shape[-1]) if mult is None else np.asarray(mult, dtype=np.float64)
    ok = ek > 0
    t0 = np.where(ok, 0.5 * (np.log(np.where(ok, ex, 1.0) + 1e-300) - np.log(np.where(ok, ek, 1.0))), 0.0)
    t1 = np.where(ok, ck / np.where(ok, ek, 1.0), 0.0)
    w0 = np.where(ok, (ex + ek) * m[None, :], 0.0)
    w1 = np.where(ok, ek * m[None, :], 0.0)
    w0 = w0 / max(w0.sum(), 1e-300)
    w1 = w1 / max(w1.sum(), 1e-300)
    T = np.stack([t0.reshape(-1), t1.reshape(-1)], 1)
    W = np.stack([w0.reshape(-1), w1.reshape(-1)], 1)
    return T, W


def normalisation(F: np.ndarray, mult: np.ndarray | None = None):
    """Weighted mean and standard deviation of each feature (weights = multiplicities)."""
    F = F.reshape(-1, NIN)
    m = np.ones(F.shape[0]) if mult is None else np.asarray(mult, dtype=np.float64).reshape(-1)
    mu = np.sum(m[:, None] * F, axis=0) / m.sum()
    var = np.sum(m[:, None] * (F - mu) ** 2, axis=0) / m.sum()
    sd = np.sqrt(var)
    sd = np.where(sd > 1e-6, sd, 1.0)  # a constant feature is passed through centred
    return mu, sd


def forward(flat: np.ndarray, F: np.ndarray):
    """Hidden activations and outputs for raw features F (n, 4)."""
    P = unpack(flat)
    X = (np.asarray(F, dtype=np.float64) - P["mu"]) / P["sd"]
    h1 = np.tanh(X @ P["W1"] + P["b1"])
    h2 = np.tanh(h1 @ P["W2"] + P["b2"])
    return X, h1, h2, h2 @ P["W3"] + P["b3"]


def loss(flat: np.ndarray, F: np.ndarray, T: np.ndarray, W: np.ndarray) -> float:
    """sum_i sum_k W_ik (o_ik - T_ik)^2."""
    o = forward(flat, F)[3]
    return float(np.sum(W * (o - T) ** 2))


def loss_grad(flat: np.ndarray, F: np.ndarray, T: np.ndarray, W: np.ndarray):
    """Loss and its gradient with respect to the NPARAM trained values (chain rule, layer by layer)."""
    P = unpack(flat)
    X, h1, h2, o = forward(flat, F)
    e = 2.0 * W * (o - T)  # dL/do
    gW3 = h2.T @ e
    gb3 = e.sum(0)
    d2 = (e @ P["W3"].T) * (1.0 - h2 ** 2)  # dL/d(pre-activation of layer 2)
    gW2 = h1.T @ d2
    gb2 = d2.sum(0)
    d1 = (d2 @ P["W2"].T) * (1.0 - h1 ** 2)
    gW1 = X.T @ d1
    gb1 = d1.sum(0)
    g = np.concatenate([a.reshape(-1) for a in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return float(np.sum(W * (o - T) ** 2)), g


def adam_step(flat: np.ndarray, g: np.ndarray, m: np.ndarray, v: np.ndarray, t: int, lr: float,
              b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update of the NPARAM trained values (t counts from 1). Returns new arrays."""
    flat = np.array(flat, dtype=np.float64)
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    flat[:NPARAM] -= lr * mh / (np.sqrt(vh) + eps)
    return flat, m, v


def train(flat: np.ndarray, F: np.ndarray, T: np.ndarray, W: np.ndarray, steps: int, lr: float):
    """Full-batch Adam for ``steps`` steps; returns the model and the loss before each step."""
    m = np.zeros(NPARAM)
    v = np.zeros(NPARAM)
    hist = []
    for t in range(1, steps + 1):
        L, g = loss_grad(flat, F, T, W)
        hist.append(L)
        flat, m, v = adam_step(flat, g, m, v, t, lr)
    return flat, hist


def scale(flat: np.ndarray, F: np.ndarray) -> np.ndarray:
    """Diagonal scale s = exp(clamp(o0)) of the learned preconditioner M = s K."""
    o = forward(flat, F)[3]
    return np.exp(np.clip(o[:, 0], -S_CLAMP, S_CLAMP))
