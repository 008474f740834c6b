"""Pins of the learned indicator's oracle (oracle/mlp_oracle.py) against
things fixed outside it: central finite differences of its own loss (the
back-propagation), the closed form of Adam's first steps (Kingma & Ba,
Algorithm 1, with bias correction), hand-built feature patches, and the
plain scheme's weights on data where the paper fixes them (Sec. 2.2 Step 3:
linear data give tau = 0, so omega = gamma; a jump drives omega_0 far from
gamma_0), which the labels are made from."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp_oracle as M
from paper_2607_24325_b300 import workloads as W

BLOCKS = ("W1", "b1", "W2", "b2", "w3", "b3")


def _kink_free_batch(seed, B=24, margin=2e-3):
    """A seeded batch and parameters with no pre-activation within `margin`
    of the ReLU kink, so central differences of step <= 1e-6 never cross it."""
    rng = np.random.default_rng(seed)
    theta = M.init_params(seed)
    theta[M.NH * M.NIN:M.NH * M.NIN + M.NH] = rng.normal(0, 0.3, M.NH)              # b1
    o = M.NH * M.NIN + M.NH + M.NH * M.NH
    theta[o:o + M.NH] = rng.normal(0, 0.3, M.NH)                                      # b2
    theta[-1] = 0.2                                                                   # b3
    X, y = [], []
    while len(X) < B:
        x = rng.normal(0, 1, M.NIN)
        _, (a1, _, a2, _, _) = M.forward(theta, x[None, :])
        if np.abs(a1).min() > margin and np.abs(a2).min() > margin:
            X.append(x)
            y.append(float(rng.uniform() < 0.3))
    return theta, np.array(X), np.array(y)


def _blocks(v):
    return dict(zip(BLOCKS, M.unpack(v)))


@pytest.mark.parametrize("seed,pos_weight", [(1, 1.0), (2, 7.5)])
def test_loss_grad_matches_central_differences(seed, pos_weight):
    theta, X, y = _kink_free_batch(seed)
    loss, g = M.loss_and_grad(theta, X, y, pos_weight)
    h = 1e-6
    rng = np.random.default_rng(100 + seed)
    fd = np.zeros_like(theta)
    # every parameter of the small blocks, a seeded sample of the big ones
    sizes = [M.NH * M.NIN, M.NH, M.NH * M.NH, M.NH, M.NH, 1]
    starts = np.cumsum([0] + sizes[:-1])
    checked = np.zeros(theta.size, dtype=bool)
    for s0, n in zip(starts, sizes):
        idx = np.arange(s0, s0 + n) if n <= 64 else s0 + rng.choice(n, 96, replace=False)
        for k in idx:
            tp, tm = theta.copy(), theta.copy()
            tp[k] += h
            tm[k] -= h
            fd[k] = (M.loss_and_grad(tp, X, y, pos_weight)[0] - M.loss_and_grad(tm, X, y, pos_weight)[0]) / (2 * h)
            checked[k] = True
    for name, s0, n in zip(BLOCKS, starts, sizes):
        sl = slice(s0, s0 + n)
        c = checked[sl]
        gv, fv = g[sl][c], fd[sl][c]
        rel = np.linalg.norm(gv - fv) / (np.linalg.norm(fv) + 1e-300)
        assert np.linalg.norm(fv) > 0, name
        assert rel <= 1e-6, (name, rel)
    # the loss itself at zero weights: p = sigmoid(b3) everywhere
    z = np.zeros_like(theta)
    z[-1] = 0.4
    l0, _ = M.loss_and_grad(z, X, y, pos_weight)
    p = 1.0 / (1.0 + math.exp(-0.4))
    wt = np.where(y > 0.5, pos_weight, 1.0)
    expect = -np.mean(wt * (y * math.log(p) + (1 - y) * math.log(1 - p)))
    assert abs(l0 - expect) <= 1e-14 * expect


def test_loss_grad_output_layer_closed_form():
    """With W1 = W2 = 0 the hidden activations are ReLU(b1) and ReLU(W2 h1 + b2)
    = ReLU(b2): dL/db3 = mean(wt (p - y)) and dL/dw3 = h2 * dL/db3."""
    theta = np.zeros(M.NPARAM)
    W1, b1, W2, b2, w3, b3 = M.unpack(theta)
    b2v = np.linspace(-1, 1, M.NH)
    w3v = np.linspace(0.5, -0.5, M.NH)
    theta = M.pack(W1, b1, W2, b2v, w3v, np.array([0.1]))
    X = np.random.default_rng(0).normal(size=(5, M.NIN))
    y = np.array([1.0, 0.0, 0.0, 1.0, 0.0])
    h2 = np.maximum(b2v, 0.0)
    z = float(h2 @ w3v + 0.1)
    p = 1.0 / (1.0 + math.exp(-z))
    wt = np.where(y > 0.5, 3.0, 1.0)
    gb3 = float(np.mean(wt * (p - y)))
    _, g = M.loss_and_grad(theta, X, y, 3.0)
    G = _blocks(g)
    assert abs(G["b3"][0] - gb3) <= 1e-15
    assert np.allclose(G["w3"], h2 * gb3, rtol=0, atol=1e-15)
    assert np.allclose(G["b2"], np.where(b2v > 0, w3v * gb3, 0.0), rtol=0, atol=1e-15)
    assert np.all(G["W1"] == 0) and np.all(G["b1"] == 0)  # ReLU(0) has zero slope here


def test_adam_first_step_closed_form():
    """At t = 1 the bias-corrected moments are g and g^2, so the update is
    theta - lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0, 7.0])
    theta = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    lr, eps = 0.01, 1e-8
    t1, m1, v1 = M.adam_step(theta, np.zeros(5), np.zeros(5), g, 1, lr, eps=eps)
    assert np.allclose(t1, theta - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g, rtol=1e-14, atol=0)      # (1 - beta1) g, rounded
    assert np.allclose(v1, 0.001 * g * g, rtol=1e-12, atol=0)  # (1 - beta2) g^2


def test_adam_second_step_hand_computed():
    """Two steps with g1 = 0.5, g2 = -0.2, lr = 0.1, beta = (0.9, 0.999),
    worked by hand:
      m1 = 0.05, v1 = 2.5e-4, theta1 = 1 - 0.1 * 0.5 / (0.5 + 1e-8)
      m2 = 0.045 - 0.02 = 0.025, v2 = 2.4975e-4 + 4e-5 = 2.8975e-4
      mhat2 = 0.025 / 0.19, vhat2 = 2.8975e-4 / 0.001999
      theta2 = theta1 - 0.1 * mhat2 / (sqrt(vhat2) + 1e-8)"""
    th = np.array([1.0])
    th1, m1, v1 = M.adam_step(th, np.zeros(1), np.zeros(1), np.array([0.5]), 1, 0.1)
    rel = 1e-14  # the hand values are exact decimals; the code rounds them
    assert abs(m1[0] - 0.05) < rel * 0.05 and abs(v1[0] - 2.5e-4) < rel * 2.5e-4
    theta1 = 1.0 - 0.1 * 0.5 / (0.5 + 1e-8)
    assert abs(th1[0] - theta1) < 1e-15
    th2, m2, v2 = M.adam_step(th1, m1, v1, np.array([-0.2]), 2, 0.1)
    assert abs(m2[0] - 0.025) < rel * 0.025
    assert abs(v2[0] - 2.8975e-4) < rel * 2.8975e-4
    theta2 = theta1 - 0.1 * (0.025 / 0.19) / (math.sqrt(2.8975e-4 / 0.001999) + 1e-8)
    assert abs(th2[0] - theta2) < 1e-14
    assert abs(th2[0] - (theta1 - 0.0345606)) < 1e-6  # 0.1 * 0.131579 / 0.380719


def test_features_hand_built_patch():
    """One 2D Euler cell (nx = ny = 1) whose padded 5x5 density patch is
    10*dy + dx: range 44, centre 22, so s = 1/(44 + 1e-3*22); the x- and
    y-moment patches are constants 2 and -3; other planes must not enter."""
    nc = 4
    P = np.full((12, 5, 5), 99.0)
    dy, dx = np.mgrid[0:5, 0:5]
    P[0] = 10.0 * dy + dx
    P[nc] = 2.0
    P[2 * nc] = -3.0
    f = M.features_from_padded(P, nc)
    assert f.shape == (1, 75)
    s = 1.0 / (44.0 + 0.022)
    assert abs(f[0, 0] - (0 - 22) * s) < 1e-15          # (dy, dx) = (0, 0)
    assert abs(f[0, 1] - (1 - 22) * s) < 1e-15          # dx fastest
    assert abs(f[0, 5] - (10 - 22) * s) < 1e-15         # next row
    assert f[0, 12] == 0.0                              # the centre
    assert abs(f[0, 24] - (44 - 22) * s) < 1e-15
    assert np.allclose(f[0, 25:50], 2.0 * s, rtol=1e-15, atol=0)
    assert np.allclose(f[0, 50:75], -3.0 * s, rtol=1e-15, atol=0)
    # a flat patch: only the kappa term scales (s = 1 / (1e-3 * 4))
    P[0] = 4.0
    f = M.features_from_padded(P, nc)
    assert np.all(f[0, :25] == 0.0)
    assert np.allclose(f[0, 25:50], 2.0 * 250.0, rtol=1e-12, atol=0)


def test_features_2x2_grid_uses_each_cells_own_patch():
    """Two cells side by side: the second cell's patch is the first's shifted
    by one column (so its first feature is the first cell's second)."""
    nc = 1
    P = np.zeros((3, 5, 6))
    P[0] = np.arange(30, dtype=float).reshape(5, 6) ** 1.5
    P[1] = 1.0
    P[2] = 0.0
    f = M.features_from_padded(P, nc)
    assert f.shape == (2, 75)
    for i in range(2):
        pr = P[0][:, i:i + 5]
        c = pr[2, 2]
        s = 1.0 / (pr.max() - pr.min() + 1e-3 * abs(c) + 1e-30)
        assert np.allclose(f[i, :25], ((pr - c) * s).ravel(), rtol=1e-14, atol=1e-15)


def test_weight_deviation_labels_special_cases():
    """The label source: linear data give omega = gamma (deviation at
    round-off), a jump gives a deviation near 1 beside it."""
    W2D = (0.99, 0.0025, 0.0025, 0.0025, 0.0025)
    N = 12
    p = oracle.Problem(dim=2, equation=oracle.EQ_BURGERS, nx=N, ny=N, lin_w=W2D, bc=(oracle.BC_OUTFLOW,) * 4)
    xc = (np.arange(N) + 0.5) / N
    U = np.zeros((3, N, N))
    U[0] = 0.3 + 2.0 * xc[None, :] - 1.0 * xc[:, None]
    U[1] = 2.0 / N          # scaled x-moment of a linear function: its slope times dx
    U[2] = -1.0 / N
    d = oracle.weight_deviation(p, U)
    assert d[2:-2, 2:-2].max() < 1e-6
    U2 = np.zeros((3, N, N))
    U2[0] = np.where(xc[None, :] < 0.5, 1.0, 0.0) + 0.0 * xc[:, None]
    d2 = oracle.weight_deviation(p, U2)
    assert d2[:, N // 2 - 1:N // 2 + 1].min() > 0.9
    assert d2[:, :N // 2 - 2].max() < 1e-6   # far from the jump: constant data


def _fd_worst(lossgrad, seed=3):
    """Worst per-block relative difference between `lossgrad`'s gradient and
    central differences of its loss (a sample of each block)."""
    theta, X, y = _kink_free_batch(seed, B=12)
    _, g = lossgrad(theta, X, y, 2.0)
    sizes = [M.NH * M.NIN, M.NH, M.NH * M.NH, M.NH, M.NH, 1]
    starts = np.cumsum([0] + sizes[:-1])
    rng = np.random.default_rng(seed)
    worst = 0.0
    for s0, n in zip(starts, sizes):
        idx = s0 + rng.choice(n, min(n, 24), replace=False)
        fd = []
        for k in idx:
            tp, tm = theta.copy(), theta.copy()
            tp[k] += 1e-6
            tm[k] -= 1e-6
            fd.append((lossgrad(tp, X, y, 2.0)[0] - lossgrad(tm, X, y, 2.0)[0]) / 2e-6)
        fd = np.array(fd)
        worst = max(worst, float(np.linalg.norm(g[idx] - fd) / np.linalg.norm(fd)))
    return worst


def test_gradient_pin_catches_a_transposed_block():
    """The finite-difference pin fails on an oracle whose W2 gradient block is
    transposed (a plausible back-propagation mistake, planted on the CPU)."""
    def planted(theta, X, y, pw):
        loss, g = M.loss_and_grad(theta, X, y, pw)
        o = M.NH * M.NIN + M.NH
        g = g.copy()
        g[o:o + M.NH * M.NH] = g[o:o + M.NH * M.NH].reshape(M.NH, M.NH).T.ravel()
        return loss, g
    assert _fd_worst(M.loss_and_grad) < 1e-6
    assert _fd_worst(planted) > 1e-2
