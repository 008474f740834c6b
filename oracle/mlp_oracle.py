"""Plain numpy FP64 oracle of the learned troubled-cell indicator.

TEST INFRASTRUCTURE ONLY (same rules as the rest of oracle/).  The paper has
no learned part: this restates the indicator's definition, which the CUDA
kernels implement independently:

* features of cell (i, j): the 5 x 5 patch (offsets -2..2) of the density's
  cell average, x-moment and y-moment, ghost cells by the scheme's boundary
  rules; with c the centre average and R the patch's average range,
  s = 1 / (R + KAPPA |c| + TINY) and the 75 features are (rho_k - c) s,
  vbar_k s, wbar_k s, ordered [field][dy][dx] with dx fastest;
* network: 75 -> 32 (ReLU) -> 32 (ReLU) -> 1, p = sigmoid(z);
* label: troubled when the plain scheme's largest |omega_m/gamma_m - 1| over
  its reconstructed fields exceeds DELTA (oracle.weight_deviation);
* loss: class-weighted binary cross entropy, mean over the batch;
* Adam (Kingma & Ba, 2015) with bias correction.
Parameters are one flat vector in the order W1 (32x75, row-major), b1 (32),
W2 (32x32), b2 (32), w3 (32), b3 (1): 3521 values.
"""
from __future__ import annotations

import numpy as np

NIN, NH = 75, 32
KAPPA = 1e-3
TINY = 1e-30
DELTA = 0.1
NPARAM = NH * NIN + NH + NH * NH + NH + NH + 1


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = theta[o:o + NH * NIN].reshape(NH, NIN); o += NH * NIN
    b1 = theta[o:o + NH]; o += NH
    W2 = theta[o:o + NH * NH].reshape(NH, NH); o += NH * NH
    b2 = theta[o:o + NH]; o += NH
    w3 = theta[o:o + NH]; o += NH
    b3 = theta[o:o + 1]; o += 1
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, b3]).astype(np.float64)


def init_params(seed: int) -> np.ndarray:
    """He-normal hidden layers, small output layer, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, np.sqrt(2.0 / NIN), size=(NH, NIN))
    W2 = rng.normal(0.0, np.sqrt(2.0 / NH), size=(NH, NH))
    w3 = rng.normal(0.0, np.sqrt(1.0 / NH), size=NH)
    return pack(W1, np.zeros(NH), W2, np.zeros(NH), w3, np.zeros(1))


def features_from_padded(P: np.ndarray, nc: int) -> np.ndarray:
    """P: padded state [nf][ny+4][nx+4]; returns features [ny*nx][75]."""
    ny, nx = P.shape[1] - 4, P.shape[2] - 4
    rho, vb, wb = P[0], P[nc], P[2 * nc]
    out = np.zeros((ny, nx, NIN))
    for j in range(ny):
        for i in range(nx):
            pr = rho[j:j + 5, i:i + 5]
            c = pr[2, 2]
            s = 1.0 / ((pr.max() - pr.min()) + KAPPA * abs(c) + TINY)
            out[j, i, 0:25] = ((pr - c) * s).ravel()
            out[j, i, 25:50] = (vb[j:j + 5, i:i + 5] * s).ravel()
            out[j, i, 50:75] = (wb[j:j + 5, i:i + 5] * s).ravel()
    return out.reshape(ny * nx, NIN)


def forward(theta, X):
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ w3 + b3[0]
    p = 1.0 / (1.0 + np.exp(-z))
    return p, (a1, h1, a2, h2, z)


def loss_and_grad(theta, X, y, pos_weight):
    """Mean class-weighted BCE and its gradient with respect to theta."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    p, (a1, h1, a2, h2, z) = forward(theta, X)
    B = X.shape[0]
    wt = np.where(y > 0.5, pos_weight, 1.0)
    # log(sigmoid(z)) and log(1 - sigmoid(z)) written without overflow
    logp = -np.logaddexp(0.0, -z)
    log1mp = -np.logaddexp(0.0, z)
    loss = -np.mean(wt * (y * logp + (1.0 - y) * log1mp))
    dz = wt * (p - y) / B
    gw3 = h2.T @ dz
    gb3 = np.array([dz.sum()])
    dh2 = np.outer(dz, w3) * (a2 > 0.0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (a1 > 0.0)
    gW1 = dh1.T @ X
    gb1 = dh1.sum(axis=0)
    return loss, pack(gW1, gb1, gW2, gb2, gw3, gb3)


def adam_step(theta, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step t >= 1); returns new theta, m, v."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
