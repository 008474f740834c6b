"""Training driver of the learned troubled-cell indicator (the network itself,
its features, labels, forward/backward passes, Adam and the tensor-core
inference all run in libhweno's kernels; this module only orchestrates).

Data: snapshots of the plain nonlinear HWENO solver (GPU, FP64) on the
shock / entropy-wave family (Mach 1.1-3 shock into a sinusoidal density
field), every cell labelled by the plain scheme's own weights:
troubled  <=>  max |omega_m / gamma_m - 1| > delta.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import hweno as hw
from . import workloads as W

W2D = (0.99, 0.0025, 0.0025, 0.0025, 0.0025)
DELTA = 0.1        # label threshold on max |omega/gamma - 1|
P_THRESHOLD = 0.5  # troubled when p > P_THRESHOLD


def shock_entropy_config(n: int, precision: int = hw.FP64) -> hw.Config:
    """[0,1]^2, inflow on the left (post-shock state), outflow elsewhere."""
    return hw.Config(dim=2, nx=n, ny=n, equation=hw.EQ_EULER, lin_w=W2D, precision=precision,
                     bc=(hw.BC_INFLOW, hw.BC_OUTFLOW, hw.BC_OUTFLOW, hw.BC_OUTFLOW))


def shock_entropy_problem(seed: int, n: int, precision: int = hw.FP64):
    """(config, initial state) of one member of the family; the shock sits on
    the cell face nearest x = 0.2 (exactly 0.2 when n is a multiple of 5)."""
    f = W.shock_entropy_2d(seed=seed, x_shock=round(0.2 * n) / n)
    prm = f.params
    cfg = shock_entropy_config(n, precision)
    post = W.prim_to_cons_2d(prm["rho2"], prm["u2"], 0.0, prm["p2"])
    cfg.bc_state = [list(post), [0.0] * 4, [0.0] * 4, [0.0] * 4]
    U0 = W.cells_2d(f, 0.0, 1.0, 0.0, 1.0, n, n, nq=4)
    return cfg, U0


@dataclass
class Dataset:
    feat: "object"   # torch float32 [N][75] on the device
    dev: "object"    # torch float32 [N]
    n: int


def generate(seeds, n: int = 160, times=(0.0, 0.02, 0.05, 0.1)) -> Dataset:
    """Features and label sources of every cell of the given snapshots."""
    import torch
    feats, devs = [], []
    for seed in seeds:
        cfg, U0 = shock_entropy_problem(seed, n)
        s = hw.Solver(cfg)
        s.set_state(torch.from_numpy(U0).cuda())
        t_now = 0.0
        for t in times:
            if t > t_now:
                s.advance(t)
                t_now = t
            F = torch.empty((n * n, 75), dtype=torch.float32, device="cuda")
            D = torch.empty((n * n,), dtype=torch.float32, device="cuda")
            hw.hweno_indicator_features(s.h, F)
            hw.hweno_indicator_labels(s.h, D)
            feats.append(F)
            devs.append(D)
        s.close()
    feat = torch.cat(feats)
    dev = torch.cat(devs)
    torch.cuda.synchronize()
    return Dataset(feat=feat, dev=dev, n=feat.shape[0])


def init_params(seed: int) -> np.ndarray:
    """He-normal hidden layers, small output layer, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, math.sqrt(2.0 / 75), size=(32, 75))
    W2 = rng.normal(0.0, math.sqrt(2.0 / 32), size=(32, 32))
    w3 = rng.normal(0.0, math.sqrt(1.0 / 32), size=32)
    return np.concatenate([W1.ravel(), np.zeros(32), W2.ravel(), np.zeros(32), w3, np.zeros(1)]).astype(np.float32)


def train(data: Dataset, epochs: int = 6, batch: int = 4096, lr: float = 3e-3, seed: int = 0,
          delta: float = DELTA, pos_weight: float | None = None, verbose: bool = False):
    """Adam on the GPU through hweno_indicator_train (one C call: the epoch
    loop, the seeded minibatch order and the class weight all live there);
    returns (parameters, per-epoch mean losses)."""
    theta, losses = hw.hweno_indicator_train(data.feat, data.dev, epochs, batch, lr, delta,
                                             pos_weight=0.0 if pos_weight is None else pos_weight,
                                             seed=seed, init_params=init_params(seed))
    if verbose:
        for ep, l in enumerate(losses):
            print(f"epoch {ep}: loss {l:.4f}")
    return theta, losses


def evaluate(theta, data: Dataset, delta: float = DELTA, p_threshold: float = P_THRESHOLD) -> dict:
    """Recall and precision of the FP32 network on a dataset."""
    import torch
    m = hw.hweno_mlp_create(1)
    try:
        hw.hweno_mlp_set_params(m, theta)
        prob = torch.empty((data.n,), dtype=torch.float32, device="cuda")
        hw.hweno_mlp_predict(m, data.feat, prob)
        torch.cuda.synchronize()
    finally:
        hw.hweno_mlp_destroy(m)
    y = data.dev > delta
    pred = prob > p_threshold
    tp = int((y & pred).sum().item())
    fn = int((y & ~pred).sum().item())
    fp = int((~y & pred).sum().item())
    return {"recall": tp / max(tp + fn, 1), "precision": tp / max(tp + fp, 1),
            "positives": float(y.float().mean().item()), "flagged": float(pred.float().mean().item())}
