"""Learned troubled-cell indicator: GPU kernels against the CPU oracles.

* features and labels of a state vs oracle.mlp_oracle / oracle.weight_deviation
* loss and gradient of a minibatch (GPU FP32) vs the FP64 numpy oracle
* one Adam step vs the oracle's update
* tensor-core inference (FP16 weights and features, FP32 accumulate) vs the
  oracle's forward pass with the same FP16 rounding, and the 3x3 dilation
* a trained network: what it gains over the plain nonlinear path
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp_oracle as MO
from paper_2607_24325_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_24325_b300 import hweno as hw          # noqa: E402
from paper_2607_24325_b300 import indicator as IND     # noqa: E402
from helpers import cfg_from                            # noqa: E402

W2D = (0.99, 0.0025, 0.0025, 0.0025, 0.0025)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _quadrant(n, precision=hw.FP64, bc=(oracle.BC_OUTFLOW,) * 4):
    prob = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=n, ny=n, lin_w=W2D, bc=bc)
    U = W.quadrant_2d(W.quadrant_states(2024), 0.43, 0.57, 0, 1, 0, 1, n, n)
    return prob, U


@pytest.mark.parametrize("precision", [hw.FP64, hw.FP32])
def test_features_match_oracle(precision):
    n = 37
    prob, U = _quadrant(n, bc=(oracle.BC_REFLECT, oracle.BC_OUTFLOW, oracle.BC_PERIODIC, oracle.BC_PERIODIC))
    U = U + 0.01 * W.random_state(2, (n, n), seed=4, euler=True, moment_scale=0.2) * (precision == hw.FP64)
    s = hw.Solver(cfg_from(prob, precision))
    s.set_state(U)
    F = torch.empty((n * n, 75), dtype=torch.float32, device="cuda")
    hw.hweno_indicator_features(s.h, F)
    got = F.cpu().numpy()
    Uref = U.astype(np.float32).astype(np.float64) if precision == hw.FP32 else U
    ref = MO.features_from_padded(oracle.padded_state(prob, Uref), prob.ncomp)
    assert np.abs(got - ref).max() < 2e-4


def test_labels_match_oracle():
    n = 33
    prob, U = _quadrant(n)
    U = U + 0.02 * W.random_state(2, (n, n), seed=8, euler=True, moment_scale=0.1)
    s = hw.Solver(cfg_from(prob, hw.FP64))
    s.set_state(U)
    D = torch.empty((n * n,), dtype=torch.float32, device="cuda")
    hw.hweno_indicator_labels(s.h, D)
    got = D.cpu().numpy().reshape(n, n)
    ref = oracle.weight_deviation(prob, U)
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-6)
    assert (ref > 0.1).mean() > 0.02      # the state has troubled cells


def _dataset(n=48, seed=3):
    prob, U = _quadrant(n)
    s = hw.Solver(cfg_from(prob, hw.FP64))
    s.set_state(U)
    s.advance(0.02)
    F = torch.empty((n * n, 75), dtype=torch.float32, device="cuda")
    D = torch.empty((n * n,), dtype=torch.float32, device="cuda")
    hw.hweno_indicator_features(s.h, F)
    hw.hweno_indicator_labels(s.h, D)
    torch.cuda.synchronize()
    return F, D


def test_gradient_matches_oracle():
    F, D = _dataset()
    theta = MO.init_params(5).astype(np.float32)
    rng = np.random.default_rng(0)
    idx = rng.choice(F.shape[0], size=700, replace=False).astype(np.int32)
    m = hw.hweno_mlp_create(1024)
    hw.hweno_mlp_set_params(m, theta)
    loss, g = hw.hweno_mlp_gradient(m, F, D, torch.from_numpy(idx).cuda(), 0.1, 4.0)
    hw.hweno_mlp_destroy(m)
    X = F.cpu().numpy().astype(np.float64)[idx]
    y = (D.cpu().numpy()[idx] > 0.1).astype(np.float64)
    lr, gr = MO.loss_and_grad(theta.astype(np.float64), X, y, 4.0)
    assert abs(loss - lr) < 1e-5 * max(1.0, abs(lr))
    assert np.abs(g - gr).max() < 5e-5 * np.abs(gr).max()


def test_adam_step_matches_oracle():
    """Two GPU Adam steps against the oracle's Adam update fed with the same
    minibatch gradients (the gradients themselves are checked above)."""
    F, D = _dataset()
    theta = MO.init_params(6).astype(np.float32)
    idx_d = torch.arange(512, dtype=torch.int32, device="cuda")
    m = hw.hweno_mlp_create(512)
    hw.hweno_mlp_set_params(m, theta)
    th = theta.astype(np.float64)
    mm, vv = np.zeros_like(th), np.zeros_like(th)
    for t in (1, 2):
        _, g = hw.hweno_mlp_gradient(m, F, D, idx_d, 0.1, 3.0)
        th, mm, vv = MO.adam_step(th, mm, vv, g.astype(np.float64), t, 1e-3)
        hw.hweno_mlp_train_step(m, F, D, idx_d, 0.1, 3.0, 1e-3)
    got = hw.hweno_mlp_get_params(m)
    hw.hweno_mlp_destroy(m)
    assert np.abs(got - th).max() < 2e-6


def _forward_fp16(W1, b1, W2, b2, w3, X):
    """The kernel's arithmetic: FP16 features, weights and hidden layer-1
    activations, FP32-or-better accumulation; returns z without b3."""
    h = lambda a: a.astype(np.float32).astype(np.float16).astype(np.float64)
    h1 = np.maximum(h(X) @ h(W1).T + b1, 0.0)
    h2 = np.maximum(h(h1) @ h(W2).T + b2, 0.0)
    return h2 @ w3


def test_tensor_core_inference_matches_fp16_oracle():
    n = 70
    prob, _ = _quadrant(n)
    U = W.random_state(2, (n, n), seed=12, euler=True, moment_scale=0.3)   # varied features
    W1, b1, W2, b2, w3, _ = MO.unpack(MO.init_params(9))
    w3 = 8.0 * w3                                                          # spread the logits
    X = MO.features_from_padded(oracle.padded_state(prob, U), prob.ncomp)
    z0 = _forward_fp16(W1, b1, W2, b2, w3, X)
    b3 = np.array([-np.median(z0)])     # about half of the cells on each side
    theta = MO.pack(W1, b1, W2, b2, w3, b3).astype(np.float32)
    s = hw.Solver(cfg_from(prob, hw.FP64))
    s.set_state(U)
    hw.hweno_indicator_load(s.h, theta, 0.5)
    sm = torch.empty((n * n,), dtype=torch.uint8, device="cuda")
    tr = torch.empty((n * n,), dtype=torch.uint8, device="cuda")
    hw.hweno_indicator_mask(s.h, sm, tr)
    torch.cuda.synchronize()
    got_t = tr.cpu().numpy().reshape(n, n).astype(bool)
    got_s = sm.cpu().numpy().reshape(n, n).astype(bool)
    z = (z0 + float(np.float32(b3[0]))).reshape(n, n)
    decided = np.abs(z) > 0.02          # FP16 rounding cannot flip these
    assert decided.mean() > 0.8
    assert np.array_equal(got_t[decided], (z > 0.0)[decided])
    assert 0.2 < got_t.mean() < 0.8
    pad = np.pad(got_t, 1)
    any3 = np.zeros_like(got_t)
    for dj in range(3):
        for di in range(3):
            any3 |= pad[dj:dj + n, di:di + n]
    assert np.array_equal(got_s, ~any3)


def test_learned_indicator_gain():
    """Train on shock / entropy-wave snapshots (seeds 1-3, 160^2) and run an
    unseen member (seed 11, 320^2) to t = 0.06.  Stated accuracy: the learned
    FP32 path's density stays within 1e-3 relative L1 of the FP64 plain
    nonlinear path (the oracle's stand-in, parity-tested elsewhere) while more
    than half of the cells take the cheap linear reconstruction."""
    data = IND.generate(seeds=[1, 2, 3], n=160, times=(0.0, 0.03, 0.06, 0.1))
    theta, losses = IND.train(data, epochs=6, seed=0)
    assert losses[-1] < losses[0]
    ev = IND.evaluate(theta, data)
    assert ev["recall"] > 0.9, ev
    n, T = 320, 0.06
    cfg64, U0 = IND.shock_entropy_problem(11, n, hw.FP64)
    ref = hw.Solver(cfg64)
    ref.set_state(U0)
    ref.advance(T)
    R = ref.get_state(device=False)
    cfg32, _ = IND.shock_entropy_problem(11, n, hw.FP32)
    plain = hw.Solver(cfg32)
    plain.set_state(U0)
    plain.advance(T)
    P = plain.get_state(device=False).astype(np.float64)
    learned = hw.Solver(cfg32)
    learned.set_state(U0)
    hw.hweno_indicator_load(learned.h, theta, IND.P_THRESHOLD)
    sm = torch.empty((n * n,), dtype=torch.uint8, device="cuda")
    hw.hweno_indicator_mask(learned.h, sm, None)
    learned.advance(T)
    Lr = learned.get_state(device=False).astype(np.float64)
    smooth_frac = float(sm.float().mean().item())
    scale = np.abs(R[0]).mean()
    e_plain = np.abs(P[0] - R[0]).mean() / scale
    e_learned = np.abs(Lr[0] - R[0]).mean() / scale
    print(f"relative L1(rho) vs FP64 plain: plain FP32 {e_plain:.3e}, learned FP32 {e_learned:.3e}; "
          f"smooth fraction {smooth_frac:.3f}; train {ev}; losses {losses}")
    assert np.isfinite(Lr).all()
    assert e_learned < 1e-3
    assert smooth_frac > 0.5
