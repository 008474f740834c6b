"""Shared test helpers: mapping an oracle problem to a library config and
the parity measure (max abs difference per field plane over the plane's max
magnitude)."""
import numpy as np

import oracle
from paper_2607_24325_b300 import hweno as hw


def cfg_from(prob: oracle.Problem, precision: int = hw.FP64) -> hw.Config:
    return hw.Config(dim=prob.dim, nx=prob.nx, ny=prob.ny if prob.dim == 2 else 1,
                     xlo=prob.xlo, xhi=prob.xhi, ylo=prob.ylo, yhi=prob.yhi,
                     equation=prob.equation, adv_x=prob.adv_x, adv_y=prob.adv_y,
                     gamma_gas=prob.gamma_gas, lin_w=tuple(prob.lin_w), eps=prob.eps,
                     weight_pow=prob.weight_pow, charwise=prob.charwise,
                     linear_weights=prob.linear_weights, cfl=prob.cfl, dt_rule=prob.dt_rule,
                     bc=tuple(prob.bc), bc_state=[list(r) for r in prob.bc_state],
                     precision=precision, smoothness=prob.smoothness,
                     bc_state2=[list(r) for r in prob.bc_state2], bc_param=[list(r) for r in prob.bc_param])


def plane_rel_err(got, ref) -> float:
    """max over field planes of max|got - ref| / (max|ref| of that plane).

    A non-finite value in `got` where `ref` is finite (or a NaN anywhere in
    the difference) counts as an infinite error, so a NaN never compares as
    "close": Python's max() would otherwise drop it."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if got.shape != ref.shape:
        raise ValueError(f"shape mismatch {got.shape} vs {ref.shape}")
    if not np.all(np.isfinite(got) | ~np.isfinite(ref)):
        return float("inf")
    worst = 0.0
    for f in range(ref.shape[0]):
        scale = np.abs(ref[f]).max() + 1e-300
        e = float(np.abs(got[f] - ref[f]).max() / scale)
        if not np.isfinite(e):
            return float("inf")
        worst = max(worst, e)
    return worst


def oracle_spread(prob, U, ax, ay=0.0, rel=2.0 ** -53, samples=4, seed=0):
    """The oracle's operator at U and its spread under random relative input
    perturbations of size `rel` (unit roundoff of the working precision):
    per-plane max|L(U') - L(U)| / max|L(U)|.  A result computed with rounding
    at that precision is only determined to within this spread."""
    L0, D0 = oracle.operator(prob, U, ax, ay)
    rng = np.random.default_rng(seed)
    sL = np.zeros(L0.shape[0])
    sD = np.zeros(D0.shape[0])
    for _ in range(samples):
        Up = U * (1.0 + rel * rng.choice([-1.0, 1.0], size=U.shape) * rng.uniform(0.5, 1.0, size=U.shape))
        L1, D1 = oracle.operator(prob, Up, ax, ay)
        for f in range(L0.shape[0]):
            sL[f] = max(sL[f], np.abs(L1[f] - L0[f]).max() / (np.abs(L0[f]).max() + 1e-300))
        for f in range(D0.shape[0]):
            sD[f] = max(sD[f], np.abs(D1[f] - D0[f]).max() / (np.abs(D0[f]).max() + 1e-300))
    return L0, D0, sL, sD


def plane_errs(got, ref):
    """Per-plane relative errors; a plane holding a NaN or an infinity that
    the reference does not have gets an infinite error."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    out = []
    for f in range(ref.shape[0]):
        bad = ~np.isfinite(got[f]) & np.isfinite(ref[f])
        e = np.abs(got[f] - ref[f]).max() / (np.abs(ref[f]).max() + 1e-300)
        out.append(np.inf if bad.any() or not np.isfinite(e) else e)
    return np.array(out)


def within_spread(got, ref, spread, floor, factor=100.0):
    """Per-plane check: error <= max(floor, factor * spread)."""
    e = plane_errs(got, ref)
    tol = np.maximum(floor, factor * np.asarray(spread))
    return bool(np.all(e <= tol)), e, tol


def window_operator(prob, U, i, j, ax, ay, r=3, rel=0.0, samples=4):
    """Oracle L and D at cell (i, j) from a (2r+1)^2 window around it (the
    operator at a cell depends on a radius-2 neighbourhood only), and their
    absolute spread under random relative input perturbations of size `rel`
    (the condition of that cell's outputs at the working precision)."""
    sub = np.ascontiguousarray(U[:, j - r:j + r + 1, i - r:i + r + 1])
    m = 2 * r + 1
    p = oracle.Problem(dim=2, equation=prob.equation, nx=m, ny=m, xlo=0, xhi=m * prob.dx, ylo=0,
                       yhi=m * prob.dy, lin_w=prob.lin_w, eps=prob.eps, weight_pow=prob.weight_pow,
                       charwise=prob.charwise, gamma_gas=prob.gamma_gas, smoothness=prob.smoothness,
                       bc=(1, 1, 1, 1))
    L, D = oracle.operator(p, sub, ax, ay)
    L0, D0 = L[:, r, r], D[:, r, r]
    sL, sD = np.zeros_like(L0), np.zeros_like(D0)
    rng = np.random.default_rng(i * 7919 + j)
    for _ in range(samples if rel > 0 else 0):
        sp = sub * (1.0 + rel * rng.choice([-1.0, 1.0], size=sub.shape) * rng.uniform(0.5, 1.0, size=sub.shape))
        L1, D1 = oracle.operator(p, sp, ax, ay)
        sL = np.maximum(sL, np.abs(L1[:, r, r] - L0))
        sD = np.maximum(sD, np.abs(D1[:, r, r] - D0))
    return L0, D0, sL, sD
