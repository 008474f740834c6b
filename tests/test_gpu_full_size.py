"""Parity at the benchmarked sizes, in the launch configuration the benchmark
times (autotuned launch shape, the whole grid or batch in one launch per
stage): one operator application of the CUDA path against the oracle on
outputs the oracle can compute one by one -- whole instances of the 1D
batch, (2r+1)^2 windows around sampled cells of the 2D grids (a cell's
outputs depend on a radius-2 neighbourhood only), with a share of the
samples on the discontinuities.

Bar per output plane: FP64 within 1e-12 of the plane's scale, the mixed
precision (FP32 storage and stencil) within 2e-5 of it; or, where the
oracle itself is ill-conditioned, within 100x its spread under unit-roundoff
input perturbations of the working precision.  The mixed path is judged on
the FP32-rounded input it actually stores."""
import dataclasses
import functools
import math

import numpy as np
import pytest

import oracle
from paper_2607_24325_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_24325_b300 import hweno as hw  # noqa: E402
from paper_2607_24325_b300 import indicator as IND  # noqa: E402
from helpers import cfg_from, oracle_spread, within_spread, window_operator  # noqa: E402

W2D = (0.99, 0.0025, 0.0025, 0.0025, 0.0025)
PRECISIONS = [hw.FP64, hw.FP32_IND64]


def _floor_rel(precision):
    return (1e-12, 2.0 ** -53) if precision == hw.FP64 else (2e-5, 2.0 ** -24)


def _stored(U, precision):
    return U if precision == hw.FP64 else U.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_batch1d_full_size_operator(precision):
    """The 256 seeded 1D Euler Riemann problems (sizes 256..8192, instance 0
    the Lax problem) in one batch: every cell of 12 instances -- the Lax
    problem, the largest, the smallest and nine drawn at random."""
    B = W.riemann_batch_1d(n=256, seed=1234)
    sizes = [int(x) for x in B.sizes]
    probs = [oracle.Problem(dim=1, equation=oracle.EQ_EULER, nx=n, bc=(oracle.BC_OUTFLOW,) * 4) for n in sizes]
    states = [B.instance(k) for k in range(len(sizes))]
    b = hw.Batch([cfg_from(p, precision) for p in probs])
    b.set_state(torch.from_numpy(b.pack(states)).cuda())
    hw.hweno_batch_autotune(b.h, reps=1)
    alphas = [oracle.alpha(p, U)[0] for p, U in zip(probs, states)]
    L, D = b.apply_operator(alphas)
    torch.cuda.synchronize()
    Ls = [x.astype(np.float64) for x in b.unpack(L)]
    Ds = [x.astype(np.float64) for x in b.unpack(D)]
    b.close()
    rng = np.random.default_rng(5)
    pick = {0, int(np.argmax(sizes)), int(np.argmin(sizes))} | set(int(k) for k in rng.integers(1, 256, 9))
    floor, rel = _floor_rel(precision)
    for k in sorted(pick):
        Lr, Dr, sL, sD = oracle_spread(probs[k], _stored(states[k], precision), alphas[k], rel=rel)
        ok, e, tol = within_spread(Ls[k], Lr, sL, floor)
        assert ok, (k, sizes[k], e, tol)
        ok, e, tol = within_spread(Ds[k], Dr, sD, floor)
        assert ok, (k, sizes[k], e, tol)


def _sampled_2d(prob, U, precision, cells, ax, ay, solver_cfg=None):
    """One operator application of the whole grid (autotuned launch shape),
    then every sampled cell against the oracle's window around it."""
    s = hw.Solver(solver_cfg if solver_cfg is not None else cfg_from(prob, precision))
    s.set_state(torch.from_numpy(U).cuda())
    hw.hweno_autotune(s.h, reps=1)
    L, D = s.apply_operator(ax, ay)
    Lh = L.double().cpu().numpy()
    Dh = D.double().cpu().numpy()
    del L, D
    s.close()
    floor, rel = _floor_rel(precision)
    Uin = _stored(U, precision)
    # plane scales; the limited-derivative planes are scaled moments (units
    # of the averages), so their scale is at least the matching average plane's
    nc = U.shape[0] // 3
    Lmax = np.abs(Lh).reshape(Lh.shape[0], -1).max(axis=1)
    Umax = np.abs(U[:nc]).reshape(nc, -1).max(axis=1)
    Dmax = np.maximum(np.abs(Dh).reshape(Dh.shape[0], -1).max(axis=1), np.concatenate([Umax, Umax]))
    for (i, j) in cells:
        Lr, Dr, sL, sD = window_operator(prob, Uin, i, j, ax, ay, rel=rel)
        assert np.all(np.abs(Lh[:, j, i] - Lr) <= np.maximum(floor * Lmax, 100.0 * sL)), (i, j)
        assert np.all(np.abs(Dh[:, j, i] - Dr) <= np.maximum(floor * Dmax, 100.0 * sD)), (i, j)


@functools.lru_cache(maxsize=1)
def _shock_entropy_state(n):
    return IND.shock_entropy_problem(11, n, hw.FP64)


def _random_cells(rng, nx, ny, count):
    return [(int(a), int(b)) for a, b in zip(rng.integers(8, nx - 8, count), rng.integers(8, ny - 8, count))]


@pytest.mark.parametrize("precision", PRECISIONS)
def test_shock_entropy_full_size_sampled(precision):
    """The shock / entropy-wave member the benchmark runs (seed 11) at
    2048^2: 40 random cells and 20 next to the shock."""
    n = 2048
    cfg, U = _shock_entropy_state(n)
    cfg = dataclasses.replace(cfg, precision=precision)
    prob = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=n, ny=n, lin_w=W2D,
                          bc=(oracle.BC_INFLOW, oracle.BC_OUTFLOW, oracle.BC_OUTFLOW, oracle.BC_OUTFLOW))
    rng = np.random.default_rng(23)
    xs = round(0.2 * n)
    cells = _random_cells(rng, n, n, 40)
    cells += [(xs + int(d), int(b)) for d, b in zip(rng.integers(-3, 3, 20), rng.integers(8, n - 8, 20))]
    _sampled_2d(prob, U, precision, cells, 4.0, 2.5, solver_cfg=cfg)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_burgers2d_full_size_sampled(precision):
    """Example 3's initial data on the benchmark's 4096^2 periodic grid."""
    n = 4096
    prob = oracle.Problem(dim=2, equation=oracle.EQ_BURGERS, nx=n, ny=n, xlo=0.0, xhi=4.0, ylo=0.0, yhi=4.0,
                          lin_w=W2D, bc=(oracle.BC_PERIODIC,) * 4)
    U = W.sine_2d_cells(n, n)
    _sampled_2d(prob, U, precision, _random_cells(np.random.default_rng(29), n, n, 50), 1.5, 1.5)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_dmr_full_size_sampled(precision):
    """The double Mach reflection's initial state on the paper's 1920 x 480
    mesh: 30 random interior cells and 30 on the oblique shock."""
    nx, ny = 1920, 480
    B = W.dmr_boundary()
    prob = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=nx, ny=ny, xlo=0.0, xhi=4.0, ylo=0.0, yhi=1.0,
                          lin_w=W2D, bc=B["bc"], bc_state=B["bc_state"], bc_state2=B["bc_state2"],
                          bc_param=B["bc_param"])
    U = W.dmr_2d(nx, ny)
    rng = np.random.default_rng(31)
    cells = _random_cells(rng, nx, ny, 30)
    for jj in rng.integers(8, ny - 8, 30):
        y = (jj + 0.5) / ny
        ii = int((1.0 / 6.0 + y / math.sqrt(3.0)) * nx / 4.0) + int(rng.integers(-2, 3))
        cells.append((ii, int(jj)))
    _sampled_2d(prob, U, precision, cells, 12.0, 10.0)
