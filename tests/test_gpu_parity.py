"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Parity bar (FP64): every field plane within 1e-12 of the oracle relative to
the plane's largest magnitude -- single operator applications on rough
seeded data (nonlinear weights fully active), every boundary condition,
grids spanning several tiles with ragged tails; whole runs on smooth data;
shock runs compared in L1 (rounding differences are amplified by the
nonlinear weights near discontinuities).
FP32: the stated bounds below, derived from the FP32 conditioning of each
operator plane (the oracle's spread under unit-roundoff input noise).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2607_24325_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_24325_b300 import hweno as hw  # noqa: E402
from helpers import cfg_from, plane_rel_err, oracle_spread, within_spread, window_operator    # noqa: E402

W2D = (0.99, 0.0025, 0.0025, 0.0025, 0.0025)
TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _operator_pair(prob, U, ax, ay=0.0, precision=hw.FP64):
    s = hw.Solver(cfg_from(prob, precision))
    s.set_state(torch.from_numpy(np.ascontiguousarray(U)).cuda())
    L, D = s.apply_operator(ax, ay)
    torch.cuda.synchronize()
    Lr, Dr = oracle.operator(prob, U, ax, ay)
    out = (L.double().cpu().numpy(), D.double().cpu().numpy(), Lr, Dr)
    s.close()
    return out


BC1 = [(oracle.BC_PERIODIC, oracle.BC_PERIODIC), (oracle.BC_OUTFLOW, oracle.BC_OUTFLOW),
       (oracle.BC_REFLECT, oracle.BC_REFLECT), (oracle.BC_INFLOW, oracle.BC_OUTFLOW)]


# ------------------------------------------------------------ 1D operator
@pytest.mark.parametrize("eq,charwise", [(oracle.EQ_ADVECTION, 1), (oracle.EQ_BURGERS, 1),
                                         (oracle.EQ_EULER, 1), (oracle.EQ_EULER, 0)])
@pytest.mark.parametrize("n", [3, 31, 97, 1000])
@pytest.mark.parametrize("bc", BC1)
def test_operator_1d_fp64(eq, charwise, n, bc):
    euler = eq == oracle.EQ_EULER
    U = W.random_state(1, (n,), seed=n + 7 * eq, euler=euler)
    st = [list(W.prim_to_cons_1d(1.2, 0.3, 0.9)) + [0.0], list(W.prim_to_cons_1d(0.8, -0.2, 1.1)) + [0.0],
          [0.0] * 4, [0.0] * 4] if euler else [[0.7, 0, 0, 0], [-0.4, 0, 0, 0], [0.0] * 4, [0.0] * 4]
    prob = oracle.Problem(dim=1, equation=eq, nx=n, xlo=-0.3, xhi=1.7, adv_x=-1.3, charwise=charwise,
                          bc=bc + (0, 0), bc_state=st)
    L, D, Lr, Dr = _operator_pair(prob, U, 2.5)
    assert plane_rel_err(L, Lr) < TOL64
    assert plane_rel_err(D, Dr) < TOL64


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_operator_1d_random_weights_and_pow2(seed):
    n = 77
    U = W.random_state(1, (n,), seed=seed, euler=True)
    prob = oracle.Problem(dim=1, equation=oracle.EQ_EULER, nx=n, lin_w=W.random_positive_weights(3, seed),
                          weight_pow=1 + seed % 2, eps=10.0 ** (-6 - seed), bc=(oracle.BC_OUTFLOW,) * 4)
    L, D, Lr, Dr = _operator_pair(prob, U, 1.7)
    assert plane_rel_err(L, Lr) < TOL64 and plane_rel_err(D, Dr) < TOL64


def test_operator_1d_linear_weights():
    n = 64
    U = W.random_state(1, (n,), seed=3, euler=True)
    prob = oracle.Problem(dim=1, equation=oracle.EQ_EULER, nx=n, linear_weights=1)
    L, D, Lr, Dr = _operator_pair(prob, U, 1.7)
    assert plane_rel_err(L, Lr) < TOL64 and plane_rel_err(D, Dr) < TOL64


# ------------------------------------------------------------ 2D operator
BC2 = [(0, 0, 0, 0), (1, 1, 1, 1), (2, 2, 2, 2), (3, 1, 2, 2), (0, 0, 1, 1), (2, 2, 0, 0), (1, 3, 3, 2)]


@pytest.mark.parametrize("eq,charwise", [(oracle.EQ_ADVECTION, 1), (oracle.EQ_BURGERS, 1),
                                         (oracle.EQ_EULER, 1), (oracle.EQ_EULER, 0)])
@pytest.mark.parametrize("nx,ny", [(3, 3), (37, 23), (64, 61)])
@pytest.mark.parametrize("bc", BC2)
def test_operator_2d_fp64(eq, charwise, nx, ny, bc):
    euler = eq == oracle.EQ_EULER
    U = W.random_state(2, (ny, nx), seed=nx * ny + eq, euler=euler, moment_scale=0.3)
    if euler:
        st = [list(W.prim_to_cons_2d(1.0 + 0.1 * k, 0.2 * k - 0.3, 0.1 - 0.1 * k, 1.0 + 0.05 * k)) for k in range(4)]
    else:
        st = [[0.3 * k - 0.5, 0, 0, 0] for k in range(4)]
    prob = oracle.Problem(dim=2, equation=eq, nx=nx, ny=ny, xlo=0, xhi=1.3, ylo=-1, yhi=0.5, adv_x=0.7,
                          adv_y=-1.1, lin_w=W2D, charwise=charwise, bc=bc, bc_state=st)
    L, D, Lr, Dr = _operator_pair(prob, U, 2.2, 1.9)
    assert plane_rel_err(L, Lr) < TOL64
    assert plane_rel_err(D, Dr) < TOL64


@pytest.mark.parametrize("seed", [0, 1])
def test_operator_2d_random_weights(seed):
    nx, ny = 45, 33
    U = W.random_state(2, (ny, nx), seed=seed, euler=True, moment_scale=0.3)
    prob = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=nx, ny=ny, lin_w=W.random_positive_weights(5, seed),
                          weight_pow=1 + seed, bc=(0, 0, 1, 1))
    L, D, Lr, Dr = _operator_pair(prob, U, 2.2, 1.9)
    assert plane_rel_err(L, Lr) < TOL64 and plane_rel_err(D, Dr) < TOL64


def test_operator_2d_large_sampled():
    """A 300 x 271 grid (10 x 10 tiles, ragged): the oracle is slow here, so
    compare a full application on Burgers and the exact symmetry of a
    transposed problem."""
    nx, ny = 300, 271
    U = W.random_state(2, (ny, nx), seed=5, moment_scale=0.3)
    prob = oracle.Problem(dim=2, equation=oracle.EQ_BURGERS, nx=nx, ny=ny, lin_w=W2D)
    L, D, Lr, Dr = _operator_pair(prob, U, 3.0, 3.0)
    assert plane_rel_err(L, Lr) < TOL64 and plane_rel_err(D, Dr) < TOL64


# ------------------------------------- Jiang-Shu (typical) indicator variant
@pytest.mark.parametrize("dim,eq,charwise", [(1, oracle.EQ_ADVECTION, 1), (1, oracle.EQ_EULER, 1),
                                             (2, oracle.EQ_BURGERS, 1), (2, oracle.EQ_EULER, 1),
                                             (2, oracle.EQ_EULER, 0)])
def test_operator_typical_indicator_fp64(dim, eq, charwise):
    """The smoothness-indicator variant the paper replaces (Eq.
    smoothness-indicator-typical and its 2D form), FP64, rough data: parity
    with the oracle, and the switch changes the result."""
    euler = eq == oracle.EQ_EULER
    if dim == 1:
        n = 203
        U = W.random_state(1, (n,), seed=41 + eq, euler=euler)
        kw = dict(dim=1, nx=n, lin_w=(0.6, 0.2, 0.2), bc=(oracle.BC_OUTFLOW, oracle.BC_REFLECT, 0, 0))
        ax, ay = 2.1, 0.0
    else:
        nx, ny = 67, 41
        U = W.random_state(2, (ny, nx), seed=43 + eq, euler=euler, moment_scale=0.3)
        kw = dict(dim=2, nx=nx, ny=ny, lin_w=W2D, bc=(0, 0, 1, 2))
        ax, ay = 2.2, 1.9
    prob = oracle.Problem(equation=eq, charwise=charwise, smoothness=oracle.BETA_TYPICAL, eps=1e-6, **kw)
    L, D, Lr, Dr = _operator_pair(prob, U, ax, ay)
    assert plane_rel_err(L, Lr) < TOL64
    assert plane_rel_err(D, Dr) < TOL64
    Lm, _ = oracle.operator(oracle.Problem(equation=eq, charwise=charwise, eps=1e-6, **kw), U, ax, ay)
    assert plane_rel_err(Lm, Lr) > 1e-6


@pytest.mark.parametrize("dim", [1, 2])
def test_operator_typical_indicator_mixed(dim):
    """FP32 storage and stencil with FP64 typical indicators, on the
    FP32-rounded input: within max(2e-5, 100 x the oracle's spread under
    FP32 unit-roundoff input noise)."""
    if dim == 1:
        N = 200
        prob = oracle.Problem(dim=1, equation=oracle.EQ_EULER, nx=N, xlo=0, xhi=2,
                              smoothness=oracle.BETA_TYPICAL)
        U = W.cells_1d(W.euler_smooth_1d(0.0), 0, 2, N)
    else:
        N = 64
        prob = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=N, ny=N, xlo=0, xhi=2, ylo=0, yhi=2, lin_w=W2D,
                              smoothness=oracle.BETA_TYPICAL)
        U = W.cells_2d(W.euler_smooth_2d(0.0), 0, 2, 0, 2, N, N)
    U32 = U.astype(np.float32).astype(np.float64)
    L, D, _, _ = _operator_pair(prob, U32, 2.5, 2.5, precision=hw.FP32_IND64)
    Lr, Dr, sL, sD = oracle_spread(prob, U32, 2.5, 2.5, rel=2.0 ** -24)
    ok, e, tol = within_spread(L, Lr, sL, 2e-5)
    assert ok, (e, tol)
    ok, e, tol = within_spread(D, Dr, sD, 2e-5)
    assert ok, (e, tol)


# ------------------- split wall and moving-shock boundaries (double Mach reflection)
def _dmr_prob(nx, ny, t=0.0):
    B = W.dmr_boundary()
    return oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=nx, ny=ny, xlo=0.0, xhi=4.0, ylo=0.0, yhi=1.0,
                          lin_w=W2D, bc=B["bc"], bc_state=B["bc_state"], bc_state2=B["bc_state2"],
                          bc_param=B["bc_param"], t=t)


def test_dmr_operator_fp64():
    """One operator application on the double Mach reflection state at
    t = 0.013 (the moving shock and the split wall in the ghost cells),
    against the oracle: the bar of ill-conditioned shock data (R11)."""
    nx, ny, t = 64, 16, 0.013
    U = W.dmr_2d(nx, ny)
    prob = _dmr_prob(nx, ny, t)
    s = hw.Solver(cfg_from(prob))
    s.set_state(U)
    hw.hweno_set_time(s.h, t)
    L, D = s.apply_operator(12.0, 9.0)
    L, D = L.cpu().numpy(), D.cpu().numpy()
    s.close()
    Lr, Dr, sL, sD = oracle_spread(prob, U, 12.0, 9.0)
    ok, e, tol = within_spread(L, Lr, sL, TOL64)
    assert ok, (e, tol)
    ok, e, tol = within_spread(D, Dr, sD, TOL64)
    assert ok, (e, tol)


def test_split_and_shock_on_x_sides_fp64():
    """The two time-dependent rules on the x sides (decided by the row's y),
    rough data, at t = 0.2."""
    nx, ny, t = 37, 45, 0.2
    U = W.random_state(2, (ny, nx), seed=61, euler=True, moment_scale=0.3)
    a = list(W.prim_to_cons_2d(1.3, 0.4, -0.2, 1.1))
    b = list(W.prim_to_cons_2d(0.7, -0.1, 0.3, 0.6))
    prob = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=nx, ny=ny, xlo=0.0, xhi=1.0, ylo=-0.5, yhi=1.0,
                          lin_w=W2D, bc=(oracle.BC_SPLIT, oracle.BC_SHOCK, oracle.BC_OUTFLOW, oracle.BC_REFLECT),
                          bc_state=[a, a, a, a], bc_state2=[b, b, b, b],
                          bc_param=[[0.3, 0.0], [-0.1, 2.0], [0.0, 0.0], [0.0, 0.0]], t=t)
    s = hw.Solver(cfg_from(prob))
    s.set_state(U)
    hw.hweno_set_time(s.h, t)
    L, D = s.apply_operator(2.2, 1.9)
    L, D = L.cpu().numpy(), D.cpu().numpy()
    s.close()
    Lr, Dr = oracle.operator(prob, U, 2.2, 1.9)
    assert plane_rel_err(L, Lr) < TOL64 and plane_rel_err(D, Dr) < TOL64


@pytest.mark.parametrize("precision", [hw.FP64, hw.FP32_IND64])
def test_dmr_short_run(precision):
    """The double Mach reflection at 96 x 24 to t = 0.004 (the boundary
    values follow the stage times): same steps and final time as the oracle;
    relative L1 of every conserved component <= 1e-10 (FP64) / 2e-5 (FP32
    stencil with FP64 indicators)."""
    nx, ny, T = 96, 24, 0.004
    U = W.dmr_2d(nx, ny)
    prob = _dmr_prob(nx, ny)
    s = hw.Solver(cfg_from(prob, precision))
    s.set_state(U)
    t, n = s.advance(T)
    G = s.get_state(device=False).astype(np.float64)
    s.close()
    R, tr, nr = oracle.run(prob, U, T)
    assert n == nr and abs(t - tr) < 1e-15
    tol = 1e-10 if precision == hw.FP64 else 2e-5
    for k in range(4):
        assert np.abs(G[k] - R[k]).mean() / np.abs(R[k]).mean() < tol, k


def test_step_advances_time():
    nx, ny = 32, 8
    prob = _dmr_prob(nx, ny)
    s = hw.Solver(cfg_from(prob))
    s.set_state(W.dmr_2d(nx, ny))
    s.step(1e-4, 12.0, 9.0)
    s.step(2e-4, 12.0, 9.0)
    t, _ = hw.hweno_get_time(s.h)
    s.close()
    assert abs(t - 3e-4) < 1e-18


# ------------------------------------------------------------ whole runs
def test_run_1d_advection_config1():
    """1D advection sin(pi x) on [0,2], N = 160, CFL 0.6, to t = 2 (FP64)."""
    N = 160
    prob = oracle.Problem(dim=1, equation=oracle.EQ_ADVECTION, nx=N, xlo=0, xhi=2, lin_w=(0.995, 0.0025, 0.0025))
    U0 = W.cells_1d(lambda x: np.sin(np.pi * x)[None], 0, 2, N)
    s = hw.Solver(cfg_from(prob))
    s.set_state(U0)
    t, n = s.advance(2.0)
    got = s.get_state(device=False)
    ref, tr, nr = oracle.run(prob, U0, 2.0)
    assert t == tr and n == nr
    assert plane_rel_err(got, ref) < TOL64
    assert np.abs(got[0] - U0[0]).mean() < 1e-5


@pytest.mark.parametrize("seed", [1, 2])
def test_run_1d_random_weights(seed):
    N = 96
    prob = oracle.Problem(dim=1, equation=oracle.EQ_BURGERS, nx=N, xlo=0, xhi=2,
                          lin_w=W.random_positive_weights(3, seed), dt_rule=oracle.DT_CFL_DX53)
    U0 = W.cells_1d(W.sine_burgers_1d(0.0), 0, 2, N)
    s = hw.Solver(cfg_from(prob))
    s.set_state(U0)
    t, n = s.advance(0.25)
    got = s.get_state(device=False)
    ref, tr, nr = oracle.run(prob, U0, 0.25)
    assert n == nr and abs(t - tr) < 1e-15
    assert plane_rel_err(got, ref) < 1e-11


def test_run_1d_euler_smooth():
    N = 80
    prob = oracle.Problem(dim=1, equation=oracle.EQ_EULER, nx=N, xlo=0, xhi=2)
    U0 = W.cells_1d(W.euler_smooth_1d(0.0), 0, 2, N)
    s = hw.Solver(cfg_from(prob))
    s.set_state(U0)
    t, n = s.advance(0.5)
    got = s.get_state(device=False)
    ref, tr, nr = oracle.run(prob, U0, 0.5)
    assert n == nr
    assert plane_rel_err(got, ref) < 1e-11


def test_run_2d_burgers_smooth():
    N = 40
    prob = oracle.Problem(dim=2, equation=oracle.EQ_BURGERS, nx=N, ny=N, xlo=0, xhi=4, ylo=0, yhi=4, lin_w=W2D,
                          dt_rule=oracle.DT_CFL_DX53)
    U0 = W.cells_2d(W.sine_burgers_2d(0.0), 0, 4, 0, 4, N, N)
    T = 0.5 / math.pi
    s = hw.Solver(cfg_from(prob))
    s.set_state(U0)
    t, n = s.advance(T)
    got = s.get_state(device=False)
    ref, tr, nr = oracle.run(prob, U0, T)
    assert n == nr
    assert plane_rel_err(got, ref) < 1e-11
    ex = W.cells_2d(W.sine_burgers_2d(T), 0, 4, 0, 4, N, N)[0]
    assert abs(np.abs(got[0] - ex).mean() / 3.87e-05 - 1) < 0.3   # Example 3 table, 40 x 40


def test_run_2d_euler_smooth_steps():
    N = 24
    prob = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=N, ny=N, xlo=0, xhi=2, ylo=0, yhi=2, lin_w=W2D)
    U0 = W.cells_2d(W.euler_smooth_2d(0.0), 0, 2, 0, 2, N, N)
    s = hw.Solver(cfg_from(prob))
    s.set_state(U0)
    t, n = s.advance(1.0, max_steps=12)
    got = s.get_state(device=False)
    ref, tr, nr = oracle.run(prob, U0, 1.0, max_steps=12)
    assert n == nr == 12 and abs(t - tr) < 1e-14
    assert plane_rel_err(got, ref) < 1e-11


def test_run_2d_quadrant_l1():
    """Four-quadrant Riemann problem (seeded states), shocks form: L1 parity."""
    N = 48
    prob = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=N, ny=N, lin_w=W2D, bc=(oracle.BC_OUTFLOW,) * 4)
    U0 = W.quadrant_2d(W.quadrant_states(2024), 0.5, 0.5, 0, 1, 0, 1, N, N)
    s = hw.Solver(cfg_from(prob))
    s.set_state(U0)
    t, n = s.advance(0.05)
    got = s.get_state(device=False)
    ref, tr, nr = oracle.run(prob, U0, 0.05)
    assert n == nr
    for k in range(4):
        assert np.abs(got[k] - ref[k]).mean() < 1e-10 * np.abs(ref[k]).mean()


def test_conservation_gpu_fp64():
    N = 128
    prob = oracle.Problem(dim=1, equation=oracle.EQ_BURGERS, nx=N, xlo=0, xhi=2)
    U0 = W.cells_1d(W.sine_burgers_1d(0.0), 0, 2, N)
    s = hw.Solver(cfg_from(prob))
    s.set_state(U0)
    s.advance(1.5)
    got = s.get_state(device=False)
    assert abs(got[0].sum() - U0[0].sum()) < 1e-12 * np.abs(U0[0]).sum()


# ------------------------------------------------------------ batch
def test_batch_operator_and_runs():
    B = W.riemann_batch_1d(n=6, seed=1234, nmin=20, nmax=300)
    cfgs, states, probs = [], [], []
    for k in range(B.sizes.size):
        p = oracle.Problem(dim=1, equation=oracle.EQ_EULER, nx=int(B.sizes[k]), bc=(oracle.BC_OUTFLOW,) * 4)
        probs.append(p)
        cfgs.append(cfg_from(p))
        states.append(B.instance(k))
    b = hw.Batch(cfgs)
    U = b.pack(states)
    b.set_state(torch.from_numpy(U).cuda())
    alphas = [1.0 + 0.5 * k for k in range(b.n)]
    L, D = b.apply_operator(alphas)
    torch.cuda.synchronize()
    Ls, Ds = b.unpack(L), b.unpack(D)
    for k, p in enumerate(probs):
        # Riemann data: the weights next to a jump are epsilon-sensitive, so the
        # bar is the oracle's own spread under FP64 unit-roundoff input noise
        Lr, Dr, sL, sD = oracle_spread(p, states[k], alphas[k])
        ok, e, tol = within_spread(Ls[k], Lr, sL, TOL64)
        assert ok, (k, e, tol)
        ok, e, tol = within_spread(Ds[k], Dr, sD, TOL64)
        assert ok, (k, e, tol)
    tf = [0.02 + 0.01 * k for k in range(b.n)]
    t, n = b.advance(tf)
    got = b.unpack(b.get_state())
    for k, p in enumerate(probs):
        ref, tr, nr = oracle.run(p, states[k], tf[k])
        assert n[k] == nr and abs(t[k] - tr) < 1e-15
        for f in range(3):
            assert np.abs(got[k][f] - ref[f]).mean() < 1e-9 * np.abs(ref[f]).mean()


# ------------------------------------------------------------ FP32
@pytest.mark.parametrize("precision", [hw.FP32, hw.FP32_IND64])
@pytest.mark.parametrize("dim,eq", [(1, oracle.EQ_EULER), (2, oracle.EQ_EULER), (2, oracle.EQ_BURGERS)])
def test_fp32_operator_within_fp32_conditioning(dim, eq, precision):
    """FP32 stencil arithmetic, judged on the FP32-rounded input: every plane
    within max(2e-5, 100 x the oracle's spread under FP32 unit-roundoff input
    noise).  The derivative-equation planes are ill-conditioned (their
    fluxes cancel to O(dx)), which the spread measures."""
    if dim == 1:
        N = 200
        prob = oracle.Problem(dim=1, equation=eq, nx=N, xlo=0, xhi=2)
        U = W.cells_1d(W.euler_smooth_1d(0.0), 0, 2, N)
    else:
        N = 64
        prob = oracle.Problem(dim=2, equation=eq, nx=N, ny=N, xlo=0, xhi=2, ylo=0, yhi=2, lin_w=W2D)
        f = W.euler_smooth_2d(0.0) if eq == oracle.EQ_EULER else W.sine_burgers_2d(0.0)
        U = W.cells_2d(f, 0, 2, 0, 2, N, N)
    U32 = U.astype(np.float32).astype(np.float64)
    L, D, _, _ = _operator_pair(prob, U32, 2.5, 2.5, precision=precision)
    Lr, Dr, sL, sD = oracle_spread(prob, U32, 2.5, 2.5, rel=2.0 ** -24)
    ok, e, tol = within_spread(L, Lr, sL, 2e-5)
    assert ok, (e, tol)
    ok, e, tol = within_spread(D, Dr, sD, 2e-5)
    assert ok, (e, tol)


@pytest.mark.parametrize("precision", [hw.FP32, hw.FP32_IND64])
def test_fp32_smooth_runs_close_to_fp64_oracle(precision):
    """Whole FP32 runs on smooth data against the FP64 oracle: the relative
    L1 difference of the cell averages stays at the FP32 rounding level."""
    N = 200
    prob = oracle.Problem(dim=1, equation=oracle.EQ_EULER, nx=N, xlo=0, xhi=2)
    U0 = W.cells_1d(W.euler_smooth_1d(0.0), 0, 2, N)
    s = hw.Solver(cfg_from(prob, precision))
    s.set_state(U0)
    t, n = s.advance(0.5)
    got = s.get_state(device=False).astype(np.float64)
    ref, tr, nr = oracle.run(prob, U0, 0.5)
    assert abs(n - nr) <= 1
    rel = [np.abs(got[k] - ref[k]).mean() / np.abs(ref[k]).mean() for k in range(3)]
    print(f"precision {precision} vs FP64 oracle, 1D Euler smooth N=200 t=0.5, relative L1:", rel)
    assert max(rel) < 5e-6
    N = 48
    p2 = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=N, ny=N, xlo=0, xhi=2, ylo=0, yhi=2, lin_w=W2D)
    V0 = W.cells_2d(W.euler_smooth_2d(0.0), 0, 2, 0, 2, N, N)
    s2 = hw.Solver(cfg_from(p2, precision))
    s2.set_state(V0)
    s2.advance(0.25)
    g2 = s2.get_state(device=False).astype(np.float64)
    r2, _, _ = oracle.run(p2, V0, 0.25)
    rel2 = [np.abs(g2[k] - r2[k]).mean() / np.abs(r2[k]).mean() for k in range(4)]
    print(f"precision {precision} vs FP64 oracle, 2D Euler smooth 48^2 t=0.25, relative L1:", rel2)
    assert max(rel2) < 5e-6


def test_nonphysical_state_reported():
    """A negative pressure put into the initial state (host-made fault) is
    reported as HWENO_ERR_NONPHYSICAL, never a device fault."""
    N = 32
    U = W.cells_1d(W.euler_smooth_1d(0.0), 0, 2, N)
    U[2, 5] = -1.0   # energy below kinetic energy: p < 0
    prob = oracle.Problem(dim=1, equation=oracle.EQ_EULER, nx=N, xlo=0, xhi=2)
    s = hw.Solver(cfg_from(prob))
    with pytest.raises(hw.HwenoError) as ei:
        s.set_state(U)
        s.advance(0.1)
    assert ei.value.status == hw.HWENO_ERR_NONPHYSICAL


def test_fp32_ind64_shock_run_l1():
    """Mixed precision through shocks (four-quadrant problem) vs the oracle:
    relative L1 of every component within 1e-5."""
    N = 48
    prob = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=N, ny=N, lin_w=W2D, bc=(oracle.BC_OUTFLOW,) * 4)
    U0 = W.quadrant_2d(W.quadrant_states(2024), 0.5, 0.5, 0, 1, 0, 1, N, N)
    s = hw.Solver(cfg_from(prob, hw.FP32_IND64))
    s.set_state(U0)
    s.advance(0.05)
    got = s.get_state(device=False).astype(np.float64)
    ref, _, _ = oracle.run(prob, U0, 0.05)
    for k in range(4):
        assert np.abs(got[k] - ref[k]).mean() < 1e-5 * np.abs(ref[k]).mean()


def test_project_matches_input_generator():
    """hweno_project (host Gauss-Legendre of a u0 callback) gives the cell
    averages and derivative moments the shared input generator computes."""
    N = 24
    cfg = hw.Config(dim=2, nx=N, ny=N + 3, xlo=0, xhi=2, ylo=-1, yhi=1, equation=hw.EQ_EULER, lin_w=W2D)
    s = hw.Solver(cfg)
    f = W.euler_smooth_2d(0.3)
    hw.hweno_project(s.h, f, nc=4, nq=6)
    got = s.get_state(device=False)
    ref = W.cells_2d(f, 0, 2, -1, 1, N, N + 3, nq=6)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
    c1 = hw.Config(dim=1, nx=50, xlo=0, xhi=2, equation=hw.EQ_BURGERS)
    s1 = hw.Solver(c1)
    f1 = W.sine_burgers_1d(0.1)
    hw.hweno_project(s1.h, lambda x, y: f1(x), nc=1, nq=5)
    np.testing.assert_allclose(s1.get_state(device=False), W.cells_1d(f1, 0, 2, 50, nq=5), rtol=0, atol=1e-13)


def test_autotune_keeps_results():
    """The autotuner only changes launch shapes: operator results before and
    after tuning are identical (same arithmetic per cell), 1D batch and 2D."""
    B = W.riemann_batch_1d(n=5, seed=3, nmin=40, nmax=400)
    cfgs = [hw.Config(dim=1, nx=int(B.sizes[k]), equation=hw.EQ_EULER, bc=(hw.BC_OUTFLOW,) * 4) for k in range(5)]
    b = hw.Batch(cfgs)
    b.set_state(torch.from_numpy(b.pack([B.instance(k) for k in range(5)])).cuda())
    L0, D0 = b.apply_operator([1.5] * 5)
    ms, shape = hw.hweno_batch_autotune(b.h, reps=2)
    assert ms > 0 and shape[0] in (2, 4, 8) and shape[1] in (4, 8, 16, 32)
    L1, D1 = b.apply_operator([1.5] * 5)
    assert torch.equal(L0, L1) and torch.equal(D0, D1)
    N = 70
    prob = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=N, ny=N, lin_w=W2D, bc=(1, 1, 1, 1))
    s = hw.Solver(cfg_from(prob))
    s.set_state(W.quadrant_2d(W.quadrant_states(5), 0.5, 0.5, 0, 1, 0, 1, N, N))
    La, Da = s.apply_operator(2.0, 2.0)
    ms, shape = hw.hweno_autotune(s.h, reps=2)
    assert shape[2] in (0, 1)
    Lb, Db = s.apply_operator(2.0, 2.0)
    assert torch.equal(La, Lb) and torch.equal(Da, Db)


def test_checkpoint_resume_is_bitwise(tmp_path):
    """Run 2N steps == run N, save, load into a fresh solver, run N (bitwise)."""
    N = 64
    prob = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=N, ny=N, lin_w=W2D, bc=(1, 1, 1, 1))
    U0 = W.quadrant_2d(W.quadrant_states(2024), 0.5, 0.5, 0, 1, 0, 1, N, N)
    a = hw.Solver(cfg_from(prob))
    a.set_state(U0)
    a.advance(1e9, max_steps=20)
    ta, _ = hw.hweno_get_time(a.h)
    b = hw.Solver(cfg_from(prob))
    b.set_state(U0)
    b.advance(1e9, max_steps=10)
    b.save(str(tmp_path / "ck.npz"))
    c = hw.Solver(cfg_from(prob))
    c.load(str(tmp_path / "ck.npz"))
    c.advance(1e9, max_steps=10)
    tc, _ = hw.hweno_get_time(c.h)
    assert ta == tc
    assert np.array_equal(a.get_state(device=False), c.get_state(device=False))


@pytest.mark.parametrize("dim", [1, 2])
def test_constant_state_is_steady(dim):
    """Degenerate case: a constant state (zero normal velocity at reflective
    walls, the same state at inflow sides) has L = 0 up to round-off under
    every boundary condition, and limited derivatives 0."""
    if dim == 1:
        st = W.prim_to_cons_1d(1.3, 0.0, 0.7)
        n = 61
        U = np.concatenate([np.repeat(st[:, None], n, axis=1), np.zeros((3, n))])
        bcs = [(0, 0), (1, 1), (2, 2), (3, 3)]
    else:
        st = W.prim_to_cons_2d(1.3, 0.0, 0.0, 0.7)
        n = 37
        U = np.concatenate([np.repeat(np.repeat(st[:, None, None], n, 1), n, 2), np.zeros((8, n, n))])
        bcs = [(0, 0, 0, 0), (1, 1, 1, 1), (2, 2, 2, 2), (3, 3, 3, 3), (2, 1, 0, 0)]
    for bc in bcs:
        stt = [list(st) + [0.0] * (4 - len(st))] * 4
        prob = oracle.Problem(dim=dim, equation=oracle.EQ_EULER, nx=n, ny=n, lin_w=W2D if dim == 2 else (0.995, 0.0025, 0.0025),
                              bc=tuple(bc) + (0,) * (4 - len(bc)), bc_state=stt)
        s = hw.Solver(cfg_from(prob))
        s.set_state(U)
        L, D = s.apply_operator(2.0, 2.0)
        L = L.cpu().numpy()
        scale = 2.0 * np.abs(st).max() / prob.dx
        assert np.abs(L).max() < 1e-13 * scale, (bc, np.abs(L).max())
        assert np.abs(D.cpu().numpy()).max() < 1e-13 * np.abs(st).max()
        s.close()


@pytest.mark.parametrize("precision", [hw.FP64, hw.FP32_IND64])
def test_full_size_sampled_parity(precision):
    """The bench's 4096^2 four-quadrant state, launch shape autotuned as in
    bench.py: one operator application, 60 sampled cells (a third on the
    discontinuities) against oracle windows.  Per output: within 1e-12 (FP64)
    or 2e-5 (mixed precision: FP32 storage and stencil) of the plane's scale,
    or within 100x the oracle's own spread at that cell under unit-roundoff
    input perturbations."""
    n = 4096
    U = W.quadrant_2d(W.quadrant_states(2024), 0.5, 0.5, 0.0, 1.0, 0.0, 1.0, n, n)
    prob = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=n, ny=n, lin_w=W2D, bc=(1, 1, 1, 1))
    s = hw.Solver(cfg_from(prob, precision))
    s.set_state(torch.from_numpy(U).cuda())
    hw.hweno_autotune(s.h, reps=1)
    ax, ay = 2.5, 2.3
    L, D = s.apply_operator(ax, ay)
    Lh = L.double().cpu().numpy()
    Dh = D.double().cpu().numpy()
    del L, D
    s.close()
    Uin = U if precision == hw.FP64 else U.astype(np.float32).astype(np.float64)
    rel = 2.0 ** -53 if precision == hw.FP64 else 2.0 ** -24
    rng = np.random.default_rng(17)
    cells = [(int(a), int(b)) for a, b in rng.integers(8, n - 8, size=(40, 2))]
    cells += [(2048 + int(d), int(b)) for d, b in zip(rng.integers(-3, 3, 10), rng.integers(8, n - 8, 10))]
    cells += [(int(b), 2048 + int(d)) for d, b in zip(rng.integers(-3, 3, 10), rng.integers(8, n - 8, 10))]
    Lmax = np.abs(Lh).reshape(Lh.shape[0], -1).max(axis=1)
    # The limited derivatives are scaled moments (units of the averages): on
    # this piecewise-constant state they are rounding noise of size ~1e-7, so
    # their scale is the larger of their own plane maximum and that of the
    # matching average plane.
    nc = U.shape[0] // 3
    Umax = np.abs(U[:nc]).reshape(nc, -1).max(axis=1)
    Dmax = np.maximum(np.abs(Dh).reshape(Dh.shape[0], -1).max(axis=1), np.concatenate([Umax, Umax]))
    tol = 1e-12 if precision == hw.FP64 else 2e-5
    for (i, j) in cells:
        Lr, Dr, sL, sD = window_operator(prob, Uin, i, j, ax, ay, rel=rel)
        assert np.all(np.abs(Lh[:, j, i] - Lr) <= np.maximum(tol * Lmax, 100.0 * sL)), (i, j)
        assert np.all(np.abs(Dh[:, j, i] - Dr) <= np.maximum(tol * Dmax, 100.0 * sD)), (i, j)
