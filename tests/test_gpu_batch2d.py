"""2D batches: many 2D instances of uneven sizes (and boundaries) in one
launch per RK stage, against the oracle instance by instance and against
single solvers of the same configurations."""
import numpy as np
import pytest

import oracle
from paper_2607_24325_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_24325_b300 import hweno as hw                          # noqa: E402
from helpers import cfg_from, plane_rel_err, oracle_spread, within_spread  # noqa: E402

W2D = (0.99, 0.0025, 0.0025, 0.0025, 0.0025)
TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _mixed_problems(eq=oracle.EQ_EULER):
    """Four instances: ragged sizes, every boundary kind, one below a tile."""
    a = list(W.prim_to_cons_2d(1.3, 0.4, -0.2, 1.1))
    b = list(W.prim_to_cons_2d(0.7, -0.1, 0.3, 0.6))
    z = [[0.0] * 4 for _ in range(4)]
    kw = dict(dim=2, equation=eq, lin_w=W2D)
    return [
        oracle.Problem(nx=37, ny=23, xlo=0.0, xhi=1.3, ylo=-1.0, yhi=0.5, bc=(0, 0, 1, 1), **kw),
        oracle.Problem(nx=64, ny=61, bc=(2, 2, 3, 1), bc_state=[a, a, a, a], **kw),
        oracle.Problem(nx=5, ny=40, xlo=-0.2, xhi=0.3, bc=(3, 1, 2, 2), bc_state=[b, b, b, b], **kw),
        oracle.Problem(nx=96, ny=31, xlo=0.0, xhi=2.0, bc=(4, 1, 1, 5), bc_state=[a, a, a, a],
                       bc_state2=[b, b, b, b], bc_param=[[0.4, 0.0], z[0][:2], z[0][:2], [0.7, 3.0]], **kw),
    ]


def _states(probs, seed=0):
    out = []
    for k, p in enumerate(probs):
        euler = p.equation == oracle.EQ_EULER
        out.append(W.random_state(2, (p.ny, p.nx), seed=seed + k, euler=euler, moment_scale=0.3))
    return out


def test_batch2d_operator_fp64():
    probs = _mixed_problems()
    states = _states(probs, seed=70)
    b = hw.Batch([cfg_from(p) for p in probs])
    b.set_state(torch.from_numpy(b.pack(states)).cuda())
    alphas = [(2.0 + 0.3 * k, 1.7 + 0.2 * k) for k in range(b.n)]
    L, D = b.apply_operator(alphas)
    Ls, Ds = b.unpack(L), b.unpack(D)
    b.close()
    for k, p in enumerate(probs):
        Lr, Dr = oracle.operator(p, states[k], *alphas[k])
        assert plane_rel_err(Ls[k], Lr) < TOL64, k
        assert plane_rel_err(Ds[k], Dr) < TOL64, k


def test_batch2d_burgers_operator_fp64():
    probs = _mixed_problems(oracle.EQ_BURGERS)[:3]
    states = _states(probs, seed=80)
    b = hw.Batch([cfg_from(p) for p in probs])
    b.set_state(torch.from_numpy(b.pack(states)).cuda())
    alphas = [(2.5, 2.5)] * b.n
    L, D = b.apply_operator(alphas)
    Ls, Ds = b.unpack(L), b.unpack(D)
    b.close()
    for k, p in enumerate(probs):
        Lr, Dr = oracle.operator(p, states[k], 2.5, 2.5)
        assert plane_rel_err(Ls[k], Lr) < TOL64 and plane_rel_err(Ds[k], Dr) < TOL64, k


def test_batch2d_runs_match_oracle_and_single_solvers():
    """Four four-quadrant problems of different seeds and sizes, each to its
    own final time: steps and times as the oracle's, states within 1e-10 in
    relative L1 (shock runs), and the same as single solvers."""
    sizes = [(48, 40), (30, 30), (71, 33), (20, 52)]
    probs, states = [], []
    for k, (nx, ny) in enumerate(sizes):
        probs.append(oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=nx, ny=ny, lin_w=W2D, bc=(1, 1, 1, 1)))
        states.append(W.quadrant_2d(W.quadrant_states(100 + k), 0.43, 0.57, 0, 1, 0, 1, nx, ny))
    tf = [0.01, 0.02, 0.015, 0.005]
    b = hw.Batch([cfg_from(p) for p in probs])
    b.set_state(torch.from_numpy(b.pack(states)).cuda())
    t, n = b.advance(tf)
    got = b.unpack(b.get_state())
    b.close()
    for k, p in enumerate(probs):
        ref, tr, nr = oracle.run(p, states[k], tf[k])
        assert n[k] == nr and abs(t[k] - tr) < 1e-15, k
        for f in range(4):
            assert np.abs(got[k][f] - ref[f]).mean() < 1e-10 * np.abs(ref[f]).mean(), (k, f)
        s = hw.Solver(cfg_from(p))
        s.set_state(states[k])
        s.advance(tf[k])
        one = s.get_state(device=False)
        s.close()
        assert np.abs(one - got[k]).max() <= 1e-12 * np.abs(one).max(), k


@pytest.mark.parametrize("precision", [hw.FP32, hw.FP32_IND64])
def test_batch2d_fp32_matches_single_solvers(precision):
    probs = _mixed_problems()
    states = [s.astype(np.float32).astype(np.float64) for s in _states(probs, seed=90)]
    b = hw.Batch([cfg_from(p, precision) for p in probs])
    b.set_state(torch.from_numpy(b.pack(states)).cuda())
    alphas = [(2.0, 1.5)] * b.n
    L, D = b.apply_operator(alphas)
    Ls = b.unpack(L)
    b.close()
    for k, p in enumerate(probs):
        s = hw.Solver(cfg_from(p, precision))
        s.set_state(states[k])
        L1, _ = s.apply_operator(2.0, 1.5)
        L1 = L1.double().cpu().numpy()
        s.close()
        # the same arithmetic in another kernel instantiation: FP32 rounding
        # order may differ; the oracle's own spread at FP32 bounds it
        Lr, _, sL, _ = oracle_spread(p, states[k], 2.0, 1.5, rel=2.0 ** -24)
        ok, e, tol = within_spread(Ls[k], L1, sL, 2e-5)
        assert ok, (k, e, tol)


def test_batch2d_autotune_and_time_dependent_boundary():
    """A batch holding the double Mach reflection next to a quadrant problem:
    the moving shock follows each instance's own time."""
    nx, ny = 64, 16
    B = W.dmr_boundary()
    dmr = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=nx, ny=ny, xlo=0.0, xhi=4.0, ylo=0.0, yhi=1.0,
                         lin_w=W2D, bc=B["bc"], bc_state=B["bc_state"], bc_state2=B["bc_state2"],
                         bc_param=B["bc_param"])
    quad = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=40, ny=40, lin_w=W2D, bc=(1, 1, 1, 1))
    s_dmr, s_quad = W.dmr_2d(nx, ny), W.quadrant_2d(W.quadrant_states(5), 0.5, 0.5, 0, 1, 0, 1, 40, 40)
    b = hw.Batch([cfg_from(dmr), cfg_from(quad)])
    b.set_state(torch.from_numpy(b.pack([s_dmr, s_quad])).cuda())
    hw.hweno_batch_autotune(b.h, reps=1)
    t, n = b.advance([0.003, 0.01])
    got = b.unpack(b.get_state())
    b.close()
    ref, tr, nr = oracle.run(dmr, s_dmr, 0.003)
    assert n[0] == nr and abs(t[0] - tr) < 1e-15
    for f in range(4):
        assert np.abs(got[0][f] - ref[f]).mean() < 1e-10 * np.abs(ref[f]).mean(), f


def test_mixed_run_single_solver_matches_one_instance_batch():
    """Many mixed-precision steps of a four-quadrant problem whose tiles next
    to the discontinuities defer rows to the FP64 indicator: the single-grid
    kernel (compile-time form of the paper's configuration) and the batch
    kernel (run-time switches, tile table) take the same steps and agree to
    FP32 rounding (a lost, doubled or misplaced tile or row would not)."""
    nx, ny = 150, 120
    p = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=nx, ny=ny, lin_w=W2D, bc=(1, 1, 1, 1))
    U0 = W.quadrant_2d(W.quadrant_states(31), 0.37, 0.61, 0, 1, 0, 1, nx, ny)
    cfg = cfg_from(p, hw.FP32_IND64)
    s = hw.Solver(cfg)
    s.set_state(U0)
    t1, n1 = s.advance(0.05)
    one = s.get_state(device=False)
    s.close()
    b = hw.Batch([cfg])
    b.set_state(torch.from_numpy(b.pack([U0.astype(np.float32).astype(np.float64)])).cuda())
    t2, n2 = b.advance([0.05])
    two = b.unpack(b.get_state())[0]
    b.close()
    assert n1 == n2[0] and n1 >= 12
    for f in range(4):
        scale = np.abs(one[f]).max()
        assert np.abs(one[f] - two[f]).max() <= 1e-3 * scale, f
        assert np.abs(one[f] - two[f]).mean() <= 1e-5 * scale, f
