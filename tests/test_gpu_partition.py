"""The slab decomposition on the GPU through the C ABI (hweno_stage,
hweno_rows, hweno_alpha_update): a 2D grid split into slabs of rows held by
one process (their halo rows move by device copies; no kernel waits on
another) advances bit for bit like the same grid as one slab, and the one-slab
run matches the oracle."""
import numpy as np
import pytest

import oracle
from paper_2607_24325_b300 import partition as PT
from paper_2607_24325_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_24325_b300 import hweno as hw  # noqa: E402

W2D = (0.99, 0.0025, 0.0025, 0.0025, 0.0025)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _run(cfg, U, world, steps, theta=None):
    slabs = [PT.Slab2D(cfg.nx, cfg.ny, world, r, periodic_y=cfg.bc[2] == hw.BC_PERIODIC) for r in range(world)]
    execs = []
    for s in slabs:
        Ul = torch.from_numpy(np.ascontiguousarray(U[:, s.global_rows(), :])).cuda()
        execs.append(PT.CudaSlab(hw, torch, s.local_config(cfg), Ul, theta))
    grp = PT.SlabGroup(cfg, slabs, execs, PT.LocalComm())
    for _ in range(steps):
        grp.step()
    out = np.concatenate([e.state().cpu().numpy()[:, s.halo_lo:s.halo_lo + s.own, :]
                          for s, e in zip(slabs, execs)], axis=1)
    for e in execs:
        e.close()
    return out, grp.t


@pytest.mark.parametrize("prec", [hw.FP64, hw.FP32_IND64, hw.FP32])
@pytest.mark.parametrize("world,periodic", [(3, False), (2, True)])
def test_slabs_equal_one_grid_bitwise(prec, world, periodic):
    n = 96   # [0, 0.75] / 96 and [0, 0.625] / 80: dyadic spacing 1/128, exact in every slab
    bc = (hw.BC_OUTFLOW,) * 4 if not periodic else (hw.BC_PERIODIC,) * 4
    cfg = hw.Config(dim=2, nx=80, ny=n, xhi=0.625, yhi=0.75, equation=hw.EQ_EULER, lin_w=W2D, bc=bc,
                    precision=prec)
    U = W.quadrant_2d(W.quadrant_states(5), 0.3, 0.4, 0.0, 0.625, 0.0, 0.75, 80, n)
    one, t1 = _run(cfg, U, 1, 4)
    split, t2 = _run(cfg, U, world, 4)
    assert t1 == t2
    assert np.isfinite(one).all()
    assert np.array_equal(one, split)


def test_one_slab_matches_the_oracle():
    n = 32
    cfg = hw.Config(dim=2, nx=n, ny=n, xhi=2.0, yhi=2.0, equation=hw.EQ_EULER, lin_w=W2D,
                    bc=(hw.BC_PERIODIC,) * 4)
    U = W.cells_2d(W.euler_smooth_2d(0.0), 0, 2, 0, 2, n, n)
    got, _ = _run(cfg, U, 2, 3)
    prob = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=n, ny=n, xhi=2.0, yhi=2.0, lin_w=W2D)
    R = U.copy()
    for _ in range(3):
        ax, ay = oracle.alpha(prob, R)
        R = oracle.step(prob, R, PT.cfl_dt(cfg, ax, ay), ax, ay)
    err = max(np.abs(got[f] - R[f]).max() / np.abs(R[f]).max() for f in range(R.shape[0]))
    assert err <= 1e-11


def test_stage_order_and_rows_are_checked():
    cfg = hw.Config(dim=2, nx=16, ny=16, equation=hw.EQ_EULER, lin_w=W2D, bc=(hw.BC_OUTFLOW,) * 4)
    s = hw.Solver(cfg)
    s.set_state(W.quadrant_2d(W.quadrant_states(5), 0.5, 0.5, 0, 1, 0, 1, 16, 16))
    with pytest.raises(hw.HwenoError):
        hw.hweno_stage(s.h, 2, 1e-3, 1.0, 1.0)          # stage 2 before stage 1
    hw.hweno_stage(s.h, 1, 1e-3, 2.0, 2.0)
    with pytest.raises(hw.HwenoError):
        hw.hweno_stage(s.h, 2, 2e-3, 2.0, 2.0)          # another dt inside the step
    hw.hweno_stage(s.h, 2, 1e-3, 2.0, 2.0)
    hw.hweno_stage(s.h, 3, 1e-3, 2.0, 2.0)
    t, _ = hw.hweno_get_time(s.h)
    assert t == 1e-3
    rows = torch.empty((cfg.nfields, 2, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(hw.HwenoError):
        hw.hweno_rows(s.h, 0, 15, rows, False)           # rows 15..16 of a 16-row grid
    with pytest.raises(hw.HwenoError):
        hw.hweno_rows(s.h, 3, 0, rows, False)            # no buffer 3
    hw.hweno_rows(s.h, 0, 14, rows, False)
    torch.cuda.synchronize()
    assert np.array_equal(rows.cpu().numpy(), s.get_state(device=False)[:, 14:16, :])
    s.close()


def test_batch_profiling_counts_stage_launches():
    cfgs = [hw.Config(dim=1, nx=n, equation=hw.EQ_EULER, bc=(hw.BC_OUTFLOW,) * 4) for n in (40, 97, 300)]
    b = hw.Batch(cfgs)
    b.set_state(b.pack([W.riemann_1d((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.5, 0.0, 1.0, c.nx) for c in cfgs]))
    b.set_profiling(True)
    b.advance(1e30, max_steps=3)
    ms, n, launches = b.profile()
    b.set_profiling(False)
    b.close()
    assert n == 9 and launches == 15 and ms > 0.0
