"""The allocation-free 1D step (hweno_step_1d_noalloc) against the regular
step (hweno_step), through the C ABI.

Some callers of the library cannot allocate device memory when they need a
step (their host gave the device memory budget to its own pool, or they run
in a loop that must not pay cudaMalloc's implicit synchronisation).  This
entry point keeps its working memory in a fixed device array inside the
library instead.  This file runs last so that a failure here never hides the
other tests, and it passes both alone in a fresh process and after them.
"""
import numpy as np
import pytest

import oracle
from paper_2607_24325_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_24325_b300 import hweno as hw  # noqa: E402
from helpers import cfg_from, plane_rel_err     # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _regular_step(cfg, U, dt, alpha):
    s = hw.Solver(cfg)
    s.set_state(U)
    s.step(dt, alpha)
    out = s.get_state(device=False)
    s.close()
    return out


@pytest.mark.parametrize("eq,n,prec", [(oracle.EQ_EULER, 997, hw.FP64), (oracle.EQ_BURGERS, 64, hw.FP64),
                                       (oracle.EQ_EULER, 300, hw.FP32)])
def test_noalloc_step_matches_regular_step_twice(eq, n, prec):
    euler = eq == oracle.EQ_EULER
    prob = oracle.Problem(dim=1, equation=eq, nx=n, xlo=0, xhi=2,
                          bc=(oracle.BC_OUTFLOW,) * 4 if euler else (oracle.BC_PERIODIC,) * 4)
    cfg = cfg_from(prob, prec)
    U0 = W.random_state(1, (n,), seed=n, euler=euler)
    dtype = torch.float64 if prec == hw.FP64 else torch.float32
    tol = 1e-12 if prec == hw.FP64 else 1e-6
    # two calls in a row: the second starts from the first one's output
    U_dev = torch.from_numpy(U0).to(dtype).cuda().contiguous()
    steps = [(1e-3, 2.5), (7e-4, 3.0)]
    ref = U0.astype(np.float64 if prec == hw.FP64 else np.float32)
    for dt, alpha in steps:
        out = torch.empty_like(U_dev)
        hw.hweno_step_1d_noalloc(cfg, U_dev, out, dt, alpha)
        torch.cuda.synchronize()
        ref = _regular_step(cfg, np.ascontiguousarray(ref), dt, alpha)
        got = out.cpu().numpy()
        assert plane_rel_err(got, ref) <= tol
        U_dev = out


def test_noalloc_rejects_oversize_and_bad_args():
    cfg = hw.Config(dim=1, nx=10_000_000, equation=hw.EQ_EULER)
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(hw.HwenoError) as ei:
        hw.hweno_step_1d_noalloc(cfg, x, x, 1e-3, 1.0)
    assert ei.value.status == hw.HWENO_ERR_ARG and "limited to" in str(ei.value)
    with pytest.raises(hw.HwenoError):
        hw.hweno_step_1d_noalloc(hw.Config(dim=2, nx=8, ny=8, lin_w=(0.99, 0.0025, 0.0025, 0.0025, 0.0025)),
                                 x, x, 1e-3, 1.0)
    with pytest.raises(hw.HwenoError):
        hw.hweno_step_1d_noalloc(hw.Config(dim=1, nx=8), x, x, -1.0, 1.0)
