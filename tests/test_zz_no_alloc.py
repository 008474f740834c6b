"""The allocation-free 1D step (hweno_step_1d_noalloc) against the regular
step (hweno_step) and the oracle, through the C ABI.

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


def _problem(eq, n, charwise=1):
    euler = eq == oracle.EQ_EULER
    return oracle.Problem(dim=1, equation=eq, nx=n, xlo=0, xhi=2, charwise=charwise,
                          bc=(oracle.BC_OUTFLOW,) * 4 if euler else (oracle.BC_PERIODIC,) * 4)


CASES = [
    (oracle.EQ_EULER, 1, 997, hw.FP64),
    (oracle.EQ_EULER, 1, 300, hw.FP32),
    (oracle.EQ_EULER, 1, 301, hw.FP32_IND64),
    (oracle.EQ_EULER, 0, 259, hw.FP32),
    (oracle.EQ_EULER, 0, 260, hw.FP64),
    (oracle.EQ_BURGERS, 1, 64, hw.FP64),
    (oracle.EQ_ADVECTION, 1, 181, hw.FP64),
    (oracle.EQ_ADVECTION, 1, 180, hw.FP32),
    (oracle.EQ_ADVECTION, 1, 179, hw.FP32_IND64),
]


@pytest.mark.parametrize("eq,charwise,n,prec", CASES)
def test_noalloc_step_matches_regular_step_twice(eq, charwise, n, prec):
    prob = _problem(eq, n, charwise)
    euler = eq == oracle.EQ_EULER
    cfg = cfg_from(prob, prec)
    U0 = W.random_state(1, (n,), seed=n, euler=euler)
    dtype = torch.float64 if prec == hw.FP64 else torch.float32
    tol = 1e-12 if prec == hw.FP64 else 1e-6
    # two calls in a row: the second starts from the first one's output
    U_dev = torch.from_numpy(U0).to(dtype).cuda().contiguous()
    dx = 2.0 / n
    steps = [(0.3 * dx / 2.5, 2.5), (0.25 * dx / 3.0, 3.0)]  # CFL 0.3 and 0.25
    ref = U0.astype(np.float64 if prec == hw.FP64 else np.float32)
    ref_or = U0.astype(np.float64)
    for dt, alpha in steps:
        out = torch.full_like(U_dev, float("nan"))
        hw.hweno_step_1d_noalloc(cfg, U_dev, out, dt, alpha)
        torch.cuda.synchronize()
        assert bool(torch.isfinite(out).all()), "non-finite output"
        ref = _regular_step(cfg, np.ascontiguousarray(ref), dt, alpha)
        got = out.cpu().numpy()
        assert plane_rel_err(got, ref) <= tol
        if prec == hw.FP64:
            ref_or = oracle.step(prob, ref_or, dt, alpha)
            assert np.isfinite(ref_or).all()
            assert plane_rel_err(got, ref_or) <= 1e-12
        U_dev = out


@pytest.mark.parametrize("eq,prec", [(oracle.EQ_EULER, hw.FP64), (oracle.EQ_ADVECTION, hw.FP64),
                                     (oracle.EQ_EULER, hw.FP32_IND64)])
def test_noalloc_step_in_place(eq, prec):
    """U_in == U_out: the step overwrites its input, which is only read
    before the last stage writes the same cell."""
    n = 413
    prob = _problem(eq, n)
    cfg = cfg_from(prob, prec)
    U0 = W.random_state(1, (n,), seed=77, euler=eq == oracle.EQ_EULER)
    dtype = torch.float64 if prec == hw.FP64 else torch.float32
    U = torch.from_numpy(U0).to(dtype).cuda().contiguous()
    ref_or = U0.astype(np.float64)
    ref = U0.astype(np.float64 if prec == hw.FP64 else np.float32)
    dx = 2.0 / n
    for dt, alpha in [(0.3 * dx / 2.5, 2.5), (0.25 * dx / 2.8, 2.8)]:
        hw.hweno_step_1d_noalloc(cfg, U, U, dt, alpha)
        torch.cuda.synchronize()
        got = U.cpu().numpy()
        assert np.isfinite(got).all()
        ref = _regular_step(cfg, np.ascontiguousarray(ref), dt, alpha)
        ref_or = oracle.step(prob, ref_or, dt, alpha)
        assert np.isfinite(ref_or).all()
        if prec == hw.FP64:
            assert plane_rel_err(got, ref_or) <= 1e-12
            assert plane_rel_err(got, ref) <= 1e-12
        else:
            assert plane_rel_err(got, ref) <= 1e-6
            # one mixed-precision step of rough data stays within FP32 conditioning of the oracle
            assert plane_rel_err(got[:3], ref_or[:3]) <= 1e-4


def test_noalloc_rejects_oversize_and_bad_args():
    cfg = hw.Config(dim=1, nx=10_000_000, equation=hw.EQ_EULER)
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(hw.HwenoError) as ei:
        hw.hweno_step_1d_noalloc(cfg, x, x, 1e-3, 1.0)
    assert ei.value.status == hw.HWENO_ERR_ARG and "limited to" in str(ei.value)
    # the advertised limit is exact: that many cells are accepted, one more is not
    limit = int(str(ei.value).split("(")[-1].split(" cells")[0])
    assert 100_000 < limit < 10_000_000
    big = torch.zeros(6 * limit, dtype=torch.float64, device="cuda")
    big[:limit] = 1.0                   # rho = 1, m = 0, E = 2.5: a valid state at rest
    big[2 * limit:3 * limit] = 2.5
    hw.hweno_step_1d_noalloc(hw.Config(dim=1, nx=limit, equation=hw.EQ_EULER, bc=(hw.BC_PERIODIC,) * 4),
                             big, big, 0.0, 0.0)
    torch.cuda.synchronize()
    with pytest.raises(hw.HwenoError):
        hw.hweno_step_1d_noalloc(hw.Config(dim=1, nx=limit + 1, equation=hw.EQ_EULER), big, big, 0.0, 0.0)
    del big
    with pytest.raises(hw.HwenoError):
        hw.hweno_step_1d_noalloc(hw.Config(dim=2, nx=8, ny=8, lin_w=(0.99, 0.0025, 0.0025, 0.0025, 0.0025)),
                                 x, x, 1e-3, 1.0)
    with pytest.raises(hw.HwenoError):
        hw.hweno_step_1d_noalloc(hw.Config(dim=1, nx=8), x, x, -1.0, 1.0)
