"""The mixed precision's FP32 screen skips the FP64 smoothness indicator only
where it provably cannot change a weight (every a_m at most 2^-24, so 1 + a_m
rounds to 1 in FP32).  So the library and a build with the screen off
(libhweno_noscreen.so: every lane of every row takes the FP64 indicator)
must give the same output bits: operator application and eight steps on
five kinds of 2D state and three of 1D, with both smoothness-indicator
forms, and a batch of three 2D problems (the batched kernel).  The library is
chosen at load time, so each build runs in a child process."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import hashlib, sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_2607_24325_b300 import hweno as hw, workloads as W, indicator as IND
W2D = (0.99, 0.0025, 0.0025, 0.0025, 0.0025)
cases = []
for sm in (hw.BETA_MOMENT, hw.BETA_TYPICAL):
    n = 128
    cases.append((f"quadrant_{sm}", hw.Config(dim=2, nx=n, ny=n, equation=hw.EQ_EULER, lin_w=W2D, bc=(1,) * 4,
                  precision=hw.FP32_IND64, smoothness=sm),
                  W.quadrant_2d(W.quadrant_states(2024), 0.5, 0.5, 0, 1, 0, 1, n, n)))
    cfg, U = IND.shock_entropy_problem(3, 96, hw.FP32_IND64)
    cfg.smoothness = sm
    cases.append((f"shock_entropy_{sm}", cfg, U))
    # a finer member of the family: smooth entropy waves whose weight
    # deviations sit near the screen's bound
    cfg, U = IND.shock_entropy_problem(11, 256, hw.FP32_IND64)
    cfg.smoothness = sm
    cases.append((f"shock_entropy_fine_{sm}", cfg, U))
    Bd = W.dmr_boundary()
    cases.append((f"dmr_{sm}", hw.Config(dim=2, nx=160, ny=40, xlo=0, xhi=4, ylo=0, yhi=1, equation=hw.EQ_EULER,
                  lin_w=W2D, bc=Bd["bc"], bc_state=Bd["bc_state"], bc_state2=Bd["bc_state2"],
                  bc_param=Bd["bc_param"], precision=hw.FP32_IND64, smoothness=sm), W.dmr_2d(160, 40)))
    cases.append((f"smooth_{sm}", hw.Config(dim=2, nx=96, ny=96, xlo=0, xhi=2, ylo=0, yhi=2, equation=hw.EQ_EULER,
                  lin_w=W2D, precision=hw.FP32_IND64, smoothness=sm),
                  W.cells_2d(W.euler_smooth_2d(0.0), 0, 2, 0, 2, 96, 96)))
    # 1D: a shock tube, smooth Euler data and a fine sine for advection
    cases.append((f"sod1d_{sm}", hw.Config(dim=1, nx=400, equation=hw.EQ_EULER, bc=(1,) * 4,
                  precision=hw.FP32_IND64, smoothness=sm),
                  W.riemann_1d((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.5, 0.0, 1.0, 400)))
    cases.append((f"smooth1d_{sm}", hw.Config(dim=1, nx=1000, xlo=0, xhi=2, equation=hw.EQ_EULER,
                  precision=hw.FP32_IND64, smoothness=sm), W.cells_1d(W.euler_smooth_1d(0.0), 0, 2, 1000)))
    cases.append((f"advection1d_{sm}", hw.Config(dim=1, nx=4096, xlo=0, xhi=2, equation=hw.EQ_ADVECTION,
                  precision=hw.FP32_IND64, smoothness=sm), W.sine_1d_cells(4096)))
for name, cfg, U in cases:
    s = hw.Solver(cfg)
    s.set_state(U)
    L, D = s.apply_operator(3.0, 2.5)
    s.advance(1e30, max_steps=8)
    G = s.get_state(device=False)
    h = hashlib.sha256()
    for a in (L.cpu().numpy(), D.cpu().numpy(), G):
        h.update(np.ascontiguousarray(a).tobytes())
    print("HASH", name, h.hexdigest())
    s.close()
# the batched 2D kernel: three four-quadrant problems of uneven sizes in one launch per stage
sizes = [(96, 70), (61, 128), (150, 33)]
cfgs = [hw.Config(dim=2, nx=nx, ny=ny, equation=hw.EQ_EULER, lin_w=W2D, bc=(1,) * 4, precision=hw.FP32_IND64)
        for nx, ny in sizes]
b = hw.Batch(cfgs)
b.set_state(b.pack([W.quadrant_2d(W.quadrant_states(40 + k), 0.45, 0.55, 0, 1, 0, 1, nx, ny)
                    for k, (nx, ny) in enumerate(sizes)]))
L, D = b.apply_operator([(3.0, 2.5)] * 3)
b.advance(1e30, max_steps=8)
h = hashlib.sha256()
for a in (L.cpu().numpy(), D.cpu().numpy(), b.get_state(device=False)):
    h.update(np.ascontiguousarray(a).tobytes())
print("HASH", "batch2d", h.hexdigest())
b.close()
'''


def _hashes(env_extra):
    env = dict(os.environ, **env_extra)
    p = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], capture_output=True, text=True,
                       env=env, timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    return dict(l.split()[1:3] for l in p.stdout.splitlines() if l.startswith("HASH "))


def test_screen_changes_no_output_bit():
    import __graft_entry__
    __graft_entry__.build()
    screened = _hashes({})
    full = _hashes({"HWENO_NOSCREEN": "1"})
    assert len(screened) == 17 and screened == full, (screened, full)
