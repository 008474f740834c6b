"""The index-checked build (libhweno_checked.so, -DHWENO_CHECKED): every
shared- and global-memory index of the stage kernels is tested against its
buffer's extent, and a bad one is recorded and skipped instead of touching
memory.  Runs ragged, below-a-tile, batched and time-dependent-boundary cases
of every precision through it and requires that no access was skipped, and
that the checked build still computes the scheme (operator parity with the
oracle).  The library is chosen at load time, so the cases run in a child
process with HWENO_CHECKED=1."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import ctypes as C, json, sys
import numpy as np
import torch
sys.path.insert(0, ROOT); sys.path.insert(0, ROOT + "/tests")
import oracle
from paper_2607_24325_b300 import hweno as hw, workloads as W
from helpers import cfg_from, plane_rel_err
assert hw.CHECKED and hw.LIB_PATH.endswith("libhweno_checked.so")
L = hw.load()
for n in ("hweno_check_stage2d", "hweno_check_stage1d", "hweno_check_probe"):
    getattr(L, n).argtypes = [C.c_void_p, C.c_int]
L.hweno_check_selftest.argtypes = [C.c_void_p]
def word(n):
    w = (C.c_uint * 4)()
    assert getattr(L, n)(w, 1) == 0
    return list(w)
out = {}
for n in ("hweno_check_stage2d", "hweno_check_stage1d", "hweno_check_probe"):
    word(n)                                           # start from zero
ok = (C.c_int * 2)()
assert L.hweno_check_selftest(ok) == 0
out["selftest"] = [ok[0], ok[1]]
out["probe"] = word("hweno_check_probe")
W2D = (0.99, 0.0025, 0.0025, 0.0025, 0.0025)
a = list(W.prim_to_cons_2d(1.3, 0.4, -0.2, 1.1))
b = list(W.prim_to_cons_2d(0.7, -0.1, 0.3, 0.6))
z2 = [0.0, 0.0]
probs = [
    oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=37, ny=23, xlo=0.0, xhi=1.3, ylo=-1.0, yhi=0.5,
                   bc=(0, 0, 1, 1), lin_w=W2D),
    oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=64, ny=61, bc=(2, 2, 3, 1), bc_state=[a, a, a, a], lin_w=W2D),
    oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=5, ny=40, xlo=-0.2, xhi=0.3, bc=(3, 1, 2, 2),
                   bc_state=[b, b, b, b], lin_w=W2D),
    oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=96, ny=31, xlo=0.0, xhi=2.0, bc=(4, 1, 1, 5),
                   bc_state=[a, a, a, a], bc_state2=[b, b, b, b], bc_param=[[0.4, 0.0], z2, z2, [0.7, 3.0]], lin_w=W2D),
    oracle.Problem(dim=2, equation=oracle.EQ_BURGERS, nx=33, ny=62, lin_w=W2D),
]
errs = []
for k, p in enumerate(probs):
    U = W.random_state(2, (p.ny, p.nx), seed=200 + k, euler=p.equation == oracle.EQ_EULER, moment_scale=0.3)
    for prec in (hw.FP64, hw.FP32, hw.FP32_IND64):
        s = hw.Solver(cfg_from(p, prec))
        s.set_state(U)
        Lg, Dg = s.apply_operator(2.0, 1.5)
        if prec == hw.FP64:
            Lr, Dr = oracle.operator(p, U, 2.0, 1.5)
            errs.append(max(plane_rel_err(Lg.cpu().numpy(), Lr), plane_rel_err(Dg.cpu().numpy(), Dr)))
        s.advance(1e30, max_steps=5)
        s.close()
# many steps of a shock problem in the mixed mode: deferred rows, packed FP64 items
q = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=150, ny=120, lin_w=W2D, bc=(1, 1, 1, 1))
s = hw.Solver(cfg_from(q, hw.FP32_IND64))
s.set_state(W.quadrant_2d(W.quadrant_states(31), 0.37, 0.61, 0, 1, 0, 1, 150, 120))
hw.hweno_autotune(s.h, reps=1)
s.advance(0.03)
s.close()
# a 2D batch of uneven sizes and a 1D batch, both precisions
bt = hw.Batch([cfg_from(p, hw.FP32_IND64) for p in probs[:4]])
bt.set_state(torch.from_numpy(bt.pack([W.random_state(2, (p.ny, p.nx), seed=300 + k, euler=True, moment_scale=0.3)
                                       for k, p in enumerate(probs[:4])])).cuda())
bt.advance([0.01] * 4)
bt.close()
one = [oracle.Problem(dim=1, equation=oracle.EQ_EULER, nx=n, bc=(1, 1, 1, 1)) for n in (5, 31, 97, 300)]
for prec in (hw.FP64, hw.FP32):
    b1 = hw.Batch([cfg_from(p, prec) for p in one])
    b1.set_state(b1.pack([W.riemann_1d((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.5, 0.0, 1.0, p.nx) for p in one]))
    b1.advance([0.05] * len(one))
    b1.close()
p1 = oracle.Problem(dim=1, equation=oracle.EQ_ADVECTION, nx=64, xlo=0.0, xhi=2.0, bc=(0, 0, 0, 0))
s = hw.Solver(cfg_from(p1, hw.FP64))
s.set_state(W.sine_1d_cells(64))
s.advance(0.5)
s.close()
torch.cuda.synchronize()
out["stage2d"] = word("hweno_check_stage2d")
out["stage1d"] = word("hweno_check_stage1d")
out["parity"] = max(errs)
print("RESULT " + json.dumps(out))
'''


def test_checked_build_skips_no_access():
    import __graft_entry__
    __graft_entry__.build()
    env = dict(os.environ, HWENO_CHECKED="1")
    p = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], capture_output=True, text=True,
                       env=env, timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    line = [l for l in p.stdout.splitlines() if l.startswith("RESULT ")][-1]
    r = json.loads(line[len("RESULT "):])
    assert r["selftest"] == [1, 0]
    assert r["probe"] == [1, 99, 7, 5]               # the check records what it should
    assert r["stage2d"][0] == 0, r["stage2d"]        # [count, site, index, extent] of the first bad access
    assert r["stage1d"][0] == 0, r["stage1d"]
    assert r["parity"] < 1e-12
