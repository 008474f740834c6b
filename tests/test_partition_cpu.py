"""The multi-GPU partitioning's host logic on CPU (paper_2607_24325_b300/
partition.py): cell-balanced sharding of batches, and the slab decomposition
of one 2D grid -- halo exchange of 2 rows per RK stage, one max-allreduce of
alpha per step -- run by gloo ranks with the oracle as each slab's stage
executor.  The split run must equal the single-grid oracle run bit for bit:
every cell's stage update reads only cells within 2 rows, which the exchange
supplies exactly, and alpha is the same maximum."""
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from paper_2607_24325_b300 import partition as PT
from paper_2607_24325_b300 import workloads as W

torch = pytest.importorskip("torch")
import torch.distributed as dist           # noqa: E402
import torch.multiprocessing as mp         # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
W2D = (0.99, 0.0025, 0.0025, 0.0025, 0.0025)


# ----------------------------------------------------------------- sharding
def test_shard_by_cells_complete_disjoint_balanced():
    rng = np.random.default_rng(3)
    cells = [int(x) for x in np.exp(rng.uniform(np.log(256), np.log(8192), 256))]
    for world in (1, 2, 3, 4, 8):
        parts = PT.shard_by_cells(cells, world)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(len(cells)))
        loads = [sum(cells[k] for k in p) for p in parts]
        # greedy largest-first: the spread is at most the largest instance
        assert max(loads) - min(loads) <= max(cells)
        assert all(p == sorted(p) for p in parts)
    assert PT.shard_by_cells([5, 1, 1, 1, 1, 1], 2) == [[0], [1, 2, 3, 4, 5]]


def test_local_extent_keeps_the_spacing():
    """Dyadic spacings are reproduced exactly; others exactly where the ulp
    of the extent allows it, else to within the extent's ulp over n."""
    rng = np.random.default_rng(0)
    exact = 0
    for _ in range(2000):
        ny = int(rng.integers(4, 5000))
        lo, hi = sorted(rng.uniform(-3, 7, 2))
        r0 = int(rng.integers(-2, ny))
        n = int(rng.integers(2, ny + 4))
        y0, y1 = PT.local_extent(lo, hi, ny, r0, n)
        dy = (hi - lo) / ny
        assert y0 == lo + r0 * dy
        got = (y1 - y0) / n
        exact += got == dy
        assert abs(got - dy) <= 2 * np.spacing(abs(y1)) / n + 2 * np.spacing(dy)
    assert exact > 0
    for ny, r0, n in [(4096 * 4, 4094, 4100), (13, 3, 6), (1024, 1000, 26)]:
        hi = ny / 8.0
        y0, y1 = PT.local_extent(0.0, hi, ny, r0, n)
        assert (y1 - y0) / n == 0.125 and y0 == r0 * 0.125


def test_split_rows_and_messages():
    assert PT.split_rows(10, 3) == [(0, 4), (4, 7), (7, 10)]
    s = PT.Slab2D(8, 10, 3, 1)
    assert (s.lo, s.hi, s.halo_lo, s.halo_hi, s.ny_local) == (0, 2, 2, 2, 7)
    assert s.global_rows() == [2, 3, 4, 5, 6, 7, 8]
    sends, recvs = s.messages()
    assert sends == [(2, 1, 3), (0, 0, 2)] and recvs == [(0, 1, 0), (2, 0, 5)]
    b = PT.Slab2D(8, 10, 3, 0)           # bottom slab, non-periodic: no halo below
    assert (b.lo, b.halo_lo, b.ny_local) == (None, 0, 6)
    p = PT.Slab2D(8, 10, 2, 0, periodic_y=True)
    assert (p.lo, p.hi) == (1, 1) and p.global_rows() == [8, 9, 0, 1, 2, 3, 4, 5, 6]
    with pytest.raises(ValueError):
        PT.Slab2D(8, 3, 2, 0)


# --------------------------------------------- the oracle as a slab executor
class OracleSlab:
    """A local grid advanced stage by stage with the oracle's operator and
    the SSP-RK3 combinations of Step 4 in the oracle's own order."""

    def __init__(self, prob, U):
        self.prob = prob
        self.U = np.array(U, dtype=np.float64)
        self.buf = {0: self.U}
        self.nc = prob.ncomp

    def alpha_update(self):
        return oracle.alpha(self.prob, self.buf[0])

    def stage(self, k, dt, ax, ay):
        nc = self.nc
        if k == 1:
            self.U0 = self.buf[0].copy()
            L, self.H0 = oracle.operator(self.prob, self.U0, ax, ay)
            A = np.empty_like(self.U0)
            A[:nc] = self.U0[:nc] + dt * L[:nc]
            A[nc:] = self.H0 + dt * L[nc:]
            self.buf[1] = A
        else:
            src = self.buf[k - 1]
            L, Hs = oracle.operator(self.prob, src, ax, ay)
            out = np.empty_like(src)
            if k == 2:
                out[:nc] = 0.75 * self.U0[:nc] + 0.25 * (src[:nc] + dt * L[:nc])
                out[nc:] = 0.75 * self.H0 + 0.25 * (Hs + dt * L[nc:])
                self.buf[2] = out
            else:
                out[:nc] = self.U0[:nc] / 3.0 + 2.0 / 3.0 * (src[:nc] + dt * L[:nc])
                out[nc:] = self.H0 / 3.0 + 2.0 / 3.0 * (Hs + dt * L[nc:])
                self.buf[0] = out

    def get_rows(self, buffer, row0, n):
        return torch.from_numpy(np.ascontiguousarray(self.buf[buffer][:, row0:row0 + n, :]))

    def empty_rows(self, n):
        return torch.empty((self.buf[0].shape[0], n, self.buf[0].shape[2]), dtype=torch.float64)

    def set_rows(self, buffer, row0, t):
        self.buf[buffer][:, row0:row0 + t.shape[1], :] = t.numpy()


def _problem(ny, periodic, equation=oracle.EQ_EULER):
    bc = (oracle.BC_PERIODIC,) * 4 if periodic else (oracle.BC_PERIODIC, oracle.BC_PERIODIC, oracle.BC_OUTFLOW,
                                                      oracle.BC_OUTFLOW)
    # dyadic spacing (1/8): every slab's extent reproduces it exactly
    return oracle.Problem(dim=2, equation=equation, nx=12, ny=ny, xhi=1.5, yhi=ny / 8.0, lin_w=W2D, bc=bc)


def _initial(prob):
    if prob.equation == oracle.EQ_EULER:
        f = W.euler_smooth_2d(0.0)
        U = W.cells_2d(f, prob.xlo, prob.xhi, prob.ylo, prob.yhi, prob.nx, prob.ny)
        rng = np.random.default_rng(1)
        U[:4] *= 1.0 + 0.05 * rng.uniform(-1, 1, size=U[:4].shape)   # rough enough to move the weights
        return U
    return W.random_state(2, (prob.ny, prob.nx), seed=2)


def _reference(prob, U, steps):
    """The single grid: alpha, the CFL dt and one oracle step, `steps` times."""
    cfg = _cfg(prob)
    for _ in range(steps):
        ax, ay = oracle.alpha(prob, U)
        U = oracle.step(prob, U, PT.cfl_dt(cfg, ax, ay), ax, ay)
    return U


class _Cfg:
    """The fields of the global config the slab driver reads."""

    def __init__(self, prob):
        self.nx, self.ny = prob.nx, prob.ny
        self.xlo, self.xhi, self.ylo, self.yhi = prob.xlo, prob.xhi, prob.ylo, prob.yhi
        self.cfl, self.dt_rule = prob.cfl, prob.dt_rule


def _cfg(prob):
    return _Cfg(prob)


def _local(prob, slab, U):
    rows = slab.global_rows()
    bc = list(prob.bc)
    if slab.lo is not None:
        bc[2] = oracle.BC_OUTFLOW
    if slab.hi is not None:
        bc[3] = oracle.BC_OUTFLOW
    y0, y1 = PT.local_extent(prob.ylo, prob.yhi, prob.ny, slab.rows[0] - slab.halo_lo, slab.ny_local)
    lp = oracle.Problem(**{**prob.__dict__, "ny": slab.ny_local, "ylo": y0, "yhi": y1, "bc": tuple(bc)})
    return lp, np.ascontiguousarray(U[:, rows, :])


def _run_slabs(prob, U, ranks, world, comm, steps):
    slabs = [PT.Slab2D(prob.nx, prob.ny, world, r, periodic_y=prob.bc[2] == oracle.BC_PERIODIC) for r in ranks]
    execs = [OracleSlab(*_local(prob, s, U)) for s in slabs]
    grp = PT.SlabGroup(_cfg(prob), slabs, execs, comm)
    for _ in range(steps):
        grp.step()
    return [(s, e.buf[0][:, s.halo_lo:s.halo_lo + s.own, :]) for s, e in zip(slabs, execs)]


@pytest.mark.parametrize("periodic,world", [(True, 3), (False, 4)])
def test_slabs_in_one_process_equal_the_single_grid(periodic, world):
    prob = _problem(13, periodic)
    U = _initial(prob)
    ref = _reference(prob, U, 3)
    for s, own in _run_slabs(prob, U, list(range(world)), world, PT.LocalComm(), 3):
        assert np.array_equal(own, ref[:, s.rows[0]:s.rows[1], :]), s.rank


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, periodic, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = _problem(11, periodic)
        U = _initial(prob)
        (s, own), = _run_slabs(prob, U, [rank], world, PT.TorchComm(device="cpu"), 3)
        out[rank] = (s.rows, own.copy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("periodic", [True, False])
def test_two_gloo_ranks_equal_the_single_grid(periodic):
    """world_size 2 over gloo: with periodic sides both neighbours of a rank
    are the other rank (the tags and the posting order keep the two halo
    messages apart)."""
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), periodic, out), nprocs=world, join=True)
        got = dict(out)
    prob = _problem(11, periodic)
    ref = _reference(prob, _initial(prob), 3)
    assert sorted(got) == [0, 1]
    for r in range(world):
        rows, own = got[r]
        assert np.array_equal(own, ref[:, rows[0]:rows[1], :]), r


def test_a_missing_exchange_is_detected():
    """Without the halo exchange the split run differs from the single grid
    (the equality above is not vacuous)."""
    prob = _problem(13, True)
    U = _initial(prob)
    ref = _reference(prob, U, 2)

    class NoExchange(PT.SlabGroup):
        def exchange(self, buffer):
            pass
    slabs = [PT.Slab2D(prob.nx, prob.ny, 3, r, periodic_y=True) for r in range(3)]
    execs = [OracleSlab(*_local(prob, s, U)) for s in slabs]
    grp = NoExchange(_cfg(prob), slabs, execs, PT.LocalComm())
    grp.step()
    grp.step()
    diff = max(np.abs(e.buf[0][:, s.halo_lo:s.halo_lo + s.own, :] - ref[:, s.rows[0]:s.rows[1], :]).max()
               for s, e in zip(slabs, execs))
    assert diff > 1e-8


def test_bench_slabs_of_stacked_copies_equal_the_stacked_grid():
    """The bench's weak-scaling layout: `world` copies of one state stacked
    along y, one copy's rows per rank (BenchSlab).  Each rank's local state
    and config come from the copy alone; advanced with the oracle as the
    executor, the slabs equal the explicitly stacked grid run as one."""
    from dataclasses import dataclass

    @dataclass
    class Cfg:                     # the fields of hw.Config the slab set-up reads
        nx: int
        ny: int
        xlo: float = 0.0
        xhi: float = 1.5
        ylo: float = 0.0
        yhi: float = 1.0
        cfl: float = 0.6
        dt_rule: int = 0
        bc: tuple = (oracle.BC_PERIODIC, oracle.BC_PERIODIC, oracle.BC_OUTFLOW, oracle.BC_OUTFLOW)
    world, nx, ny = 3, 12, 8
    cfg = Cfg(nx=nx, ny=ny, yhi=ny / 8.0)
    prob1 = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=nx, ny=ny, xhi=1.5, yhi=ny / 8.0, lin_w=W2D,
                           bc=cfg.bc)
    U = _initial(prob1)
    stacked = oracle.Problem(**{**prob1.__dict__, "ny": ny * world, "yhi": ny * world / 8.0})
    ref = _reference(stacked, np.concatenate([U] * world, axis=1), 2)
    slabs, execs = [], []
    for r in range(world):
        bs = PT.BenchSlab.for_rank(cfg, U, world, r)
        assert bs.cfg_global.ny == ny * world and bs.slab.own == ny
        lc = bs.slab.local_config(bs.cfg_global)
        lp = oracle.Problem(**{**prob1.__dict__, "ny": lc.ny, "ylo": lc.ylo, "yhi": lc.yhi, "bc": tuple(lc.bc)})
        slabs.append(bs.slab)
        execs.append(OracleSlab(lp, bs.local_state()))
    grp = PT.SlabGroup(PT.BenchSlab.for_rank(cfg, U, world, 0).cfg_global, slabs, execs, PT.LocalComm())
    grp.step()
    grp.step()
    for s, e in zip(slabs, execs):
        assert np.array_equal(e.buf[0][:, s.halo_lo:s.halo_lo + s.own, :], ref[:, s.rows[0]:s.rows[1], :]), s.rank
