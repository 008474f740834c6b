"""Multi-GPU partitioning of the hot path (host logic; every arithmetic step
of the scheme runs in libhweno's kernels).

Two natural splits:

* independent problems of a batch are dealt to ranks by cells
  (`shard_by_cells`): no exchange at all;
* one 2D grid is cut into slabs of rows, one per rank (`Slab2D`).  A cell's
  update in one RK stage reads a stencil of radius 1 around each of the cells
  whose reconstructions meet at its faces, so its dependency radius is 2
  cells per stage (Sec. 2.2 Step 1 stencils and the fluxes of Eq.
  2D-semi-discrete-scheme-uniform).  Each rank therefore holds its rows plus
  2 halo rows on each side that has a neighbour, runs every stage on that
  local grid, and before the next stage replaces its halo rows with the
  neighbours' edge rows of the stage output (one exchange per RK stage).
  The global Lax-Friedrichs constants alpha are the maxima over every cell
  of the grid: one max-allreduce per step (every rank then forms the same
  dt).  Halo rows of the local grid are computed too, from partly wrong
  stencils at the local grid's edge, and are overwritten by the exchange
  before anything reads them.

The slab driver (`SlabGroup`) is written against two small interfaces, an
executor that runs a local grid's stages (`CudaSlab`: a libhweno solver) and
a communicator (`TorchComm`: torch.distributed point-to-point and
all-reduce, NCCL across GPUs, gloo on CPU; `LocalComm`: ranks held by one
process).  Several ranks may live in one process: their halo rows then move
by device copies.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

HALO = 2   # dependency radius of one RK stage, in cells


def shard_by_cells(cells, world: int) -> list:
    """Deal instances to `world` ranks so that the ranks' total cells are
    balanced: largest first, each to the rank with the fewest cells so far
    (ties to the lower rank).  Returns each rank's instance indices in
    ascending order; every instance appears exactly once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(cells)), key=lambda k: (-int(cells[k]), k))
    load = [0] * world
    out = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(k)
        load[r] += int(cells[k])
    return [sorted(v) for v in out]


def split_rows(ny: int, world: int) -> list:
    """Row ranges [(r0, r1)] of `world` slabs of an ny-row grid, sizes
    differing by at most one (the first ny % world slabs one row taller)."""
    base, extra = divmod(ny, world)
    out, r0 = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((r0, r0 + n))
        r0 += n
    return out


@dataclass
class Slab2D:
    """Rank `rank`'s slab of an nx x ny grid split along y into `world`
    slabs of at least HALO rows each."""
    nx: int
    ny: int
    world: int
    rank: int
    periodic_y: bool = False
    rows: tuple = field(init=False)

    def __post_init__(self):
        self.rows = split_rows(self.ny, self.world)[self.rank]
        if min(b - a for a, b in split_rows(self.ny, self.world)) < HALO:
            raise ValueError(f"every slab needs at least {HALO} rows")

    @property
    def own(self) -> int:
        return self.rows[1] - self.rows[0]

    @property
    def lo(self):
        """Rank below (None at a non-periodic bottom side)."""
        if self.world == 1:
            return None
        if self.rank > 0:
            return self.rank - 1
        return self.world - 1 if self.periodic_y else None

    @property
    def hi(self):
        if self.world == 1:
            return None
        if self.rank < self.world - 1:
            return self.rank + 1
        return 0 if self.periodic_y else None

    @property
    def halo_lo(self) -> int:
        return HALO if self.lo is not None else 0

    @property
    def halo_hi(self) -> int:
        return HALO if self.hi is not None else 0

    @property
    def ny_local(self) -> int:
        return self.own + self.halo_lo + self.halo_hi

    def global_rows(self) -> list:
        """Global row index of every local row (wrapped on periodic grids)."""
        r0 = self.rows[0] - self.halo_lo
        return [(r0 + k) % self.ny for k in range(self.ny_local)]

    def local_config(self, cfg, bc_halo: int = 1):
        """The local grid's config: ny_local rows covering the global rows
        of global_rows(); a side with a neighbour takes `bc_halo` (any rule:
        its ghost cells only feed halo rows, which the exchange overwrites)."""
        y0, y1 = local_extent(cfg.ylo, cfg.yhi, cfg.ny, self.rows[0] - self.halo_lo, self.ny_local)
        bc = list(cfg.bc)
        if self.lo is not None:
            bc[2] = bc_halo
        if self.hi is not None:
            bc[3] = bc_halo
        return replace(cfg, ny=self.ny_local, ylo=y0, yhi=y1, bc=tuple(bc))

    def messages(self):
        """The exchange of one stage output, from this rank's side:
        sends [(peer, tag, first local row)] and receives [(peer, tag, first
        local row)], HALO rows each, in the order every rank posts them
        (sends up, sends down, receives from below, receives from above) so
        that point-to-point matching in posting order pairs them even when
        both neighbours are one rank.  Tag 1 travels up, tag 0 down."""
        sends, recvs = [], []
        top = self.halo_lo + self.own - HALO
        if self.hi is not None:
            sends.append((self.hi, 1, top))
        if self.lo is not None:
            sends.append((self.lo, 0, self.halo_lo))
        if self.lo is not None:
            recvs.append((self.lo, 1, 0))
        if self.hi is not None:
            recvs.append((self.hi, 0, self.halo_lo + self.own))
        return sends, recvs


def local_extent(ylo: float, yhi: float, ny: int, first_row: int, n: int) -> tuple:
    """(y0, y1) of n rows starting at global row `first_row` of the grid
    [ylo, yhi] with ny rows.  The kernels form the spacing from the extent,
    so y1 is chosen, where one exists within a few hundred ulps, such that
    (y1 - y0) / n rounds to exactly the global spacing (yhi - ylo) / ny;
    then every flux rounds as on the whole grid.  Always so for dyadic
    spacings (y0 and y0 + n dy exact); otherwise, when the ulp of y1 exceeds
    n ulps of the spacing, the local spacing can be one ulp off and the split
    run agrees with the whole grid to round-off only."""
    import math
    dy = (yhi - ylo) / ny
    y0 = ylo + first_row * dy
    c = y0 + n * dy
    u = math.ulp(c)
    for k in range(256):
        for cand in ((c,) if k == 0 else (c + k * u, c - k * u)):
            if (cand - y0) / n == dy:
                return y0, cand
    return y0, c


def cfl_dt(cfg, ax: float, ay: float) -> float:
    """The CFL time step of Sec. 2.2 (dt = CFL / (ax/hx + ay/hy), hx = dx or
    dx^(5/3) for order studies), the device control's formula on the host."""
    dx = (cfg.xhi - cfg.xlo) / cfg.nx
    dy = (cfg.yhi - cfg.ylo) / cfg.ny
    r53 = cfg.dt_rule == 1
    hx = dx ** (5.0 / 3.0) if r53 else dx
    hy = dy ** (5.0 / 3.0) if r53 else dy
    rate = ax / hx + ay / hy
    return cfg.cfl / rate if rate > 0.0 else float("inf")


# ------------------------------------------------------------- executors
class CudaSlab:
    """A slab's local grid on the GPU: a libhweno solver driven stage by
    stage (hweno_stage), its rows moved by hweno_rows."""

    def __init__(self, hw, torch, cfg, U_local, theta=None, p_threshold=0.5):
        self.hw, self.torch = hw, torch
        self.cfg = cfg
        self.s = hw.Solver(cfg)
        if theta is not None:
            hw.hweno_indicator_load(self.s.h, theta, p_threshold)
        self.s.set_state(U_local)
        self.dtype = torch.float64 if cfg.precision == hw.FP64 else torch.float32

    @property
    def stream(self) -> int:
        return self.s.stream

    def alpha_update(self):
        return self.hw.hweno_alpha_update(self.s.h)

    def stage(self, k, dt, ax, ay):
        self.hw.hweno_stage(self.s.h, k, dt, ax, ay)

    def get_rows(self, buffer, row0, n):
        t = self.torch.empty((self.cfg.nfields, n, self.cfg.nx), dtype=self.dtype, device="cuda")
        self.hw.hweno_rows(self.s.h, buffer, row0, t, False)
        self.torch.cuda.ExternalStream(self.s.stream).synchronize()
        return t

    def set_rows(self, buffer, row0, t):
        self.hw.hweno_rows(self.s.h, buffer, row0, t.contiguous(), True)
        self.torch.cuda.ExternalStream(self.s.stream).synchronize()

    def empty_rows(self, n):
        return self.torch.empty((self.cfg.nfields, n, self.cfg.nx), dtype=self.dtype, device="cuda")

    def state(self):
        return self.s.get_state()

    def close(self):
        self.s.close()


# ---------------------------------------------------------- communicators
class LocalComm:
    """Every rank in this process: no messages leave it."""

    def allreduce_max(self, values):
        return list(values)

    def exchange(self, sends, recvs):
        if sends or recvs:
            raise RuntimeError("LocalComm has no remote ranks")


class TorchComm:
    """torch.distributed: max-allreduce of alpha and point-to-point halo
    messages (batch_isend_irecv, posted in the order of Slab2D.messages)."""

    def __init__(self, device=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        self.device = device if device is not None else ("cuda" if dist.get_backend() == "nccl" else "cpu")

    def allreduce_max(self, values):
        t = self.torch.tensor([float(v) for v in values], dtype=self.torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return [float(x) for x in t.tolist()]

    def exchange(self, sends, recvs):
        """sends / recvs: [(peer, tag, tensor)] in posting order."""
        ops = [self.dist.P2POp(self.dist.isend, t, peer, tag=tag) for peer, tag, t in sends]
        ops += [self.dist.P2POp(self.dist.irecv, t, peer, tag=tag) for peer, tag, t in recvs]
        if ops:
            for req in self.dist.batch_isend_irecv(ops):
                req.wait()


# ----------------------------------------------------------------- driver
class SlabGroup:
    """The slabs of one grid that this process holds (`slabs` and their
    `execs`, one executor per slab), advanced together step by step: the
    global alpha (max over every slab of every process), the CFL dt from it,
    then per stage: every slab's stage, then the halo exchange of that
    stage's output."""

    # buffer written by each stage: 1 -> stage-1 output, 2 -> stage-2, 3 -> state
    OUT = {1: 1, 2: 2, 3: 0}

    def __init__(self, cfg, slabs, execs, comm, cfl_cfg=None):
        self.cfg = cfg                 # the global grid's config (dt, spacing)
        self.slabs = list(slabs)
        self.execs = list(execs)
        self.comm = comm
        self.by_rank = {s.rank: k for k, s in enumerate(self.slabs)}
        self.t = 0.0
        self.steps = 0
        self.alpha = None
        self.exchange_ms = 0.0

    def global_alpha(self):
        ax = ay = 0.0
        for e in self.execs:
            a, b = e.alpha_update()
            ax, ay = max(ax, a), max(ay, b)
        ax, ay = self.comm.allreduce_max([ax, ay])
        return ax, ay

    def exchange(self, buffer):
        remote_sends, remote_recvs, pending = [], [], []
        for k, (slab, ex) in enumerate(zip(self.slabs, self.execs)):
            sends, recvs = slab.messages()
            for peer, tag, row0 in sends:
                t = ex.get_rows(buffer, row0, HALO)
                if peer in self.by_rank:
                    # a rank of this process: write straight into its halo
                    q = self.by_rank[peer]
                    dst = [r for p, g, r in self.slabs[q].messages()[1] if p == slab.rank and g == tag]
                    self.execs[q].set_rows(buffer, dst[0], t)
                else:
                    remote_sends.append((peer, tag, t))
            for peer, tag, row0 in recvs:
                if peer not in self.by_rank:
                    t = ex.empty_rows(HALO)
                    remote_recvs.append((peer, tag, t))
                    pending.append((k, row0, t))
        self.comm.exchange(remote_sends, remote_recvs)
        for k, row0, t in pending:
            self.execs[k].set_rows(buffer, row0, t)

    def step(self, t_final=float("inf")):
        if self.alpha is None:
            self.alpha = self.global_alpha()
        ax, ay = self.alpha
        dt = cfl_dt(self.cfg, ax, ay)
        if not dt > 0.0:
            raise RuntimeError(f"non-physical state: alpha = ({ax}, {ay})")
        if self.t + dt >= t_final:
            dt = t_final - self.t
        for k in (1, 2, 3):
            for e in self.execs:
                e.stage(k, dt, ax, ay)
            self.exchange(self.OUT[k])
        tn = self.t + dt
        finite = t_final < float("inf")
        self.t = t_final if (finite and t_final - tn <= 1e-15 * abs(t_final)) else tn
        self.steps += 1
        self.alpha = self.global_alpha()
        return dt

    def advance(self, t_final=float("inf"), max_steps=2 ** 31 - 1):
        n = 0
        while self.t < t_final and n < max_steps:
            self.step(t_final)
            n += 1
        return self.t, n


# ------------------------------------------------------------ bench helpers
@dataclass
class BenchSlab:
    """One rank's slab of a weak-scaling grid: `world` copies of a single-GPU
    state stacked along y (each rank owns one copy's rows; neighbouring
    copies meet at a state jump and exchange halos like any other rows)."""
    cfg_global: object
    slab: Slab2D
    U_copy: object   # numpy [nf, ny, nx] of one copy

    @staticmethod
    def for_rank(cfg, U_copy, world, rank):
        ny = cfg.ny
        g = replace(cfg, ny=ny * world, ylo=cfg.ylo, yhi=cfg.ylo + (cfg.yhi - cfg.ylo) * world)
        return BenchSlab(g, Slab2D(cfg.nx, ny * world, world, rank, periodic_y=False), U_copy)

    def local_state(self):
        import numpy as np
        ny = self.U_copy.shape[1]
        rows = [r % ny for r in self.slab.global_rows()]
        return np.ascontiguousarray(self.U_copy[:, rows, :])


def time_slab_arm(hw, torch, bs: BenchSlab, steps, warmup, local, theta=None):
    """Warm-up and timed steps of one rank's slab (CUDA events on the
    solver's stream around the timed steps, stage kernels profiled)."""
    import torch.distributed as dist
    cfg_local = bs.slab.local_config(bs.cfg_global)
    U = torch.from_numpy(bs.local_state())
    ex = CudaSlab(hw, torch, cfg_local, U.cuda(), theta)
    grp = SlabGroup(bs.cfg_global, [bs.slab], [ex], TorchComm())
    grp.advance(max_steps=warmup)
    ex.s.set_state(U.cuda())
    grp = SlabGroup(bs.cfg_global, [bs.slab], [ex], TorchComm())
    ex.s.set_profiling(True)
    torch.cuda.synchronize()
    dist.barrier()
    stream = torch.cuda.ExternalStream(ex.stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    grp.advance(max_steps=steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    stage_ms, stage_n, launches = ex.s.profile()
    ex.s.set_profiling(False)
    o0 = bs.slab.halo_lo
    rho = ex.state()[0][o0:o0 + bs.slab.own].double().clone()
    ex.close()
    return {"ms": ms, "stage_ms": stage_ms / max(stage_n, 1), "stage_launches": stage_n,
            "launches": 3 * steps, "clocks": {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"],
                                             "samples": 0},
            "rho": rho, "smooth_fraction": None, "cells_local": cfg_local.nx * cfg_local.ny}


def e2e_slab(hw, torch, bs: BenchSlab, steps):
    """End to end on one rank's slab: per step its local state host -> device,
    one step (three stages, three exchanges), the state device -> host."""
    import time
    cfg_local = bs.slab.local_config(bs.cfg_global)
    dtype = torch.float64 if cfg_local.precision == hw.FP64 else torch.float32
    a = torch.from_numpy(bs.local_state()).to(dtype).pin_memory()
    b = torch.empty_like(a).pin_memory()
    ex = CudaSlab(hw, torch, cfg_local, a.cuda())
    grp = SlabGroup(bs.cfg_global, [bs.slab], [ex], TorchComm())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    src, dst = a, b
    for _ in range(steps):
        hw.hweno_set_state(ex.s.h, src)
        grp.alpha = None
        grp.step()
        hw.hweno_get_state(ex.s.h, dst)
        src, dst = dst, src
    el = time.perf_counter() - t0
    ex.close()
    nbytes = a.numel() * a.element_size()
    return {"units": bs.slab.own * cfg_local.nx * 3 * steps, "seconds": el, "unit": "cell-updates/s",
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "what": "per step and rank: the local state host->device from pinned memory, one SSP-RK3 step with "
                    "its halo exchanges, the local state device->host"}
