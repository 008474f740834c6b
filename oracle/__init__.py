"""ctypes binding of the plain FP64 CPU oracle (``hweno_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is a slow, serial, obviously correct
restatement of the fifth-order derivative-based HWENO scheme with unified
stencils (arxiv 2607.24325, Sec. 2.1, Sec. 2.2, Remark 1, Appendix A).  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may
import it; the CUDA library never does, and the two share no code.

Arrays are numpy float64 in the layout documented in ``hweno_oracle.h``:
``U[f][j][i]`` with ``f = d*nc + k`` (d = 0 cell averages, 1 x-derivative
moments, 2 y-derivative moments), x fastest, no ghost cells.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hweno_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

EQ_ADVECTION, EQ_BURGERS, EQ_EULER = 0, 1, 2
BC_PERIODIC, BC_OUTFLOW, BC_REFLECT, BC_INFLOW, BC_SPLIT, BC_SHOCK = 0, 1, 2, 3, 4, 5
DT_CFL, DT_CFL_DX53 = 0, 1
BETA_MOMENT, BETA_TYPICAL = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "hweno_oracle.h"))
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("equation", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
        ("xlo", C.c_double), ("xhi", C.c_double), ("ylo", C.c_double), ("yhi", C.c_double),
        ("adv_x", C.c_double), ("adv_y", C.c_double), ("gamma_gas", C.c_double),
        ("lin_w", C.c_double * 5), ("eps", C.c_double),
        ("weight_pow", C.c_int), ("charwise", C.c_int), ("linear_weights", C.c_int),
        ("dt_rule", C.c_int), ("bc", C.c_int * 4), ("bc_state", (C.c_double * 4) * 4),
        ("cfl", C.c_double), ("bc_state2", (C.c_double * 4) * 4), ("bc_param", (C.c_double * 2) * 4),
        ("t", C.c_double), ("smoothness", C.c_int),
    ]


@dataclass
class Problem:
    """Problem statement u_t + div F(u) = 0 on a uniform grid (Sec. 2)."""
    dim: int = 1
    equation: int = EQ_ADVECTION
    nx: int = 16
    ny: int = 1
    xlo: float = 0.0
    xhi: float = 1.0
    ylo: float = 0.0
    yhi: float = 1.0
    adv_x: float = 1.0
    adv_y: float = 1.0
    gamma_gas: float = 1.4
    lin_w: tuple = (0.995, 0.0025, 0.0025)
    eps: float = 1e-8
    weight_pow: int = 1  # beta + eps (2D tables pin 1; the 2D text prints beta^2)
    charwise: int = 1
    linear_weights: int = 0
    dt_rule: int = DT_CFL
    bc: tuple = (BC_PERIODIC,) * 4
    bc_state: list = field(default_factory=lambda: [[0.0] * 4 for _ in range(4)])
    cfl: float = 0.6
    smoothness: int = BETA_MOMENT  # BETA_TYPICAL: the Jiang-Shu integral indicator
    bc_state2: list = field(default_factory=lambda: [[0.0] * 4 for _ in range(4)])  # BC_SHOCK second state
    bc_param: list = field(default_factory=lambda: [[0.0, 0.0] for _ in range(4)])  # BC_SPLIT / BC_SHOCK
    t: float = 0.0  # time of the state (time-dependent boundaries)

    @property
    def ncomp(self) -> int:
        if self.equation != EQ_EULER:
            return 1
        return 3 if self.dim == 1 else 4

    @property
    def nfields(self) -> int:
        return self.ncomp * (self.dim + 1)

    @property
    def shape(self) -> tuple:
        ny = self.ny if self.dim == 2 else 1
        return (self.nfields, ny, self.nx) if self.dim == 2 else (self.nfields, self.nx)

    @property
    def dx(self) -> float:
        return (self.xhi - self.xlo) / self.nx

    @property
    def dy(self) -> float:
        return (self.yhi - self.ylo) / self.ny

    def _c(self) -> _Problem:
        s = _Problem()
        s.dim, s.equation, s.nx = self.dim, self.equation, self.nx
        s.ny = self.ny if self.dim == 2 else 1
        s.xlo, s.xhi, s.ylo, s.yhi = self.xlo, self.xhi, self.ylo, self.yhi
        s.adv_x, s.adv_y, s.gamma_gas = self.adv_x, self.adv_y, self.gamma_gas
        w = list(self.lin_w) + [0.0] * (5 - len(self.lin_w))
        for k in range(5):
            s.lin_w[k] = w[k]
        s.eps = self.eps
        s.weight_pow = self.weight_pow
        s.charwise, s.linear_weights, s.dt_rule = self.charwise, self.linear_weights, self.dt_rule
        for k in range(4):
            s.bc[k] = self.bc[k]
            for c in range(4):
                s.bc_state[k][c] = self.bc_state[k][c]
        s.cfl = self.cfl
        s.smoothness = self.smoothness
        for k in range(4):
            for c in range(4):
                s.bc_state2[k][c] = self.bc_state2[k][c]
            for c in range(2):
                s.bc_param[k][c] = self.bc_param[k][c]
        s.t = self.t
        return s


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        pp = C.POINTER(_Problem)
        L.or_operator.argtypes = [pp, dp, C.c_double, C.c_double, dp, dp]
        L.or_alpha.argtypes = [pp, dp, dp, dp]
        L.or_dt.argtypes = [pp, C.c_double, C.c_double]
        L.or_dt.restype = C.c_double
        L.or_step.argtypes = [pp, dp, C.c_double, C.c_double, C.c_double]
        L.or_run.argtypes = [pp, dp, C.c_double, C.c_int, dp, C.POINTER(C.c_int)]
        L.or_coef_maps_1d.argtypes = [dp, dp, dp]
        L.or_coef_maps_2d.argtypes = [dp, dp]
        L.or_recon_cell_1d.argtypes = [pp, dp, C.c_double, dp]
        L.or_recon_cell_2d.argtypes = [pp, dp, C.c_double, C.c_double, dp]
        L.or_euler_jacobian.argtypes = [C.c_int, C.c_int, dp, C.c_double, dp]
        L.or_euler_eigen.argtypes = [C.c_int, C.c_int, dp, C.c_double, dp, dp]
        L.or_weight_deviation.argtypes = [pp, dp, dp]
        L.or_padded_state.argtypes = [pp, dp, dp]
        L.or_flop_count.argtypes = [C.c_int]
        L.or_flop_count.restype = C.c_longlong
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _state(prob: Problem, U) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    if U.size != int(np.prod(prob.shape)):
        raise ValueError(f"state has {U.size} values, expected shape {prob.shape}")
    return U.reshape(prob.shape).copy()


def operator(prob: Problem, U, ax: float, ay: float = 0.0):
    """One application of the spatial operator: returns (L, dhat)."""
    U = _state(prob, U)
    L = np.zeros_like(U)
    nd = prob.ncomp * prob.dim
    dh = np.zeros((nd,) + U.shape[1:])
    ps = prob._c()
    rc = lib().or_operator(C.byref(ps), _ptr(U), ax, ay, _ptr(L), _ptr(dh))
    if rc:
        raise RuntimeError(f"or_operator failed ({rc})")
    return L, dh


def alpha(prob: Problem, U):
    U = _state(prob, U)
    ax, ay = C.c_double(), C.c_double()
    ps = prob._c()
    if lib().or_alpha(C.byref(ps), _ptr(U), C.byref(ax), C.byref(ay)):
        raise RuntimeError("or_alpha failed")
    return ax.value, ay.value


def dt(prob: Problem, ax: float, ay: float = 0.0) -> float:
    ps = prob._c()
    return lib().or_dt(C.byref(ps), ax, ay)


def step(prob: Problem, U, dt_: float, ax: float, ay: float = 0.0) -> np.ndarray:
    U = _state(prob, U)
    ps = prob._c()
    if lib().or_step(C.byref(ps), _ptr(U), dt_, ax, ay):
        raise RuntimeError("or_step failed")
    return U


def run(prob: Problem, U, t_final: float, max_steps: int = 10**9):
    """Advance to t_final; returns (U, t, steps)."""
    U = _state(prob, U)
    t = C.c_double()
    n = C.c_int()
    ps = prob._c()
    rc = lib().or_run(C.byref(ps), _ptr(U), t_final, min(max_steps, 2**31 - 1), C.byref(t), C.byref(n))
    if rc:
        raise RuntimeError(f"or_run failed ({rc}) at t={t.value} after {n.value} steps")
    return U, t.value, n.value


def coef_maps_1d():
    G0, G1, G2 = np.zeros(25), np.zeros(4), np.zeros(4)
    lib().or_coef_maps_1d(_ptr(G0), _ptr(G1), _ptr(G2))
    return G0.reshape(5, 5), G1.reshape(2, 2), G2.reshape(2, 2)


def coef_maps_2d():
    G0, Gm = np.zeros(15 * 17), np.zeros(36)
    lib().or_coef_maps_2d(_ptr(G0), _ptr(Gm))
    return G0.reshape(15, 17), Gm.reshape(4, 3, 3)


def recon_cell_1d(prob: Problem, inp, dx: float) -> dict:
    a = np.ascontiguousarray(inp, dtype=np.float64)
    out = np.zeros(11)
    ps = prob._c()
    lib().or_recon_cell_1d(C.byref(ps), _ptr(a), dx, _ptr(out))
    return {"uL": out[0], "uR": out[1], "dL": out[2], "dR": out[3], "vhat": out[4],
            "omega": out[5:8].copy(), "beta": out[8:11].copy()}


def recon_cell_2d(prob: Problem, q, dx: float, dy: float) -> dict:
    a = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros(48)
    ps = prob._c()
    lib().or_recon_cell_2d(C.byref(ps), _ptr(a), dx, dy, _ptr(out))
    return {"faces": out[:36].reshape(4, 3, 3).copy(), "vhat": out[36], "what": out[37],
            "omega": out[38:43].copy(), "beta": out[43:48].copy()}


def euler_jacobian(dim: int, direction: int, U, gamma_gas: float = 1.4) -> np.ndarray:
    n = 3 if dim == 1 else 4
    u = np.ascontiguousarray(U, dtype=np.float64)
    A = np.zeros(n * n)
    lib().or_euler_jacobian(dim, direction, _ptr(u), gamma_gas, _ptr(A))
    return A.reshape(n, n)


def euler_eigen(dim: int, direction: int, U, gamma_gas: float = 1.4):
    n = 3 if dim == 1 else 4
    u = np.ascontiguousarray(U, dtype=np.float64)
    R, L = np.zeros(n * n), np.zeros(n * n)
    lib().or_euler_eigen(dim, direction, _ptr(u), gamma_gas, _ptr(R), _ptr(L))
    return R.reshape(n, n), L.reshape(n, n)


def weight_deviation(prob: Problem, U) -> np.ndarray:
    """Per cell max |omega_m/gamma_m - 1| of the plain scheme's weights (label source)."""
    U = _state(prob, U)
    dev = np.zeros(U.shape[1:])
    ps = prob._c()
    if lib().or_weight_deviation(C.byref(ps), _ptr(U), _ptr(dev)):
        raise RuntimeError("or_weight_deviation failed")
    return dev


def padded_state(prob: Problem, U) -> np.ndarray:
    U = _state(prob, U)
    shape = (prob.nfields, prob.ny + 4, prob.nx + 4) if prob.dim == 2 else (prob.nfields, prob.nx + 4)
    out = np.zeros(shape)
    ps = prob._c()
    if lib().or_padded_state(C.byref(ps), _ptr(U), _ptr(out)):
        raise RuntimeError("or_padded_state failed")
    return out


def flop_count(reset: bool = False) -> int:
    """The oracle's running count of the method's flops (plain evaluation of
    each formula, charged for the grid's own cells and faces)."""
    return int(lib().or_flop_count(1 if reset else 0))
