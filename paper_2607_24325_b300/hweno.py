"""Thin Python binding of libhweno (``include/hweno.h``).

Argument marshalling only: every step of the scheme runs in the CUDA
kernels behind the C ABI.  The module-level functions carry the C entry
points' names; ``Solver`` and ``Batch`` are small conveniences over them.
Device buffers are torch CUDA tensors; host buffers are numpy arrays (or CPU
tensors).  If ``libhweno.so`` is missing this module raises -- there is no
fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# HWENO_CHECKED=1 in the environment loads the index-checked build
# (libhweno_checked.so: the same entry points plus include/hweno_checked.h's);
# HWENO_NOSCREEN=1 the build without the mixed precision's FP32 screen
# (libhweno_noscreen.so, for the test that the screen changes no output bit).
CHECKED = os.environ.get("HWENO_CHECKED") == "1"
NOSCREEN = os.environ.get("HWENO_NOSCREEN") == "1"
LIB_PATH = os.path.join(_HERE, "libhweno_checked.so" if CHECKED else
                        ("libhweno_noscreen.so" if NOSCREEN else "libhweno.so"))

HWENO_OK, HWENO_ERR_ARG, HWENO_ERR_CUDA, HWENO_ERR_NONPHYSICAL = 0, 1, 2, 3
HWENO_ERR_TIMEOUT, HWENO_ERR_OOM, HWENO_ERR_STATE = 4, 5, 6
EQ_ADVECTION, EQ_BURGERS, EQ_EULER = 0, 1, 2
BC_PERIODIC, BC_OUTFLOW, BC_REFLECT, BC_INFLOW, BC_SPLIT, BC_SHOCK = 0, 1, 2, 3, 4, 5
FP64, FP32, FP32_IND64 = 0, 1, 2
DT_CFL, DT_CFL_DX53 = 0, 1
BETA_MOMENT, BETA_TYPICAL = 0, 1

# every extern "C" symbol include/hweno.h declares
EXPORTS = (
    "hweno_last_error", "hweno_version", "hweno_create", "hweno_destroy", "hweno_stream",
    "hweno_shape", "hweno_set_state", "hweno_get_state", "hweno_alpha", "hweno_apply_operator",
    "hweno_step", "hweno_advance", "hweno_set_profiling", "hweno_profile", "hweno_peak_fma",
    "hweno_selftest_convert", "hweno_selftest_rcp64",
    "hweno_batch_create", "hweno_batch_destroy",
    "hweno_batch_stream", "hweno_batch_layout", "hweno_batch_set_state", "hweno_batch_get_state",
    "hweno_batch_advance", "hweno_batch_apply_operator", "hweno_step_1d_noalloc",
    "hweno_batch_set_profiling", "hweno_batch_profile", "hweno_stage", "hweno_rows", "hweno_alpha_update",
    "hweno_indicator_train", "hweno_train_permutation",
    "hweno_indicator_features", "hweno_indicator_labels", "hweno_indicator_load", "hweno_indicator_off",
    "hweno_indicator_mask", "hweno_mlp_create", "hweno_mlp_destroy", "hweno_mlp_set_params",
    "hweno_mlp_get_params", "hweno_mlp_gradient", "hweno_mlp_train_step", "hweno_mlp_mean_loss",
    "hweno_mlp_predict", "hweno_project", "hweno_autotune", "hweno_batch_autotune",
    "hweno_get_time", "hweno_set_time",
)
MLP_NPARAM = 3521


class hweno_train_opts(C.Structure):
    _fields_ = [("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_double), ("delta", C.c_double),
                ("pos_weight", C.c_double), ("seed", C.c_ulonglong)]


class hweno_config(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
        ("xlo", C.c_double), ("xhi", C.c_double), ("ylo", C.c_double), ("yhi", C.c_double),
        ("equation", C.c_int), ("adv_x", C.c_double), ("adv_y", C.c_double), ("gamma_gas", C.c_double),
        ("lin_w", C.c_double * 5), ("eps", C.c_double), ("weight_pow", C.c_int),
        ("charwise", C.c_int), ("linear_weights", C.c_int), ("cfl", C.c_double), ("dt_rule", C.c_int),
        ("bc", C.c_int * 4), ("bc_state", (C.c_double * 4) * 4), ("precision", C.c_int),
        ("smoothness", C.c_int), ("bc_state2", (C.c_double * 4) * 4), ("bc_param", (C.c_double * 2) * 4),
    ]


@dataclass
class Config:
    """Python mirror of ``hweno_config`` with the paper's defaults."""
    dim: int = 1
    nx: int = 16
    ny: int = 1
    xlo: float = 0.0
    xhi: float = 1.0
    ylo: float = 0.0
    yhi: float = 1.0
    equation: int = EQ_ADVECTION
    adv_x: float = 1.0
    adv_y: float = 1.0
    gamma_gas: float = 1.4
    lin_w: tuple = (0.995, 0.0025, 0.0025)
    eps: float = 1e-8
    weight_pow: int = 1
    charwise: int = 1
    linear_weights: int = 0
    cfl: float = 0.6
    dt_rule: int = DT_CFL
    bc: tuple = (BC_PERIODIC,) * 4
    bc_state: list = field(default_factory=lambda: [[0.0] * 4 for _ in range(4)])
    precision: int = FP64
    smoothness: int = BETA_MOMENT
    bc_state2: list = field(default_factory=lambda: [[0.0] * 4 for _ in range(4)])  # BC_SHOCK second state
    bc_param: list = field(default_factory=lambda: [[0.0, 0.0] for _ in range(4)])  # BC_SPLIT / BC_SHOCK

    @property
    def ncomp(self) -> int:
        return 1 if self.equation != EQ_EULER else (3 if self.dim == 1 else 4)

    @property
    def nfields(self) -> int:
        return self.ncomp * (self.dim + 1)

    @property
    def ncells(self) -> int:
        return self.nx * (self.ny if self.dim == 2 else 1)

    def to_c(self) -> hweno_config:
        c = hweno_config()
        c.dim, c.nx, c.ny = self.dim, self.nx, self.ny if self.dim == 2 else 1
        c.xlo, c.xhi, c.ylo, c.yhi = self.xlo, self.xhi, self.ylo, self.yhi
        c.equation, c.adv_x, c.adv_y, c.gamma_gas = self.equation, self.adv_x, self.adv_y, self.gamma_gas
        w = list(self.lin_w) + [0.0] * (5 - len(self.lin_w))
        for k in range(5):
            c.lin_w[k] = w[k]
        c.eps, c.weight_pow, c.charwise, c.linear_weights = self.eps, self.weight_pow, self.charwise, self.linear_weights
        c.cfl, c.dt_rule, c.precision = self.cfl, self.dt_rule, self.precision
        c.smoothness = self.smoothness
        for k in range(4):
            for q in range(4):
                c.bc_state2[k][q] = self.bc_state2[k][q]
            for q in range(2):
                c.bc_param[k][q] = self.bc_param[k][q]
        for k in range(4):
            c.bc[k] = self.bc[k]
            for q in range(4):
                c.bc_state[k][q] = self.bc_state[k][q]
        return c


class HwenoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libhweno status {status}: {msg}")
        self.status = status


_lib = None
U0_FN = C.CFUNCTYPE(None, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p)


def load():
    """Load libhweno.so (never a fallback: raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp, cp = C.c_void_p, C.POINTER(hweno_config)
    L.hweno_last_error.restype = C.c_char_p
    L.hweno_version.restype = C.c_char_p
    L.hweno_create.argtypes = [cp, vp, C.POINTER(vp)]
    L.hweno_destroy.argtypes = [vp]
    L.hweno_destroy.restype = None
    L.hweno_stream.argtypes = [vp]
    L.hweno_stream.restype = vp
    L.hweno_shape.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_size_t)]
    L.hweno_set_state.argtypes = [vp, vp, C.c_int]
    L.hweno_get_state.argtypes = [vp, vp, C.c_int]
    L.hweno_alpha.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.hweno_apply_operator.argtypes = [vp, C.c_double, C.c_double, vp, vp]
    L.hweno_step.argtypes = [vp, C.c_double, C.c_double, C.c_double]
    L.hweno_advance.argtypes = [vp, C.c_double, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    L.hweno_set_profiling.argtypes = [vp, C.c_int]
    L.hweno_profile.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
    L.hweno_peak_fma.argtypes = [C.c_int, C.POINTER(C.c_double)]
    L.hweno_selftest_convert.argtypes = [vp, vp, vp, vp, C.c_int]
    L.hweno_selftest_rcp64.argtypes = [vp, vp, C.c_int]
    L.hweno_batch_create.argtypes = [C.c_int, cp, vp, C.POINTER(vp)]
    L.hweno_batch_destroy.argtypes = [vp]
    L.hweno_batch_destroy.restype = None
    L.hweno_batch_stream.argtypes = [vp]
    L.hweno_batch_stream.restype = vp
    L.hweno_batch_layout.argtypes = [vp, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
    L.hweno_batch_set_state.argtypes = [vp, vp, C.c_int]
    L.hweno_batch_get_state.argtypes = [vp, vp, C.c_int]
    L.hweno_batch_advance.argtypes = [vp, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_double),
                                      C.POINTER(C.c_int)]
    L.hweno_batch_apply_operator.argtypes = [vp, C.POINTER(C.c_double), vp, vp]
    L.hweno_batch_set_profiling.argtypes = [vp, C.c_int]
    L.hweno_stage.argtypes = [vp, C.c_int, C.c_double, C.c_double, C.c_double]
    L.hweno_indicator_train.argtypes = [vp, vp, C.c_longlong, C.POINTER(hweno_train_opts), C.POINTER(C.c_float),
                                        C.POINTER(C.c_float), C.POINTER(C.c_double), vp]
    L.hweno_train_permutation.argtypes = [C.c_ulonglong, C.c_int, C.c_longlong, C.POINTER(C.c_int)]
    L.hweno_train_permutation.restype = None
    L.hweno_rows.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp, C.c_int]
    L.hweno_alpha_update.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.hweno_batch_profile.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                                      C.POINTER(C.c_longlong)]
    L.hweno_step_1d_noalloc.argtypes = [cp, vp, vp, C.c_double, C.c_double, vp]
    fp, ip = C.POINTER(C.c_float), C.POINTER(C.c_int)
    L.hweno_indicator_features.argtypes = [vp, vp]
    L.hweno_indicator_labels.argtypes = [vp, vp]
    L.hweno_indicator_load.argtypes = [vp, fp, C.c_int, C.c_double]
    L.hweno_indicator_off.argtypes = [vp]
    L.hweno_indicator_mask.argtypes = [vp, vp, vp]
    L.hweno_mlp_create.argtypes = [C.c_int, vp, C.POINTER(vp)]
    L.hweno_mlp_destroy.argtypes = [vp]
    L.hweno_mlp_destroy.restype = None
    L.hweno_mlp_set_params.argtypes = [vp, fp]
    L.hweno_mlp_get_params.argtypes = [vp, fp]
    L.hweno_mlp_gradient.argtypes = [vp, vp, vp, vp, C.c_int, C.c_double, C.c_double, fp, C.POINTER(C.c_double)]
    L.hweno_mlp_train_step.argtypes = [vp, vp, vp, vp, C.c_int, C.c_double, C.c_double, C.c_double]
    L.hweno_mlp_mean_loss.argtypes = [vp, C.POINTER(C.c_double)]
    L.hweno_mlp_predict.argtypes = [vp, vp, C.c_longlong, vp]
    L.hweno_project.argtypes = [vp, U0_FN, vp, C.c_int]
    L.hweno_get_time.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    L.hweno_set_time.argtypes = [vp, C.c_double]
    L.hweno_autotune.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    L.hweno_batch_autotune.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    _lib = L
    return L


def _check(st: int):
    if st != HWENO_OK:
        raise HwenoError(st, load().hweno_last_error().decode())


def _buf(x):
    """(pointer, on_device) of a torch tensor or numpy array (contiguous)."""
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data, 0
    import torch
    assert isinstance(x, torch.Tensor) and x.is_contiguous()
    return x.data_ptr(), 1 if x.is_cuda else 0


def _current_stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


# ---- module-level functions with the C entry points' names ----
def hweno_version() -> str:
    return load().hweno_version().decode()


def hweno_last_error() -> str:
    return load().hweno_last_error().decode()


def hweno_create(cfg: Config, stream=None):
    h = C.c_void_p()
    c = cfg.to_c()
    _check(load().hweno_create(C.byref(c), stream if stream is not None else _current_stream(), C.byref(h)))
    return h


def hweno_destroy(h):
    load().hweno_destroy(h)


def hweno_stream(h) -> int:
    return load().hweno_stream(h)


def hweno_set_state(h, U):
    p, dev = _buf(U)
    _check(load().hweno_set_state(h, C.c_void_p(p), dev))


def hweno_get_state(h, U):
    p, dev = _buf(U)
    _check(load().hweno_get_state(h, C.c_void_p(p), dev))


def hweno_alpha(h):
    ax, ay = C.c_double(), C.c_double()
    _check(load().hweno_alpha(h, C.byref(ax), C.byref(ay)))
    return ax.value, ay.value


def hweno_apply_operator(h, alpha_x, alpha_y, L_out, dhat_out):
    pl, _ = _buf(L_out)
    pd, _ = _buf(dhat_out)
    _check(load().hweno_apply_operator(h, alpha_x, alpha_y, C.c_void_p(pl), C.c_void_p(pd)))


def hweno_step(h, dt, alpha_x, alpha_y=0.0):
    _check(load().hweno_step(h, dt, alpha_x, alpha_y))


def hweno_advance(h, t_final, max_steps=2**31 - 1):
    t, n = C.c_double(), C.c_int()
    _check(load().hweno_advance(h, t_final, int(max_steps), C.byref(t), C.byref(n)))
    return t.value, n.value


def hweno_set_profiling(h, enable: bool):
    _check(load().hweno_set_profiling(h, 1 if enable else 0))


def hweno_profile(h):
    ms, n, k = C.c_double(), C.c_longlong(), C.c_longlong()
    _check(load().hweno_profile(h, C.byref(ms), C.byref(n), C.byref(k)))
    return ms.value, n.value, k.value


def hweno_stage(h, stage: int, dt: float, alpha_x: float, alpha_y: float = 0.0):
    _check(load().hweno_stage(h, int(stage), dt, alpha_x, alpha_y))


def hweno_rows(h, buffer: int, row0: int, rows, to_solver: bool):
    """rows: a CUDA tensor [nf, nrows, nx] of the solver's element type."""
    nrows = int(rows.shape[1])
    _check(load().hweno_rows(h, int(buffer), int(row0), nrows, C.c_void_p(_buf(rows)[0]), 1 if to_solver else 0))


def hweno_alpha_update(h):
    ax, ay = C.c_double(), C.c_double()
    _check(load().hweno_alpha_update(h, C.byref(ax), C.byref(ay)))
    return ax.value, ay.value


def hweno_batch_set_profiling(h, enable: bool):
    _check(load().hweno_batch_set_profiling(h, 1 if enable else 0))


def hweno_batch_profile(h):
    ms, n, k = C.c_double(), C.c_longlong(), C.c_longlong()
    _check(load().hweno_batch_profile(h, C.byref(ms), C.byref(n), C.byref(k)))
    return ms.value, n.value, k.value


def hweno_peak_fma(precision: int) -> float:
    f = C.c_double()
    _check(load().hweno_peak_fma(precision, C.byref(f)))
    return f.value


def hweno_selftest_convert(f_in, d_in):
    """f_in: float32 device tensor, d_in: float64 device tensor of the same
    length; returns (f_in widened to float64, d_in rounded to float32) as the
    library's integer-ALU conversions compute them."""
    import torch
    n = f_in.numel()
    if d_in.numel() != n or f_in.dtype != torch.float32 or d_in.dtype != torch.float64:
        raise ValueError("f_in float32 and d_in float64 of equal length")
    f_in, d_in = f_in.contiguous(), d_in.contiguous()
    wide = torch.empty(n, dtype=torch.float64, device=f_in.device)
    narrow = torch.empty(n, dtype=torch.float32, device=f_in.device)
    _check(load().hweno_selftest_convert(f_in.data_ptr(), wide.data_ptr(), d_in.data_ptr(), narrow.data_ptr(), n))
    return wide, narrow


def hweno_selftest_rcp64(x_in):
    """x_in: float64 device tensor; returns 1 / x_in as the library's FP64
    kernels compute the reciprocal."""
    import torch
    if x_in.dtype != torch.float64:
        raise ValueError("x_in float64")
    x_in = x_in.contiguous()
    y = torch.empty_like(x_in)
    _check(load().hweno_selftest_rcp64(x_in.data_ptr(), y.data_ptr(), x_in.numel()))
    return y


def hweno_batch_create(cfgs, stream=None):
    arr = (hweno_config * len(cfgs))(*[c.to_c() for c in cfgs])
    h = C.c_void_p()
    _check(load().hweno_batch_create(len(cfgs), arr, stream if stream is not None else _current_stream(),
                                     C.byref(h)))
    return h


def hweno_batch_destroy(h):
    load().hweno_batch_destroy(h)


def hweno_batch_stream(h) -> int:
    return load().hweno_batch_stream(h)


def hweno_batch_layout(h, n):
    total = C.c_size_t()
    offs = (C.c_size_t * (n + 1))()
    _check(load().hweno_batch_layout(h, C.byref(total), offs))
    return total.value, np.array(offs[:], dtype=np.int64)


def hweno_batch_set_state(h, U):
    p, dev = _buf(U)
    _check(load().hweno_batch_set_state(h, C.c_void_p(p), dev))


def hweno_batch_get_state(h, U):
    p, dev = _buf(U)
    _check(load().hweno_batch_get_state(h, C.c_void_p(p), dev))


def hweno_batch_advance(h, t_final, max_steps=2**31 - 1):
    n = len(t_final)
    tf = (C.c_double * n)(*[float(x) for x in t_final])
    t = (C.c_double * n)()
    s = (C.c_int * n)()
    _check(load().hweno_batch_advance(h, tf, int(max_steps), t, s))
    return np.array(t[:]), np.array(s[:])


def hweno_batch_apply_operator(h, alpha, L_out, dhat_out):
    n = len(alpha)
    a = (C.c_double * n)(*[float(x) for x in alpha])
    pl, _ = _buf(L_out)
    pd, _ = _buf(dhat_out)
    _check(load().hweno_batch_apply_operator(h, a, C.c_void_p(pl), C.c_void_p(pd)))


def hweno_step_1d_noalloc(cfg: Config, U_in, U_out, dt, alpha, stream=None):
    """One SSP-RK3 step of a 1D problem without any device allocation (its
    working memory is a fixed 16 MiB device array inside the library); for
    callers that cannot allocate device memory.  U_in, U_out: CUDA tensors."""
    c = cfg.to_c()
    pi, _ = _buf(U_in)
    po, _ = _buf(U_out)
    _check(load().hweno_step_1d_noalloc(C.byref(c), C.c_void_p(pi), C.c_void_p(po), dt, alpha,
                                        stream if stream is not None else _current_stream()))


def _fvec(theta):
    a = np.ascontiguousarray(theta, dtype=np.float32)
    assert a.size == MLP_NPARAM, a.size
    return a, a.ctypes.data_as(C.POINTER(C.c_float))


def hweno_indicator_features(h, feat_out):
    _check(load().hweno_indicator_features(h, C.c_void_p(_buf(feat_out)[0])))


def hweno_indicator_labels(h, dev_out):
    _check(load().hweno_indicator_labels(h, C.c_void_p(_buf(dev_out)[0])))


def hweno_indicator_load(h, theta, p_threshold=0.5):
    a, pa = _fvec(theta)
    _check(load().hweno_indicator_load(h, pa, a.size, p_threshold))


def hweno_indicator_off(h):
    _check(load().hweno_indicator_off(h))


def hweno_indicator_mask(h, smooth_out=None, troubled_out=None):
    ps = C.c_void_p(_buf(smooth_out)[0]) if smooth_out is not None else None
    pt = C.c_void_p(_buf(troubled_out)[0]) if troubled_out is not None else None
    _check(load().hweno_indicator_mask(h, ps, pt))


def hweno_indicator_train(feat, dev, epochs, batch, lr, delta, pos_weight=0.0, seed=0, init_params=None,
                          stream=None):
    """The whole GPU training (see include/hweno.h); returns (parameters
    float32[3521], per-epoch mean losses)."""
    n = int(dev.numel())
    o = hweno_train_opts(int(epochs), int(batch), float(lr), float(delta), float(pos_weight), int(seed))
    out = np.zeros(MLP_NPARAM, dtype=np.float32)
    losses = np.zeros(int(epochs), dtype=np.float64)
    init = None
    if init_params is not None:
        a, init = _fvec(init_params)
    _check(load().hweno_indicator_train(C.c_void_p(_buf(feat)[0]), C.c_void_p(_buf(dev)[0]), n, C.byref(o), init,
                                        out.ctypes.data_as(C.POINTER(C.c_float)),
                                        losses.ctypes.data_as(C.POINTER(C.c_double)),
                                        stream if stream is not None else _current_stream()))
    return out, [float(x) for x in losses]


def hweno_train_permutation(seed: int, epoch: int, n: int) -> np.ndarray:
    out = np.empty(int(n), dtype=np.int32)
    load().hweno_train_permutation(int(seed), int(epoch), int(n), out.ctypes.data_as(C.POINTER(C.c_int)))
    return out


def hweno_mlp_create(max_batch, stream=None):
    h = C.c_void_p()
    _check(load().hweno_mlp_create(int(max_batch), stream if stream is not None else _current_stream(),
                                   C.byref(h)))
    return h


def hweno_mlp_destroy(h):
    load().hweno_mlp_destroy(h)


def hweno_mlp_set_params(h, theta):
    a, pa = _fvec(theta)
    _check(load().hweno_mlp_set_params(h, pa))


def hweno_mlp_get_params(h):
    out = np.zeros(MLP_NPARAM, dtype=np.float32)
    _check(load().hweno_mlp_get_params(h, out.ctypes.data_as(C.POINTER(C.c_float))))
    return out


def hweno_mlp_gradient(h, feat, dev, idx, delta, pos_weight):
    g = np.zeros(MLP_NPARAM, dtype=np.float32)
    loss = C.c_double()
    _check(load().hweno_mlp_gradient(h, C.c_void_p(_buf(feat)[0]), C.c_void_p(_buf(dev)[0]),
                                     C.c_void_p(_buf(idx)[0]), int(idx.numel()), delta, pos_weight,
                                     g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss)))
    return loss.value, g


def hweno_mlp_train_step(h, feat, dev, idx, delta, pos_weight, lr):
    _check(load().hweno_mlp_train_step(h, C.c_void_p(_buf(feat)[0]), C.c_void_p(_buf(dev)[0]),
                                       C.c_void_p(_buf(idx)[0]), int(idx.numel()), delta, pos_weight, lr))


def hweno_mlp_mean_loss(h):
    x = C.c_double()
    _check(load().hweno_mlp_mean_loss(h, C.byref(x)))
    return x.value


def hweno_mlp_predict(h, feat, prob_out):
    n = prob_out.numel()
    _check(load().hweno_mlp_predict(h, C.c_void_p(_buf(feat)[0]), n, C.c_void_p(_buf(prob_out)[0])))


def hweno_project(h, u0, nc, nq=6):
    """u0(x, y) -> array (nc, n) of the conserved components at n points."""
    def cb(n, x, y, u, ctx):
        xs = np.ctypeslib.as_array(x, shape=(n,))
        ys = np.ctypeslib.as_array(y, shape=(n,))
        out = np.ctypeslib.as_array(u, shape=(n, nc))
        out[:] = np.asarray(u0(xs, ys), dtype=np.float64).reshape(nc, n).T
    fn = U0_FN(cb)
    _check(load().hweno_project(h, fn, None, int(nq)))


def hweno_get_time(h):
    t, n = C.c_double(), C.c_int()
    _check(load().hweno_get_time(h, C.byref(t), C.byref(n)))
    return t.value, n.value


def hweno_set_time(h, t):
    _check(load().hweno_set_time(h, float(t)))


def hweno_autotune(h, reps=3):
    ms = C.c_double()
    shp = (C.c_int * 3)()
    _check(load().hweno_autotune(h, int(reps), C.byref(ms), shp))
    return ms.value, tuple(shp)


def hweno_batch_autotune(h, reps=3):
    ms = C.c_double()
    shp = (C.c_int * 3)()
    _check(load().hweno_batch_autotune(h, int(reps), C.byref(ms), shp))
    return ms.value, tuple(shp)


# ---- conveniences ----
class Solver:
    """One grid.  State tensors are [nf, ny, nx] (2D) or [nf, nx] (1D)."""

    def __init__(self, cfg: Config, stream=None):
        import torch
        self.cfg = cfg
        self.dtype = torch.float64 if cfg.precision == FP64 else torch.float32
        self.h = hweno_create(cfg, stream)
        self.shape = (cfg.nfields, cfg.ny, cfg.nx) if cfg.dim == 2 else (cfg.nfields, cfg.nx)

    def close(self):
        if self.h is not None:
            hweno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def stream(self) -> int:
        return hweno_stream(self.h)

    def set_state(self, U):
        import torch
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.float64 if self.cfg.precision == FP64 else np.float32)
        else:
            U = U.to(self.dtype).contiguous()
        assert tuple(U.shape) == self.shape, (U.shape, self.shape)
        hweno_set_state(self.h, U)
        self._keep = U

    def get_state(self, device: bool = True):
        import torch
        if device:
            out = torch.empty(self.shape, dtype=self.dtype, device="cuda")
        else:
            out = np.empty(self.shape, dtype=np.float64 if self.cfg.precision == FP64 else np.float32)
        hweno_get_state(self.h, out)
        return out

    def alpha(self):
        return hweno_alpha(self.h)

    def apply_operator(self, alpha_x, alpha_y=0.0):
        import torch
        L = torch.empty(self.shape, dtype=self.dtype, device="cuda")
        nd = self.cfg.ncomp * self.cfg.dim
        D = torch.empty((nd,) + self.shape[1:], dtype=self.dtype, device="cuda")
        hweno_apply_operator(self.h, alpha_x, alpha_y, L, D)
        return L, D

    def step(self, dt, alpha_x, alpha_y=0.0):
        hweno_step(self.h, dt, alpha_x, alpha_y)

    def advance(self, t_final, max_steps=2**31 - 1):
        return hweno_advance(self.h, t_final, max_steps)

    def save(self, path: str):
        """Checkpoint: state, time and the config's fields to an .npz file."""
        import dataclasses
        t, _ = hweno_get_time(self.h)
        cfg = {k: np.asarray(v) for k, v in dataclasses.asdict(self.cfg).items()}
        np.savez(path, U=self.get_state(device=False), t=np.float64(t), **{"cfg_" + k: v for k, v in cfg.items()})

    def load(self, path: str):
        """Resume from save(): same grid and scheme required."""
        z = np.load(path)
        if tuple(z["U"].shape) != self.shape:
            raise ValueError("checkpoint state shape does not match this solver")
        self.set_state(np.ascontiguousarray(z["U"]))
        hweno_set_time(self.h, float(z["t"]))

    def set_profiling(self, enable: bool = True):
        hweno_set_profiling(self.h, enable)

    def profile(self):
        """(summed stage-kernel ms, stage launches, kernels launched by advance)."""
        return hweno_profile(self.h)


class Batch:
    """Independent problems of uneven sizes (all 1D or all 2D), advanced
    together: one launch per RK stage covers every instance."""

    def __init__(self, cfgs, stream=None):
        import torch
        self.cfgs = list(cfgs)
        self.n = len(self.cfgs)
        c0 = self.cfgs[0]
        self.dtype = torch.float64 if c0.precision == FP64 else torch.float32
        self.h = hweno_batch_create(self.cfgs, stream)
        self.total, self.offsets = hweno_batch_layout(self.h, self.n)
        self.nf = c0.nfields

    def close(self):
        if self.h is not None:
            hweno_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def stream(self) -> int:
        return hweno_batch_stream(self.h)

    def pack(self, states):
        """Concatenate per-instance [nf, n_k] (1D) or [nf, ny_k, nx_k] (2D)
        arrays into [nf, total]."""
        return np.concatenate([np.asarray(s, dtype=np.float64).reshape(self.nf, -1) for s in states], axis=1)

    def unpack(self, U):
        U = U.cpu().numpy() if hasattr(U, "cpu") else U
        out = []
        for k, c in enumerate(self.cfgs):
            part = U[:, self.offsets[k]:self.offsets[k + 1]]
            out.append(part.reshape(U.shape[0], c.ny, c.nx) if c.dim == 2 else part)
        return out

    def set_state(self, U):
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.float64 if self.dtype.itemsize == 8 else np.float32)
        else:
            U = U.to(self.dtype).contiguous()
        hweno_batch_set_state(self.h, U)
        self._keep = U

    def get_state(self, device: bool = True):
        import torch
        if device:
            out = torch.empty((self.nf, self.total), dtype=self.dtype, device="cuda")
        else:
            out = np.empty((self.nf, self.total), dtype=np.float64 if self.dtype.itemsize == 8 else np.float32)
        hweno_batch_get_state(self.h, out)
        return out

    def advance(self, t_final, max_steps=2**31 - 1):
        if np.isscalar(t_final):
            t_final = [t_final] * self.n
        return hweno_batch_advance(self.h, t_final, max_steps)

    def set_profiling(self, enable: bool = True):
        hweno_batch_set_profiling(self.h, enable)

    def profile(self):
        """(summed stage-kernel ms, stage launches, kernels launched by advance)."""
        return hweno_batch_profile(self.h)

    def apply_operator(self, alpha):
        """alpha: per instance alpha (1D) or (alpha_x, alpha_y) pairs (2D)."""
        import torch
        c0 = self.cfgs[0]
        L = torch.empty((self.nf, self.total), dtype=self.dtype, device="cuda")
        D = torch.empty((c0.ncomp * c0.dim, self.total), dtype=self.dtype, device="cuda")
        flat = np.asarray(alpha, dtype=np.float64).reshape(-1)
        hweno_batch_apply_operator(self.h, flat, L, D)
        return L, D
