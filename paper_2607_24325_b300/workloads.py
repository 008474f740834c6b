"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no step of the HWENO method: it only turns an analytic or
seeded problem description into the initial cell averages and derivative
moments (the problem's input data, Sec. 2.1 and 2.2 definitions of u-bar,
v-bar, w-bar), and gives the exact solutions used to measure errors.  Both the
CUDA path and the CPU oracle consume what it produces; neither is imported
here.

Layouts follow the library: ``U[f][j][i]`` (2D) or ``U[f][i]`` (1D), with
``f = d*nc + k``: d = 0 cell averages, 1 x-derivative moments, 2 y-derivative
moments; k the conserved component.  1D moments are means of u_x; 2D moments
are the scaled moments (1/dy) int u_x and (1/dx) int u_y.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = 1.4


def gauss_unit(n: int):
    """Gauss-Legendre nodes and weights on [-1/2, 1/2], weights summing to 1."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * x, 0.5 * w


# --------------------------------------------------------------------------
# Conservative variables
# --------------------------------------------------------------------------
def prim_to_cons_1d(rho, u, p, gamma=GAMMA):
    rho, u, p = np.broadcast_arrays(*(np.asarray(a, dtype=np.float64) for a in (rho, u, p)))
    return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])


def prim_to_cons_2d(rho, u, v, p, gamma=GAMMA):
    rho, u, v, p = np.broadcast_arrays(*(np.asarray(a, dtype=np.float64) for a in (rho, u, v, p)))
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


# --------------------------------------------------------------------------
# Cell averages and derivative moments of a smooth (or piecewise smooth with
# jumps on cell faces) initial condition.
# --------------------------------------------------------------------------
def cells_1d(f, xlo: float, xhi: float, nx: int, nq: int = 8) -> np.ndarray:
    """f(x) -> array (nc, *x.shape).  Returns U (2*nc, nx).

    u-bar by nq-point Gauss quadrature; v-bar, the mean of u_x over the cell,
    is exactly (u(x_{i+1/2}^-) - u(x_{i-1/2}^+)) / dx, evaluated with the
    one-sided limits from inside the cell."""
    dx = (xhi - xlo) / nx
    xc = xlo + (np.arange(nx) + 0.5) * dx
    s, w = gauss_unit(nq)
    pts = xc[None, :] + dx * s[:, None]                      # (nq, nx)
    vals = np.asarray(f(pts), dtype=np.float64)               # (nc, nq, nx)
    ubar = np.einsum("q,kqx->kx", w, vals)
    tiny = 1e-12 * dx
    right = np.asarray(f(xc + 0.5 * dx - tiny), dtype=np.float64)
    left = np.asarray(f(xc - 0.5 * dx + tiny), dtype=np.float64)
    # Use the exact face points when f is continuous there; the one-sided
    # nudge above only matters for jumps placed on faces.
    rf = np.asarray(f(xc + 0.5 * dx), dtype=np.float64)
    lf = np.asarray(f(xc - 0.5 * dx), dtype=np.float64)
    right = np.where(np.abs(rf - right) < 1e-6 * (1 + np.abs(rf)), rf, right)
    left = np.where(np.abs(lf - left) < 1e-6 * (1 + np.abs(lf)), lf, left)
    vbar = (right - left) / dx
    return np.concatenate([ubar, vbar], axis=0)


def cells_2d(f, xlo, xhi, ylo, yhi, nx, ny, nq: int = 8) -> np.ndarray:
    """f(x, y) -> array (nc, *x.shape).  Returns U (3*nc, ny, nx).

    u-bar by nq x nq tensor Gauss; v-bar = (1/dy) int u_x dOmega is the
    y-Gauss mean of the face difference u(x_{i+1/2}, y) - u(x_{i-1/2}, y);
    w-bar likewise in x.  Jumps must lie on cell faces (one-sided limits)."""
    dx, dy = (xhi - xlo) / nx, (yhi - ylo) / ny
    xc = xlo + (np.arange(nx) + 0.5) * dx
    yc = ylo + (np.arange(ny) + 0.5) * dy
    s, w = gauss_unit(nq)
    tx, ty = 1e-12 * dx, 1e-12 * dy
    X = xc[None, None, :] + dx * s[:, None, None]     # (q, 1, nx)
    Y = yc[None, :, None] + dy * s[:, None, None]     # (q, ny, 1)
    # u-bar: sum over qx, qy
    ubar = 0.0
    for a in range(nq):
        for b in range(nq):
            ubar = ubar + w[a] * w[b] * np.asarray(
                f(xc[None, :] + dx * s[a], yc[:, None] + dy * s[b]), dtype=np.float64)
    def face(xx, yy, xn, yn):
        """u at a face point: the exact point where u is continuous there, the
        one-sided limit from inside the cell (nudged point) at a jump."""
        exact = np.asarray(f(xx, yy), dtype=np.float64)
        inner = np.asarray(f(xn, yn), dtype=np.float64)
        return np.where(np.abs(exact - inner) < 1e-6 * (1 + np.abs(exact)), exact, inner)

    vbar = 0.0
    wbar = 0.0
    for b in range(nq):
        yy = yc[:, None] + dy * s[b]
        xr, xl = xc[None, :] + 0.5 * dx, xc[None, :] - 0.5 * dx
        vbar = vbar + w[b] * (face(xr, yy, xr - tx, yy) - face(xl, yy, xl + tx, yy))
    for a in range(nq):
        xx = xc[None, :] + dx * s[a]
        yt, yb = yc[:, None] + 0.5 * dy, yc[:, None] - 0.5 * dy
        wbar = wbar + w[a] * (face(xx, yt, xx, yt - ty) - face(xx, yb, xx, yb + ty))
    del X, Y
    return np.concatenate([ubar, vbar, wbar], axis=0)


# --------------------------------------------------------------------------
# Riemann problems with exact cell averages (jump anywhere).
# --------------------------------------------------------------------------
def riemann_1d(stateL, stateR, x0, xlo, xhi, nx, gamma=GAMMA) -> np.ndarray:
    """Piecewise-constant (rho, u, p) states split at x0.  Exact u-bar (cell
    fractions); v-bar = jump/dx in the cell that strictly contains x0, zero
    elsewhere (a jump on a face gives zero moments)."""
    UL = prim_to_cons_1d(*stateL, gamma=gamma)
    UR = prim_to_cons_1d(*stateR, gamma=gamma)
    dx = (xhi - xlo) / nx
    xl = xlo + np.arange(nx) * dx
    frac_left = np.clip((x0 - xl) / dx, 0.0, 1.0)        # fraction of the cell left of x0
    ubar = UL[:, None] * frac_left[None, :] + UR[:, None] * (1.0 - frac_left[None, :])
    inside = (frac_left > 0.0) & (frac_left < 1.0)
    vbar = np.where(inside[None, :], (UR - UL)[:, None] / dx, 0.0)
    return np.concatenate([ubar, vbar], axis=0)


def quadrant_2d(states, xs, ys, xlo, xhi, ylo, yhi, nx, ny, gamma=GAMMA) -> np.ndarray:
    """Four-quadrant Riemann problem.  states[q] = (rho, u, v, p) for the
    quadrants q = 0 (x>xs, y>ys), 1 (x<xs, y>ys), 2 (x<xs, y<ys),
    3 (x>xs, y<ys).  Exact u-bar by area fractions; exact scaled moments
    from the jumps crossing the cell."""
    Q = [prim_to_cons_2d(*s, gamma=gamma) for s in states]  # each (4,)
    dx, dy = (xhi - xlo) / nx, (yhi - ylo) / ny
    xl = xlo + np.arange(nx) * dx
    yl = ylo + np.arange(ny) * dy
    fx = np.clip((xs - xl) / dx, 0.0, 1.0)   # fraction with x < xs
    fy = np.clip((ys - yl) / dy, 0.0, 1.0)   # fraction with y < ys
    FX, FY = np.meshgrid(fx, fy)             # (ny, nx)
    ubar = (Q[0][:, None, None] * ((1 - FX) * (1 - FY))[None]
            + Q[1][:, None, None] * (FX * (1 - FY))[None]
            + Q[2][:, None, None] * (FX * FY)[None]
            + Q[3][:, None, None] * ((1 - FX) * FY)[None])
    inx = ((FX > 0) & (FX < 1))[None]
    iny = ((FY > 0) & (FY < 1))[None]
    # v-bar = (1/dy) int [u(x_{i+1/2},y) - u(x_{i-1/2},y)] dy = mean over y of
    # the x jump: upper part (fraction 1-FY) jumps Q1->Q0, lower part Q2->Q3.
    jx = (Q[0] - Q[1])[:, None, None] * (1 - FY)[None] + (Q[3] - Q[2])[:, None, None] * FY[None]
    jy = (Q[1] - Q[2])[:, None, None] * FX[None] + (Q[0] - Q[3])[:, None, None] * (1 - FX)[None]
    vbar = np.where(inx, jx, 0.0)
    wbar = np.where(iny, jy, 0.0)
    return np.concatenate([ubar, vbar, wbar], axis=0)


# --------------------------------------------------------------------------
# The paper's smooth examples and their exact solutions.
# --------------------------------------------------------------------------
def burgers_exact_1d(x, t, u0, du0, iters: int = 60):
    """u = u0(x - u t) by Newton (smooth for t < breaking time)."""
    x = np.asarray(x, dtype=np.float64)
    u = u0(x)
    for _ in range(iters):
        g = u - u0(x - u * t)
        dg = 1.0 + t * du0(x - u * t)
        u = u - g / dg
    return u


def sine_burgers_1d(t):
    """Example 1: u0 = 0.5 + sin(pi x) on [0, 2], exact for t < 1/pi."""
    u0 = lambda x: 0.5 + np.sin(np.pi * x)
    du0 = lambda x: np.pi * np.cos(np.pi * x)
    return lambda x: burgers_exact_1d(x, t, u0, du0)[None]


def sine_burgers_2d(t):
    """Example 3: u0 = 0.5 + sin(pi (x+y)/2) on [0, 4]^2; u = u0(s - 2 u t) with s = x + y."""
    u0 = lambda s: 0.5 + np.sin(0.5 * np.pi * s)
    du0 = lambda s: 0.5 * np.pi * np.cos(0.5 * np.pi * s)

    def f(x, y):
        s = np.asarray(x + y, dtype=np.float64)
        u = u0(s)
        for _ in range(60):
            g = u - u0(s - 2.0 * u * t)
            dg = 1.0 + 2.0 * t * du0(s - 2.0 * u * t)
            u = u - g / dg
        return u[None]
    return f


def euler_smooth_1d(t, gamma=GAMMA):
    """Example 2: rho = 1 + 0.2 sin(pi (x - t)), u = 1, p = 1 on [0, 2]."""
    return lambda x: prim_to_cons_1d(1.0 + 0.2 * np.sin(np.pi * (x - t)), 1.0, 1.0, gamma)


def euler_smooth_2d(t, gamma=GAMMA):
    """Example 4: rho = 1 + 0.2 sin(pi (x + y - 2t)), u = v = p = 1 on [0, 2]^2."""
    return lambda x, y: prim_to_cons_2d(1.0 + 0.2 * np.sin(np.pi * (x + y - 2.0 * t)), 1.0, 1.0, 1.0,
                                        gamma)


# --------------------------------------------------------------------------
# Seeded batches and families.
# --------------------------------------------------------------------------
@dataclass
class RiemannBatch:
    sizes: np.ndarray          # cells per instance
    states: np.ndarray         # (n, 2, 3): left/right (rho, u, p)
    x0: float = 0.5
    xlo: float = 0.0
    xhi: float = 1.0

    def instance(self, k: int) -> np.ndarray:
        return riemann_1d(self.states[k, 0], self.states[k, 1], self.x0, self.xlo, self.xhi,
                          int(self.sizes[k]))


def riemann_batch_1d(n: int = 256, seed: int = 1234, nmin: int = 256, nmax: int = 8192,
                     include_lax: bool = True) -> RiemannBatch:
    """Seeded 1D Euler Riemann problems on [0,1] with the jump at 0.5:
    rho, p ~ U[0.1, 10], u ~ U[-2, 2] per side; sizes log-uniform in
    [nmin, nmax].  Instance 0 is the Lax problem (Example 5, shifted)."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.1, 10.0, size=(n, 2))
    u = rng.uniform(-2.0, 2.0, size=(n, 2))
    p = rng.uniform(0.1, 10.0, size=(n, 2))
    sizes = np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=n)).astype(np.int64)
    sizes = np.clip(sizes, nmin, nmax)
    states = np.stack([rho, u, p], axis=-1)            # (n, 2, 3)
    if include_lax and n > 0:
        states[0, 0] = (0.445, 0.698, 3.528)
        states[0, 1] = (0.5, 0.0, 0.571)
    return RiemannBatch(sizes=sizes, states=states)


def quadrant_states(seed: int = 2024):
    """Seeded four-quadrant states: rho, p ~ U[0.1, 1.5], u, v ~ U[-1, 1]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(4):
        rho, p = rng.uniform(0.1, 1.5, size=2)
        u, v = rng.uniform(-1.0, 1.0, size=2)
        out.append((rho, u, v, p))
    return out


def shock_entropy_2d(seed: int = 7, x_shock: float = 0.2, gamma=GAMMA):
    """Shock / entropy-wave family on [0,1]^2: a normal shock of Mach
    M ~ U[1.1, 3] at x = x_shock moving right into a still gas with
    rho = 1 + 0.2 sin(k (x cos th + y sin th)), p = 1; k = pi * U{5..20},
    th ~ U[0, pi/2).  Post-shock state from the Rankine-Hugoniot relations.
    Returns f(x, y) for cells_2d (the jump must lie on a cell face)."""
    rng = np.random.default_rng(seed)
    M = rng.uniform(1.1, 3.0)
    k = math.pi * int(rng.integers(5, 21))
    th = rng.uniform(0.0, 0.5 * math.pi)
    amp = 0.2
    g = gamma
    # post-shock state for a shock moving at speed s = M c1 into gas at rest (rho1=1, p1=1)
    rho1, p1 = 1.0, 1.0
    c1 = math.sqrt(g * p1 / rho1)
    rho2 = rho1 * (g + 1) * M * M / ((g - 1) * M * M + 2)
    p2 = p1 * (2 * g * M * M - (g - 1)) / (g + 1)
    u2 = M * c1 * (1.0 - rho1 / rho2)

    def f(x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        x, y = np.broadcast_arrays(x, y)
        pre = x >= x_shock
        rho = np.where(pre, 1.0 + amp * np.sin(k * (x * math.cos(th) + y * math.sin(th))), rho2)
        u = np.where(pre, 0.0, u2)
        p = np.where(pre, p1, p2)
        return prim_to_cons_2d(rho, u, 0.0 * x, p, gamma)
    f.params = {"mach": M, "k": k, "theta": th, "rho2": rho2, "u2": u2, "p2": p2}
    return f


def random_positive_weights(n: int, seed: int) -> tuple:
    """Seeded positive linear weights summing to one (U(0.05, 1), normalised)."""
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.05, 1.0, size=n)
    return tuple(float(a) for a in (w / w.sum()))


def random_state(dim: int, shape, seed: int, euler: bool = False, gamma=GAMMA,
                 moment_scale: float = 0.5) -> np.ndarray:
    """Seeded rough data (every cell independent) for single-operator parity:
    scalar u-bar ~ N(0, 1); Euler rho, p ~ U[0.5, 1.5], velocities ~ U[-1, 1];
    derivative moments ~ moment_scale * N(0, 1) (times rho-scale for Euler).
    Returns U with dim+1 groups of nc fields over `shape` (cells)."""
    rng = np.random.default_rng(seed)
    shape = tuple(shape)
    if not euler:
        ub = rng.normal(size=(1,) + shape)
        mom = moment_scale * rng.normal(size=(dim,) + shape)
        return np.concatenate([ub, mom], axis=0)
    rho = rng.uniform(0.5, 1.5, size=shape)
    p = rng.uniform(0.5, 1.5, size=shape)
    if dim == 1:
        u = rng.uniform(-1, 1, size=shape)
        ub = prim_to_cons_1d(rho, u, p, gamma)
        nc = 3
    else:
        u = rng.uniform(-1, 1, size=shape)
        v = rng.uniform(-1, 1, size=shape)
        ub = prim_to_cons_2d(rho, u, v, p, gamma)
        nc = 4
    mom = moment_scale * rng.normal(size=(dim * nc,) + shape)
    return np.concatenate([ub, mom], axis=0)


# --------------------------------------------------------------------------
# Double Mach reflection (the paper's Sec. 3 example after Woodward and
# Colella): a Mach 10 shock at 60 degrees to a reflecting wall on
# [0, 4] x [0, 1]; the shock line x = 1/6 + y / sqrt(3) at t = 0 moves with
# speed 10 along its normal, so it meets the top boundary at
# x = 1/6 + (1 + 20 t) / sqrt(3).
# --------------------------------------------------------------------------
DMR_DOMAIN = (0.0, 4.0, 0.0, 1.0)
DMR_X0 = 1.0 / 6.0
_SQ3 = math.sqrt(3.0)


def dmr_states(gamma=GAMMA):
    """(post-shock, pre-shock) conservative states (rho, rho u, rho v, E)."""
    post = prim_to_cons_2d(8.0, 8.25 * math.sin(math.pi / 3.0), -8.25 * math.cos(math.pi / 3.0), 116.5, gamma=gamma)
    pre = prim_to_cons_2d(1.4, 0.0, 0.0, 1.0, gamma=gamma)
    return np.asarray(post, dtype=np.float64), np.asarray(pre, dtype=np.float64)


def dmr_boundary(gamma=GAMMA) -> dict:
    """Boundary description of the example, as plain numbers shared by the
    library config and the oracle problem: left inflow (post-shock), right
    outflow, bottom split wall (post-shock for x < 1/6, reflective after),
    top moving shock (post-shock behind x0 + s t, pre-shock ahead).  Codes:
    1 outflow, 3 inflow, 4 split, 5 moving shock."""
    post, pre = dmr_states(gamma)
    z = [0.0] * 4
    return {"bc": (3, 1, 4, 5),
            "bc_state": [list(post), z, list(post), list(post)],
            "bc_state2": [z, z, z, list(pre)],
            "bc_param": [[0.0, 0.0], [0.0, 0.0], [DMR_X0, 0.0], [DMR_X0 + 1.0 / _SQ3, 20.0 / _SQ3]]}


def _clip_int(z, h):
    """Antiderivative of clip(z, 0, h) (zero at z <= 0)."""
    z = np.asarray(z, dtype=np.float64)
    return np.where(z <= 0.0, 0.0, np.where(z < h, 0.5 * z * z, 0.5 * h * h + h * (z - h)))


def dmr_2d(nx, ny, gamma=GAMMA) -> np.ndarray:
    """Exact cell averages and scaled moments of the initial state on the
    example's domain: post-shock where x < 1/6 + y / sqrt(3).  The average
    takes the exact area fraction left of the line; v-bar and w-bar are the
    exact face-difference means (the jump times the share of the face-to-face
    segment the line crosses)."""
    post, pre = dmr_states(gamma)
    xlo, xhi, ylo, yhi = DMR_DOMAIN
    dx, dy = (xhi - xlo) / nx, (yhi - ylo) / ny
    xl = (xlo + np.arange(nx) * dx)[None, :]
    yb = (ylo + np.arange(ny) * dy)[:, None]
    yt = yb + dy
    b = 1.0 / _SQ3                        # x_s(y) = DMR_X0 + b y
    z0 = DMR_X0 + b * yb - xl             # x_s - x_left at the cell's bottom and top
    z1 = DMR_X0 + b * yt - xl
    frac = (_clip_int(z1, dx) - _clip_int(z0, dx)) / (b * dx * dy)   # share with x < x_s(y)
    frac = np.clip(frac, 0.0, 1.0)
    ubar = post[:, None, None] * frac[None] + pre[:, None, None] * (1.0 - frac)[None]
    # v-bar: y-share of the cell where the line lies between the two x faces
    ylo_cross = (xl - DMR_X0) / b
    yhi_cross = (xl + dx - DMR_X0) / b
    sv = np.clip(np.minimum(yt, yhi_cross) - np.maximum(yb, ylo_cross), 0.0, None) / dy
    vbar = (pre - post)[:, None, None] * sv[None]
    # w-bar: x-share of the cell where the line lies between the two y faces
    xs_b = DMR_X0 + b * yb
    xs_t = DMR_X0 + b * yt
    sw = np.clip(np.minimum(xl + dx, xs_t) - np.maximum(xl, xs_b), 0.0, None) / dx
    wbar = (post - pre)[:, None, None] * sw[None]
    return np.concatenate([ubar, vbar, wbar], axis=0)


def quadrant_batch_2d(n: int = 48, seed: int = 2025, nmin: int = 96, nmax: int = 768):
    """Seeded batch of 2D four-quadrant Riemann problems on [0,1]^2 of uneven
    sizes: nx, ny log-uniform in [nmin, nmax] independently, quadrant states
    quadrant_states(seed + k), split point U[0.3, 0.7]^2.  Returns (sizes
    [(nx, ny)], states [U_k])."""
    rng = np.random.default_rng(seed)
    nx = np.clip(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=n)).astype(np.int64), nmin, nmax)
    ny = np.clip(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=n)).astype(np.int64), nmin, nmax)
    split = rng.uniform(0.3, 0.7, size=(n, 2))
    sizes = [(int(nx[k]), int(ny[k])) for k in range(n)]
    states = [quadrant_2d(quadrant_states(seed + k), split[k, 0], split[k, 1], 0.0, 1.0, 0.0, 1.0, *sizes[k])
              for k in range(n)]
    return sizes, states


# --------------------------------------------------------------------------
# Closed-form cell data of sine waves at large sizes (the throughput runs of
# Examples 1 and 3): the cell mean of sin(k s) over [s - h/2, s + h/2] is
# sin(k s) sin(k h / 2) / (k h / 2).
# --------------------------------------------------------------------------
def _sinc_half(k, h):
    z = 0.5 * k * h
    return math.sin(z) / z


def sine_1d_cells(n: int, xlo: float = 0.0, xhi: float = 2.0, k: float = math.pi, offset: float = 0.0):
    """u0 = offset + sin(k x): exact cell averages and v-bar (the mean of u_x,
    i.e. the face difference over dx), [2, n]."""
    dx = (xhi - xlo) / n
    xc = xlo + (np.arange(n) + 0.5) * dx
    ubar = offset + np.sin(k * xc) * _sinc_half(k, dx)
    vbar = (np.sin(k * (xc + 0.5 * dx)) - np.sin(k * (xc - 0.5 * dx))) / dx
    return np.stack([ubar, vbar])


def sine_2d_cells(nx: int, ny: int, xlo: float = 0.0, xhi: float = 4.0, ylo: float = 0.0, yhi: float = 4.0,
                  k: float = 0.5 * math.pi, offset: float = 0.5):
    """u0 = offset + sin(k (x + y)) (Example 3 with offset 0.5 and k = pi/2):
    exact cell averages and scaled moments, [3, ny, nx]."""
    dx, dy = (xhi - xlo) / nx, (yhi - ylo) / ny
    xc = (xlo + (np.arange(nx) + 0.5) * dx)[None, :]
    yc = (ylo + (np.arange(ny) + 0.5) * dy)[:, None]
    sx, sy = _sinc_half(k, dx), _sinc_half(k, dy)
    ubar = offset + np.sin(k * (xc + yc)) * sx * sy
    vbar = (np.sin(k * (xc + 0.5 * dx + yc)) - np.sin(k * (xc - 0.5 * dx + yc))) * sy
    wbar = (np.sin(k * (xc + yc + 0.5 * dy)) - np.sin(k * (xc + yc - 0.5 * dy))) * sx
    return np.stack([ubar, vbar, wbar])
