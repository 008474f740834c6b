"""Algorithmic flop count of one cell update in one RK stage.

TEST INFRASTRUCTURE AND A STORED-VALUE SCRIPT (same rules as the rest of
oracle/).  The count is the method's own arithmetic, not any implementation's:
every formula of Sec. 2.1 / 2.2 Steps 1-4 and Remark 1 charged as its plain
evaluation -- add, subtract, multiply, divide, square root 1 flop; absolute
values and comparisons free; a product with a constant (map coefficient,
basis value at a fixed point, factorial, Gauss or linear weight, gamma, grid
spacing, alpha, dt) 1 flop, none for a constant +-1, the term dropped for a
constant 0; a sum of k terms k - 1 adds; a quantity used more than once
formed once.  Each cell is reconstructed once per stage (per pass for
characteristic 2D Euler, a pass needing its own two faces and one limited
derivative) and owns its right (and top) face; alpha is formed once per step.

`per_cell_stage(prob)` composes the count step by step from the coefficient
maps; the instrumented oracle (`oracle.flop_count`) charges the same rules
where it evaluates each formula, and tests/test_flop_count.py requires the two
to agree exactly.  Run as a script it prints the counts of the benchmark
workloads.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from . import (EQ_ADVECTION, EQ_BURGERS, EQ_EULER, BETA_TYPICAL, Problem, coef_maps_1d, coef_maps_2d)

GAUSS = (-np.sqrt(15.0) / 10.0, 0.0, np.sqrt(15.0) / 10.0)
EXP2 = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2), (3, 0), (2, 1), (1, 2), (0, 3),
        (4, 0), (3, 1), (2, 2), (1, 3), (0, 4)]


def dot(c) -> int:
    """Plain dot product with constant coefficients c."""
    c = [float(x) for x in np.ravel(c) if x != 0.0]
    if not c:
        return 0
    return sum(1 for x in c if abs(x) != 1.0) + len(c) - 1


def weights(nlin: int, pow2: bool) -> int:
    """Step 3: tau (nlin differences, nlin - 1 adds, 1/nlin), tau^2, per
    weight (beta^2) + eps, quotient, 1 +, gamma x; their sum; normalisation."""
    np_ = nlin + 1
    return nlin + (nlin - 1) + 1 + 1 + np_ * (4 + pow2) + nlin + np_


def recon_1d(prob: Problem) -> int:
    G0, G1, G2 = coef_maps_1d()
    n = 2                                                # dx v-bar of the two neighbours
    n += sum(dot(r) for r in G0) + sum(dot(r) for r in G1) + sum(dot(r) for r in G2)
    if prob.smoothness == BETA_TYPICAL:
        n += (1 + 5 * 2 + 5) + 1 + 1                     # quartic form (6 terms), two lines
    else:
        n += 2 + (1 + 3 * 2 + 3)                         # beta_1,2; beta_0 = c1^2 + sum (l! c_l)^2
    n += 0 if prob.linear_weights else weights(2, prob.weight_pow == 2)
    n += 2 * (2 + 2 + 1 + 3 + 2) + 3 * 2                 # Eq. hweno-reconstruction-1D, as in the oracle
    face_u = dot([(-0.5) ** l for l in range(5)])
    face_d = 4 + 3                                       # 4 terms, constants l (-+1/2)^(l-1) / dx
    return n + 2 * face_u + 2 * face_d + 2


def face_2d(face: int) -> int:
    n = 0
    for s in GAUSS:
        xi, eta = ((-0.5 if face == 0 else 0.5), s) if face < 2 else (s, (-0.5 if face == 2 else 0.5))
        n += dot([xi ** m * eta ** k for m, k in EXP2])
        n += dot([m * xi ** (m - 1) * eta ** k if m else 0.0 for m, k in EXP2]) + 1
        n += dot([k * xi ** m * eta ** (k - 1) if k else 0.0 for m, k in EXP2]) + 1
    return n


def vhat_2d() -> int:
    def dif(m):
        return 0.5 ** m - (-0.5) ** m

    def avg(k):
        return (0.5 ** (k + 1) - (-0.5) ** (k + 1)) / (k + 1)
    return dot([dif(m) * avg(k) for m, k in EXP2])


def recon_2d_core(prob: Problem) -> int:
    """Steps 1-3 of one field up to the combined polynomial."""
    G0, Gm = coef_maps_2d()
    n = sum(dot(r) for r in G0) + sum(dot(r) for m in range(4) for r in Gm[m])
    if prob.smoothness == BETA_TYPICAL:
        n += (2 * 1 + 27 * 2 + 28) + 4 * 3
    else:
        n += (3 * 1 + 11 * 2 + 13) + 4 * 3
    n += 0 if prob.linear_weights else weights(4, prob.weight_pow == 2)
    n += 3 * (8 + 7 + 3) + 12 * 2                         # Eq. hweno-reconstruction-2D
    return n


def flux_point(prob: Problem) -> int:
    fam, nc = prob.dim + 1, prob.ncomp
    if prob.equation == EQ_ADVECTION:
        state = fam
    elif prob.equation == EQ_BURGERS:
        state = 2 + (fam - 1)
    elif prob.dim == 1:
        state = 7 + 2 + 9 + 10
    else:
        state = 11 + 4 + 12 + 2 * 19
    return 2 * state + 5 * fam * nc


def alpha_per_cell(prob: Problem) -> int:
    if prob.equation != EQ_EULER:
        return 0
    return 10 if prob.dim == 1 else 14


def per_step_parts(prob: Problem) -> tuple:
    """(flops of one stage's operator per cell without the RK update,
    RK flops of the three stages per cell, alpha per cell per step)."""
    nc, nf = prob.ncomp, prob.nfields
    chr_ = prob.equation == EQ_EULER and prob.charwise
    if prob.dim == 1:
        rec = nc * recon_1d(prob)
        if chr_:
            rec += 11 + 6 + 16 + 5 * 15 + 5 * 12
        op = rec + flux_point(prob) + 2 * nc * 2
    else:
        if chr_:
            per_pass = [6 + 18 + 17 * 23 + nc * (recon_2d_core(prob) + face_2d(2 * d) + face_2d(2 * d + 1)
                                                 + vhat_2d()) + 19 * 20 for d in (0, 1)]
            rec = 14 + sum(per_pass)
        else:
            rec = nc * (recon_2d_core(prob) + sum(face_2d(f) for f in range(4)) + 2 * vhat_2d())
        face = 3 * flux_point(prob) + 3 * nc * 5
        op = rec + 2 * face + 3 * nc * 4
    return op, nf * (2 + 5 + 5), alpha_per_cell(prob)


def per_cell_stage(prob: Problem) -> Fraction:
    """Algorithmic flops of one cell update in one RK stage (alpha's once per
    step shared by the three stages)."""
    op, rk, a = per_step_parts(prob)
    return Fraction(3 * op + rk + a, 3)


def measured_step_total(prob: Problem, U, dt: float, ax: float, ay: float = 0.0) -> int:
    """The instrumented oracle's count for alpha of U and one SSP-RK3 step."""
    from . import alpha, flop_count, step
    flop_count(reset=True)
    alpha(prob, U)
    step(prob, U, dt, ax, ay)
    return flop_count(reset=True)


W2D = (0.99, 0.0025, 0.0025, 0.0025, 0.0025)
BENCH_WORKLOADS = {
    "advection1d": Problem(dim=1, equation=EQ_ADVECTION),
    "burgers1d": Problem(dim=1, equation=EQ_BURGERS),
    "euler1d_char": Problem(dim=1, equation=EQ_EULER, charwise=1),
    "euler1d_component": Problem(dim=1, equation=EQ_EULER, charwise=0),
    "burgers2d": Problem(dim=2, equation=EQ_BURGERS, lin_w=W2D),
    "euler2d_char": Problem(dim=2, equation=EQ_EULER, lin_w=W2D, charwise=1),
    "euler2d_char_typical": Problem(dim=2, equation=EQ_EULER, lin_w=W2D, charwise=1, smoothness=BETA_TYPICAL),
    "euler2d_component": Problem(dim=2, equation=EQ_EULER, lin_w=W2D, charwise=0),
}


if __name__ == "__main__":
    for name, prob in BENCH_WORKLOADS.items():
        v = per_cell_stage(prob)
        print(f"    {name!r}: {float(v):.4f},")
