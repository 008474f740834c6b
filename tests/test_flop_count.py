"""The algorithmic flop count of a cell update (oracle/flops.py, composed
step by step from the paper's formulas and the coefficient maps) against the
instrumented oracle, which charges the same counting rules where it evaluates
each formula: the two must agree exactly on every scheme variant, so neither
a step left out of the composition nor a formula charged twice goes
unnoticed.  The benchmark's roofline numerator is this count."""
import numpy as np
import pytest

import oracle
from oracle import flops as F
from paper_2607_24325_b300 import workloads as W

W2D = (0.99, 0.0025, 0.0025, 0.0025, 0.0025)


def _variants():
    out = dict(F.BENCH_WORKLOADS)
    out["advection2d"] = oracle.Problem(dim=2, equation=oracle.EQ_ADVECTION, lin_w=W2D)
    out["burgers1d_pow2"] = oracle.Problem(dim=1, equation=oracle.EQ_BURGERS, weight_pow=2)
    out["burgers1d_typical"] = oracle.Problem(dim=1, equation=oracle.EQ_BURGERS, smoothness=oracle.BETA_TYPICAL)
    out["euler2d_component_pow2"] = oracle.Problem(dim=2, equation=oracle.EQ_EULER, lin_w=W2D, charwise=0,
                                                   weight_pow=2)
    return out


@pytest.mark.parametrize("name", sorted(_variants()))
def test_instrumented_oracle_equals_the_composed_count(name):
    base = _variants()[name]
    n = 11
    prob = oracle.Problem(**{**base.__dict__, "nx": n, "ny": n if base.dim == 2 else 1, "xhi": 2.0,
                             "yhi": 2.0})
    cells = n ** prob.dim
    U = W.random_state(prob.dim, (n, n) if prob.dim == 2 else (n,), seed=5, euler=prob.equation == oracle.EQ_EULER,
                       moment_scale=0.1)
    ax, ay = oracle.alpha(prob, U)
    total = F.measured_step_total(prob, U, 1e-4, ax, ay)
    op, rk, a = F.per_step_parts(prob)
    assert total == cells * (3 * op + rk + a), (name, total / cells, 3 * op + rk + a)


def test_count_scales_with_cells_only():
    """Per cell the count does not depend on the grid (periodic sides)."""
    prob = oracle.Problem(dim=2, equation=oracle.EQ_BURGERS, lin_w=W2D, xhi=2.0, yhi=2.0)
    per = []
    for n in (6, 9):
        p = oracle.Problem(**{**prob.__dict__, "nx": n, "ny": n})
        U = W.random_state(2, (n, n), seed=1)
        per.append(F.measured_step_total(p, U, 1e-4, *oracle.alpha(p, U)) / n ** 2)
    assert per[0] == per[1]


def test_hand_counted_1d_advection():
    """1D linear advection counted by hand from the printed appendix rows.
    Step 1: dx v-bar of the two neighbours (2); c0_0..c0_4 have 5, 4, 5, 4, 5
    nonzero entries, none of them +-1 once divided by the row's denominator
    (960, 16, 8, 4, 4), so 2k - 1 flops a row (41); c1_0 = u_i and c2_0 =
    u_{i+1} are copies, c1_1 and c2_1 one difference each (2).  Step 2: two
    squares for beta_1, beta_2 and c1^2 + (2 c2)^2 + (6 c3)^2 + (24 c4)^2
    (10).  Step 3: 22.  The combination 26, the face values and v-hat 32, the
    flux at the right face 14, L 4, the three stages' updates 12 per field."""
    G0, G1, G2 = oracle.coef_maps_1d()
    assert [int((r != 0).sum()) for r in G0] == [5, 4, 5, 4, 5]
    assert sum(F.dot(r) for r in G0) == 41
    assert sum(F.dot(r) for r in G1) + sum(F.dot(r) for r in G2) == 2
    rec = 2 + 41 + 2 + 12 + 22 + 26 + 32
    p = oracle.Problem(dim=1, equation=oracle.EQ_ADVECTION)
    op, rk, a = F.per_step_parts(p)
    assert (op, rk, a) == (rec + 14 + 4, 2 * 12, 0)
    assert F.per_cell_stage(p) == 163
