"""Soundness of the mixed-precision screens' bounds, replayed on the CPU.

The screens (hweno_device.cuh screen1 in 1D, hweno_stencil2d.cuh coef2 and
screen2 in 2D) skip the FP64 smoothness indicator where FP32 arithmetic
proves every a_m = tau^2 / (beta_m^p + eps) of Step 3 (Sec. 2.1 / 2.2) to be
at most 2^-24, so that 1 + a_m rounds to 1 in FP32.  Here their formulas run in IEEE single precision (numpy float32, round to nearest;
the approximate square root taken at the low end of its error bound, the
side that weakens the bound) on adversarial stencils -- smooth samples of
every resolution, near-constant data on large offsets, rough data, single
jumps, extreme scales -- and every stencil it clears must have an a_m, from
the same FP32 inputs in FP64, below 2^-24.  It must also clear the smooth
stencils whose a_m is far below the threshold (the screen is useful)."""
import numpy as np
import pytest

f32 = np.float32


def _screen(um, u0, up, a, b, eps, pow2):
    """screen1's arithmetic, elementwise in float32."""
    dm, dp = um - u0, up - u0
    S = np.maximum(np.maximum(np.abs(dm), np.abs(dp)), np.maximum(np.abs(a), np.abs(b)))
    E = S * f32(2.0 ** -16)
    sd, df, ab, ba = dm + dp, dp - dm, a + b, b - a
    c1 = f32(0.8125) * df - f32(0.3125) * ab
    c2 = f32(1.25) * sd - f32(0.375) * ba
    c3 = f32(0.25) * (ab - df)
    c4 = f32(0.25) * ba - f32(0.5) * sd
    b0 = c1 * c1 + f32(4) * (c2 * c2) + f32(36) * (c3 * c3) + f32(576) * (c4 * c4)
    b1, b2 = dm * dm, dp * dp
    sq = (np.sqrt(b0.astype(np.float64)) * (1 - 2.0 ** -21)).astype(f32)   # sqrt.approx, low side
    D0 = f32(2.0 ** -18) * b0 + E * (f32(50) * sq + f32(617) * E)
    D1, D2 = f32(2.0 ** -20) * b1, f32(2.0 ** -20) * b2
    tau = f32(0.5) * (np.abs(b0 - b1) + np.abs(b0 - b2))
    ut = tau * (f32(1) + f32(2.0 ** -20)) + D0 + f32(0.5) * (D1 + D2)
    L = np.maximum(np.minimum(np.minimum(b0 - D0, b1 - D1), b2 - D2), f32(0))
    dlo = (L * L if pow2 else L) + f32(eps)
    return ut * ut < f32(2.0 ** -25) * dlo


def _exact_a(um, u0, up, vm, vp, dx, eps, pow2):
    """The FP64 indicator of the mixed path from the same FP32 inputs."""
    Um, U0, Up = (x.astype(np.float64) for x in (um, u0, up))
    A = np.float64(dx) * vm.astype(np.float64)
    B = np.float64(dx) * vp.astype(np.float64)
    S, D, AB, BA = Um + Up, Up - Um, A + B, B - A
    e1 = 13 / 16 * D - 5 / 16 * AB
    e2 = 5 / 4 * S - 5 / 2 * U0 - 3 / 8 * BA
    e3 = 0.25 * (AB - D)
    e4 = U0 - 0.5 * S + 0.25 * BA
    beta = [e1 * e1 + 4 * e2 * e2 + 36 * e3 * e3 + 576 * e4 * e4, (U0 - Um) ** 2, (Up - U0) ** 2]
    tau = 0.5 * (np.abs(beta[0] - beta[1]) + np.abs(beta[0] - beta[2]))
    return np.max([tau * tau / ((bm * bm if pow2 else bm) + eps) for bm in beta], axis=0)


def _stencils(rng, n):
    out = []
    # smooth: a sine sampled at resolution h (cell averages and mean derivatives exactly)
    for h in (1e-1, 1e-2, 1e-3, 1e-4, 1e-5):
        x = rng.uniform(0, 10, n)
        k, amp, off = rng.uniform(0.5, 5, n), rng.uniform(0.01, 2, n), rng.uniform(-10, 10, n)

        def avg(xc):
            return off + amp * (np.cos(k * (xc - h / 2)) - np.cos(k * (xc + h / 2))) / (k * h)

        def dmean(xc):
            return amp * (np.sin(k * (xc + h / 2)) - np.sin(k * (xc - h / 2))) / h
        out.append((avg(x - h), avg(x), avg(x + h), dmean(x - h), dmean(x + h), h))
    # near-constant on large offsets
    base = rng.uniform(-1e3, 1e3, n)
    tiny = rng.normal(0, 1e-4, (5, n))
    out.append((base + tiny[0], base + tiny[1], base + tiny[2], tiny[3], tiny[4], 1e-3))
    # rough and jumps
    r = rng.normal(0, 1, (5, n))
    out.append((r[0], r[1], r[2], r[3], r[4], 1e-2))
    jump = np.where(rng.uniform(size=n) < 0.5, 1.0, 0.0)
    out.append((np.zeros(n), jump, jump + 1e-7 * rng.normal(size=n), np.zeros(n), np.zeros(n), 1e-2))
    # extreme scales
    s = 10.0 ** rng.uniform(-6, 6, n)
    r = rng.normal(0, 1, (5, n))
    out.append((s * (1 + 1e-6 * r[0]), s, s * (1 + 1e-6 * r[2]), s * 1e-6 * r[3], s * 1e-6 * r[4], 1.0))
    return out


@pytest.mark.parametrize("eps", [1e-6, 1e-8, 1e-12])
@pytest.mark.parametrize("pow2", [False, True])
def test_screen1_bound_is_sound(eps, pow2):
    rng = np.random.default_rng(int(eps ** -0.25) + pow2)
    cleared = smooth_tiny = smooth_cleared = 0
    for um, u0, up, vm, vp, h in _stencils(rng, 6000):
        um, u0, up, vm, vp = (np.asarray(x, dtype=f32) for x in (um, u0, up, vm, vp))
        dx = f32(h)
        q = _screen(um, u0, up, dx * vm, dx * vp, eps, pow2)
        a = _exact_a(um, u0, up, vm, vp, dx, eps, pow2)
        assert np.all(a[q] <= 2.0 ** -24), (h, a[q].max())
        cleared += int(q.sum())
        tiny = a < 2.0 ** -40
        smooth_tiny += int(tiny.sum())
        smooth_cleared += int((q & tiny).sum())
    assert cleared > 0
    assert smooth_cleared > 0.5 * smooth_tiny


# ------------------------------------------------------------------- 2D
def _coef2_f32(q):
    """The stage kernel's FP32 coefficient map (centre-shifted, coef2) and the
    four linear slopes, elementwise in float32; q: [17][n]."""
    q5 = q[4]
    d = [q[k] - q5 for k in range(9)]
    d1, d2, d3, d4, d6, d7, d8, d9 = d[0], d[1], d[2], d[3], d[5], d[6], d[7], d[8]
    q10, q11, q12, q13, q14, q15, q16, q17 = (q[k] for k in range(9, 17))
    s13, s79, m13, m79 = d1 + d3, d7 + d9, d1 - d3, d7 - d9
    sc, cx, ax, ay = s13 + s79, m13 - m79, m13 + m79, s13 - s79
    ex, ey, dxe, dye = d4 + d6, d2 + d8, d6 - d4, d8 - d2
    s1011, m1110, s1213, m1213 = q10 + q11, q11 - q10, q12 + q13, q12 - q13
    s1415, m1415, s1617, m1716 = q14 + q15, q14 - q15, q16 + q17, q17 - q16
    F = lambda x: f32(x)
    c = [None] * 15
    c[1] = (F(2) * ax + F(19) * dxe - F(6) * s1011 + F(3) * s1213) * F(1 / 24)
    c[2] = (F(2) * ay + F(19) * dye + F(3) * s1415 - F(6) * s1617) * F(1 / 24)
    c[3] = (F(2) * ey + F(62) * ex - sc - F(18) * m1110) * F(1 / 48)
    c[4] = F(-0.375) * cx - F(0.625) * (m1213 + m1415)
    c[5] = (F(2) * ex + F(62) * ey - sc - F(18) * m1716) * F(1 / 48)
    c[6] = (F(4) * (s1011 - dxe) - ax - F(2) * s1213) * F(0.05)
    c[7] = F(-0.25) * ay - F(0.5) * dye
    c[8] = F(-0.25) * ax - F(0.5) * dxe
    c[9] = (F(4) * (s1617 - dye) - ay - F(2) * s1415) * F(0.05)
    c[10] = F(0.25) * m1110 - F(0.5) * ex
    c[11] = F(0.25) * cx + F(0.5) * m1213
    c[12] = F(0.25) * sc - F(0.5) * (ex + ey)
    c[13] = F(0.25) * cx + F(0.5) * m1415
    c[14] = F(0.25) * m1716 - F(0.5) * ey
    return c, (-d4, d6, -d2, d8), d


def _screen2(q, eps, pow2):
    """screen2's arithmetic (the moment form), elementwise in float32."""
    c, (dW, dE, dS, dN), d = _coef2_f32(q)
    S = np.zeros_like(q[0])
    for k in range(9):
        if k != 4:
            S = np.maximum(S, np.abs(d[k]))
    for k in range(9, 17):
        S = np.maximum(S, np.abs(q[k]))
    E = S * f32(2.0 ** -16)
    b0 = (c[1] * c[1] + c[2] * c[2] + c[4] * c[4]
          + f32(4) * (c[3] * c[3] + c[5] * c[5] + c[7] * c[7] + c[8] * c[8])
          + f32(36) * (c[6] * c[6] + c[9] * c[9] + c[11] * c[11] + c[13] * c[13])
          + f32(576) * (c[10] * c[10] + c[14] * c[14]) + f32(16) * c[12] * c[12])
    sq = (np.sqrt(b0.astype(np.float64)) * (1 - 2.0 ** -21)).astype(f32)
    D0 = f32(2.0 ** -18) * b0 + E * (f32(73) * sq + f32(1331) * E)
    bs = [b0, dW * dW + dS * dS, dE * dE + dS * dS, dE * dE + dN * dN, dW * dW + dN * dN]
    Ds = [D0] + [f32(2.0 ** -20) * b for b in bs[1:]]
    tau = f32(0.25) * ((np.abs(b0 - bs[1]) + np.abs(b0 - bs[2])) + (np.abs(b0 - bs[3]) + np.abs(b0 - bs[4])))
    ut = tau * (f32(1) + f32(2.0 ** -20)) + D0 + f32(0.25) * ((Ds[1] + Ds[2]) + (Ds[3] + Ds[4]))
    L = b0 - D0
    for m in range(1, 5):
        L = np.minimum(L, bs[m] - Ds[m])
    L = np.maximum(L, f32(0))
    dlo = (L * L if pow2 else L) + f32(eps)
    return ut * ut < f32(2.0 ** -25) * dlo


def _exact_a2(q, eps, pow2):
    """a_m from the same FP32 inputs in FP64, through the oracle's Step 1 maps
    (the appendix), beta_0 = sum (m! n! c)^2, beta_m = slope^2 sums."""
    import oracle
    G0, Gm = oracle.coef_maps_2d()
    Q = q.astype(np.float64)
    c = G0 @ Q
    fact = [1, 1, 1, 2, 1, 2, 6, 2, 2, 6, 24, 6, 4, 6, 24]
    b0 = sum((fact[l] * c[l]) ** 2 for l in range(1, 15))
    soff = [[(0, 0), (-1, 0), (0, -1)], [(0, 0), (1, 0), (0, -1)], [(0, 0), (1, 0), (0, 1)], [(0, 0), (-1, 0), (0, 1)]]
    bm = []
    for m in range(4):
        a3 = np.stack([Q[(dy + 1) * 3 + (dx + 1)] for dx, dy in soff[m]])
        cm = Gm[m] @ a3
        bm.append(cm[1] ** 2 + cm[2] ** 2)
    beta = [b0] + bm
    tau = 0.25 * sum(np.abs(b0 - b) for b in bm)
    return np.max([tau * tau / ((b * b if pow2 else b) + eps) for b in beta], axis=0)


def _stencils2(rng, n):
    out = []
    offs = [(-1, -1), (0, -1), (1, -1), (-1, 0), (0, 0), (1, 0), (-1, 1), (0, 1), (1, 1)]
    fn = [(-1, 0), (1, 0), (0, -1), (0, 1)]
    for h in (1e-1, 1e-2, 1e-3, 1e-4):
        x, y = rng.uniform(0, 10, n), rng.uniform(0, 10, n)
        kx, ky = rng.uniform(0.3, 5, n), rng.uniform(0.3, 5, n)
        amp, off, ph = rng.uniform(0.01, 2, n), rng.uniform(-10, 10, n), rng.uniform(0, 6.3, n)
        sx, sy = np.sinc(kx * h / 2 / np.pi), np.sinc(ky * h / 2 / np.pi)

        def avg(i, j):
            return off + amp * np.sin(kx * (x + i * h) + ky * (y + j * h) + ph) * sx * sy

        def vbar(i, j):   # cell mean of d u / d xi = h u_x
            return h * amp * kx * np.cos(kx * (x + i * h) + ky * (y + j * h) + ph) * sx * sy

        def wbar(i, j):
            return h * amp * ky * np.cos(kx * (x + i * h) + ky * (y + j * h) + ph) * sx * sy
        q = [avg(i, j) for i, j in offs] + [vbar(i, j) for i, j in fn] + [wbar(i, j) for i, j in fn]
        out.append(np.stack(q))
    base = rng.uniform(-1e3, 1e3, n)
    t = rng.normal(0, 1e-4, (17, n))
    out.append(np.concatenate([base + t[:9], t[9:]]))
    out.append(rng.normal(0, 1, (17, n)))
    jump = np.zeros((17, n))
    jump[[2, 5, 8]] = 1.0
    out.append(jump + 1e-7 * rng.normal(size=(17, n)))
    s = 10.0 ** rng.uniform(-6, 6, n)
    r = rng.normal(0, 1, (17, n))
    out.append(np.concatenate([s * (1 + 1e-6 * r[:9]), s * 1e-6 * r[9:]]))
    return out


@pytest.mark.parametrize("eps", [1e-6, 1e-8, 1e-12])
@pytest.mark.parametrize("pow2", [False, True])
def test_screen2_bound_is_sound(eps, pow2):
    rng = np.random.default_rng(int(eps ** -0.25) * 3 + pow2)
    cleared = smooth_tiny = smooth_cleared = 0
    for q in _stencils2(rng, 4000):
        q = q.astype(f32)
        ok = _screen2(q, eps, pow2)
        a = _exact_a2(q, eps, pow2)
        assert np.all(a[ok] <= 2.0 ** -24), a[ok].max() / 2.0 ** -24
        cleared += int(ok.sum())
        tiny = a < 2.0 ** -40
        smooth_tiny += int(tiny.sum())
        smooth_cleared += int((ok & tiny).sum())
    assert cleared > 0
    assert smooth_cleared > 0.5 * smooth_tiny
