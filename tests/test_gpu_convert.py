"""The integer-ALU FP32 <-> FP64 conversions of the mixed-precision path
against IEEE 754 (numpy's conversions): widening must be exact and
narrowing must round to nearest, ties to even, bit for bit — on special
values, every exponent, random bit patterns and constructed rounding ties."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_24325_b300 import hweno as hw   # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _floats(rng):
    special = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45, 1.1754942e-38,
                        1.17549435e-38, 3.4028235e38, -3.4028235e38, 0.1, 1.0 / 3.0], dtype=np.float32)
    bits = rng.integers(0, 2 ** 32, size=200_000, dtype=np.uint64).astype(np.uint32)
    every_exp = (np.arange(256, dtype=np.uint32) << 23) | np.uint32(0x2AAAAA)
    return np.concatenate([special, bits.view(np.float32), every_exp.view(np.float32),
                           (-every_exp.view(np.float32))])


def _doubles(rng):
    with np.errstate(over="ignore"):   # exponents past the FP32 range become infinities, then dropped
        f = np.ldexp(rng.uniform(1.0, 2.0, 50_000), rng.integers(-140, 130, 50_000)).astype(np.float32)
    f = f[np.isfinite(f) & (f != 0)]
    fd = f.astype(np.float64)
    half = np.spacing(np.abs(f)).astype(np.float64) / 2.0
    ties = fd + half                                    # exactly half-way: ties to even
    around = np.concatenate([np.nextafter(ties, np.inf), np.nextafter(ties, -np.inf)])
    rnd = np.ldexp(rng.uniform(-2.0, 2.0, 100_000), rng.integers(-160, 140, 100_000))
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 3.4028235677973366e38, 3.4028235e38 * 1.0000001,
                        1e-40, -1e-45, 1.1754943508222875e-38, 1.0, -1.0, 1e300, -1e-300])
    return np.concatenate([special, fd, ties, -ties, around, rnd])


def _same(got, ref):
    both_nan = np.isnan(got) & np.isnan(ref)
    same_bits = got.view(np.uint64 if got.dtype == np.float64 else np.uint32) == \
        ref.view(np.uint64 if ref.dtype == np.float64 else np.uint32)
    return both_nan | same_bits


def test_conversions_match_ieee():
    rng = np.random.default_rng(5)
    f = _floats(rng)
    d = _doubles(rng)
    n = max(f.size, d.size)
    f = np.resize(f, n)
    d = np.resize(d, n)
    wide, narrow = hw.hweno_selftest_convert(torch.from_numpy(f).cuda(), torch.from_numpy(d).cuda())
    w = wide.cpu().numpy()
    nr = narrow.cpu().numpy()
    with np.errstate(invalid="ignore"):   # NaN payloads among the random bit patterns
        ok_w = _same(w, f.astype(np.float64))
    with np.errstate(over="ignore"):
        ref_n = d.astype(np.float32)
    ok_n = _same(nr, ref_n)
    assert ok_w.all(), f[~ok_w][:8]
    assert ok_n.all(), d[~ok_n][:8]


def test_conversion_rejects_bad_args():
    with pytest.raises(Exception):
        hw.hweno_selftest_convert(torch.zeros(3, device="cuda"), torch.zeros(4, dtype=torch.float64, device="cuda"))


def test_rcp64_faithful():
    """The FP64 kernels' reciprocal (Newton-Raphson from the hardware's
    approximate FP64 reciprocal) is within one unit in the last place of the
    correctly rounded 1/x (numpy's IEEE division) wherever x and 1/x are
    normal, of either sign; zeros, infinities and NaN give IEEE's results,
    subnormal arguments and results are flushed (+-inf, +-0)."""
    rng = np.random.default_rng(11)
    sig = rng.uniform(1.0, 2.0, 400_000)
    x = np.ldexp(sig, rng.integers(-1022, 1023, sig.size)) * rng.choice([-1.0, 1.0], sig.size)
    # next to powers of two, and a fine walk over one binade's significands
    p2 = np.ldexp(1.0, np.arange(-1022, 1023, 3))
    walk = 1.0 + np.arange(1, 8192) * 2.0 ** -13 + rng.uniform(-1, 1, 8191) * 2.0 ** -40
    edge = np.concatenate([np.nextafter(p2, 0.0), p2, np.nextafter(p2, np.inf), walk])
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324, 2.2250738585072009e-308,
                        2.2250738585072014e-308, -2.2250738585072014e-308, 4.450147717014403e-308,
                        1.7976931348623157e308, -1.7976931348623157e308, 8.98846567431158e307,
                        4.49423283715579e307, 1.0, -1.0, 0.1, 3.0, 1.4])
    x = np.concatenate([special, edge, -edge, x])
    y = hw.hweno_selftest_rcp64(torch.from_numpy(x).cuda()).cpu().numpy()
    tiny = 2.2250738585072014e-308
    with np.errstate(divide="ignore", over="ignore"):
        ref = 1.0 / x
    ref = np.where(np.abs(x) < tiny, np.copysign(np.inf, x), ref)            # subnormal argument
    ref = np.where((np.abs(ref) < tiny) & (ref != 0), np.copysign(0.0, ref), ref)  # subnormal result
    both_nan = np.isnan(y) & np.isnan(ref)
    same_sign = np.signbit(y) == np.signbit(ref)
    ulps = np.abs(y.view(np.int64) - ref.view(np.int64))
    ok = both_nan | (same_sign & (ulps <= 1))
    assert ok.all(), (x[~ok][:6], y[~ok][:6], ref[~ok][:6])
    # exactly representable quotients (powers of two, +-1) and the special values are exact
    exact = np.isin(np.arange(x.size), np.arange(special.size)) & ~np.isin(x, [0.1, 3.0, 1.4])
    assert (both_nan | (ulps == 0))[exact].all()
    assert (ulps[~np.isnan(ref)] == 0).mean() > 0.9
