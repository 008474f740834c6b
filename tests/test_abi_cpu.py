"""The C-ABI library loads and exports every declared symbol; its argument
validation rejects bad problem statements before touching a GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

import __graft_entry__
from paper_2607_24325_b300 import hweno as hw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()


def _declared(checked_only=False):
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h") and (fn == "hweno_checked.h") == checked_only:
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(hweno_\w+)\s*\(", txt)
    return sorted(set(names))


def test_every_declared_symbol_is_exported():
    declared = _declared()
    assert declared, "no declarations found"
    out = subprocess.run(["nm", "-D", "--defined-only", hw.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(hweno_\w+)", out))
    missing = [n for n in declared if n not in exported]
    assert not missing, missing
    lib = hw.load()
    for n in declared:
        assert getattr(lib, n) is not None
    assert set(hw.EXPORTS) == set(declared)


def test_checked_build_exports_both_headers():
    """libhweno_checked.so: every entry point of the normal library plus the
    check-word readers of include/hweno_checked.h."""
    from paper_2607_24325_b300 import build as B
    declared = _declared() + _declared(checked_only=True)
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_CHECKED], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(hweno_\w+)", out))
    missing = [n for n in declared if n not in exported]
    assert not missing, missing
    plain = subprocess.run(["nm", "-D", "--defined-only", hw.LIB_PATH], capture_output=True, text=True,
                           check=True).stdout
    assert not [n for n in _declared(checked_only=True) if re.search(rf"\sT\s{n}\b", plain)]


def test_version_and_error_string():
    assert "sm_103a" in hw.hweno_version()
    assert isinstance(hw.hweno_last_error(), str)


BAD = [
    (dict(dim=3), "dim"),
    (dict(nx=2), "at least 3"),
    (dict(lin_w=(0.5, 0.3, 0.3)), "sum to 1"),
    (dict(lin_w=(1.0, 0.0, 0.0)), "positive"),
    (dict(bc=(hw.BC_PERIODIC, hw.BC_OUTFLOW, 0, 0)), "paired"),
    (dict(weight_pow=3), "weight_pow"),
    (dict(cfl=0.0), "cfl"),
    (dict(equation=7), "equation"),
    (dict(precision=5), "precision"),
    (dict(equation=hw.EQ_EULER, gamma_gas=1.0), "gamma_gas"),
    (dict(xhi=0.0), "domain"),
    (dict(bc=(hw.BC_SPLIT, hw.BC_OUTFLOW, 0, 0)), "2D grid"),
    (dict(bc=(hw.BC_OUTFLOW, 6, 0, 0)), "boundary"),
    (dict(smoothness=2), "smoothness"),
    (dict(xhi=float("inf")), "finite"),
    (dict(eps=float("inf")), "eps"),
    (dict(cfl=float("nan")), "cfl"),
    (dict(equation=hw.EQ_EULER, gamma_gas=float("inf")), "gamma_gas"),
    (dict(adv_x=float("nan")), "advection speeds"),
]


@pytest.mark.parametrize("kw,msg", BAD)
def test_create_rejects_bad_config(kw, msg):
    cfg = hw.Config(**{**dict(dim=1, nx=16), **kw})
    h = C.c_void_p()
    c = cfg.to_c()
    st = hw.load().hweno_create(C.byref(c), None, C.byref(h))
    assert st == hw.HWENO_ERR_ARG
    assert msg in hw.hweno_last_error()
    assert not h.value


def test_null_arguments_are_reported():
    lib = hw.load()
    assert lib.hweno_create(None, None, None) == hw.HWENO_ERR_ARG
    assert lib.hweno_set_state(None, None, 0) == hw.HWENO_ERR_ARG
    assert lib.hweno_advance(None, 1.0, 1, None, None) == hw.HWENO_ERR_ARG
    assert lib.hweno_batch_create(0, None, None, None) == hw.HWENO_ERR_ARG


def test_batch_rejects_mixed_parameters():
    a = hw.Config(dim=1, nx=16)
    b = hw.Config(dim=1, nx=32, equation=hw.EQ_BURGERS)
    arr = (hw.hweno_config * 2)(a.to_c(), b.to_c())
    h = C.c_void_p()
    assert hw.load().hweno_batch_create(2, arr, None, C.byref(h)) == hw.HWENO_ERR_ARG
    assert "batch-wide" in hw.hweno_last_error()
    c2 = hw.Config(dim=2, nx=8, ny=8, lin_w=(0.99, 0.0025, 0.0025, 0.0025, 0.0025))
    arr2 = (hw.hweno_config * 2)(c2.to_c(), a.to_c())
    assert hw.load().hweno_batch_create(2, arr2, None, C.byref(h)) == hw.HWENO_ERR_ARG
    assert "same dim" in hw.hweno_last_error()
    c3 = hw.Config(dim=2, nx=8, ny=8, lin_w=(0.98, 0.005, 0.005, 0.005, 0.005))
    arr3 = (hw.hweno_config * 2)(c2.to_c(), c3.to_c())
    assert hw.load().hweno_batch_create(2, arr3, None, C.byref(h)) == hw.HWENO_ERR_ARG
    assert "batch-wide" in hw.hweno_last_error()


def test_train_permutation_is_splitmix64_fisher_yates():
    """The training order restated from the published definitions: SplitMix64
    (Steele, Lea and Flood, 2014) from the state seed + (e + 1) *
    0xD1B54A32D192ED03, Fisher-Yates from the top index down with
    j = next() mod (i + 1).  Host code of the library; no GPU needed."""
    M = (1 << 64) - 1

    def perm(seed, e, n):
        st = (seed + (e + 1) * 0xD1B54A32D192ED03) & M
        out = list(range(n))
        for i in range(n - 1, 0, -1):
            st = (st + 0x9E3779B97F4A7C15) & M
            z = st
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
            z ^= z >> 31
            j = z % (i + 1)
            out[i], out[j] = out[j], out[i]
        return out
    from paper_2607_24325_b300 import hweno as hw
    for seed, e, n in [(0, 0, 1), (0, 0, 17), (77, 3, 1000), (2 ** 63 + 5, 1, 333)]:
        got = hw.hweno_train_permutation(seed, e, n)
        assert got.tolist() == perm(seed, e, n)
        assert sorted(got.tolist()) == list(range(n))
