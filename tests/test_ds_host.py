"""The double-single helpers of the complex128 fused pass, on the host.

The fused complex128 pass splits every double amplitude into two floats,
applies the gates with error-free transformations in single precision and
joins the result back into doubles (qs_ds.cuh).  These functions are written
for host and device alike; here their host build is checked against exact
rational arithmetic (fractions.Fraction), without a GPU:

  * split: h + l equals d truncated to 48 significant bits (|d - h - l| <=
    2^-47 |d|), h is d truncated to 24 bits; tiny and zero inputs;
  * join: the double nearest h + l (within half a unit in the last place),
    including the case below a power of two where the spacing halves;
  * the complex 2x2 row a x + b y (also with real a, b: the row of a real
    gate such as RY), the complex product and the butterfly: errors within a
    few units of 2^-48 of the terms' magnitudes.
"""
import ctypes
import math
import os
import shutil
import subprocess
from fractions import Fraction as F

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_quant_ph_0201042_gb300", "csrc")


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("ds") / "libds_shim.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(ROOT, "tests", "ds_shim.cpp"), "-o", out], check=True)
    L = ctypes.CDLL(out)
    f4 = ctypes.POINTER(ctypes.c_float)
    L.shim_split.argtypes = [ctypes.c_double, f4, f4]
    L.shim_split_const.argtypes = [ctypes.c_double, f4, f4]
    L.shim_join.argtypes = [ctypes.c_float, ctypes.c_float]
    L.shim_join.restype = ctypes.c_double
    L.shim_cmad2.argtypes = [f4] * 5
    L.shim_rmad2.argtypes = [f4] * 5
    L.shim_cmul.argtypes = [f4] * 3
    L.shim_butterfly.argtypes = [f4, f4]
    L.shim_mul1.argtypes = [ctypes.c_float] * 4 + [f4, f4]
    return L


def split(L, d):
    h, l = ctypes.c_float(), ctypes.c_float()
    L.shim_split(d, ctypes.byref(h), ctypes.byref(l))
    return h.value, l.value


def split_const(L, d):
    h, l = ctypes.c_float(), ctypes.c_float()
    L.shim_split_const(d, ctypes.byref(h), ctypes.byref(l))
    return h.value, l.value


def arr(v):
    return (ctypes.c_float * 4)(*[float(np.float32(x)) for x in v])


def val(h, l):
    return F(h) + F(l)


def test_split_is_a_48_bit_truncation(shim):
    r = np.random.default_rng(1)
    cases = [0.0, -0.0, 1.0, -1.0, 0.5, 2.0 ** -15, 1 / 3, -2 / 3, math.pi / 8, 2.0 ** -126, -2.0 ** -74,
             2.0 ** -73 * 1.7, 1.0 - 2.0 ** -53, np.nextafter(1.0, 0.0)]
    cases += list(r.uniform(-1, 1, 2000)) + list(r.standard_normal(500) * 2.0 ** -20)
    cases += list(np.ldexp(r.uniform(0.5, 1, 300), r.integers(-120, 0, 300)))
    for d in cases:
        d = float(d)
        h, l = split(shim, d)
        assert np.float32(h) == h and np.float32(l) == l
        if abs(d) < 2.0 ** -126:
            assert h == 0 and l == 0
            continue
        # h: d truncated to 24 significant bits, same sign
        m, e = math.frexp(d)
        assert F(h) == F(math.trunc(m * 2 ** 24)) * F(2) ** (e - 24)
        err = abs(F(d) - val(h, l))
        if abs(d) >= 2.0 ** -74:
            assert err <= F(abs(d)) * F(2) ** -47, d
        else:
            assert l == 0 and err <= F(2) ** -97


def test_join_rounds_to_nearest(shim):
    r = np.random.default_rng(2)
    for _ in range(3000):
        e = int(r.integers(-60, 1))
        h = float(np.float32(np.ldexp(r.uniform(0.5, 1.0), e) * (1 if r.random() < 0.5 else -1)))
        ulp = float(np.spacing(np.float32(abs(h))))
        l = float(np.float32(r.uniform(-0.5, 0.5) * ulp))
        exact = val(h, l)
        got = shim.shim_join(h, l)
        # within half a double ulp of the exact sum
        assert abs(F(got) - exact) <= F(float(np.spacing(abs(got)))) / 2, (h, l)


def test_join_below_a_power_of_two(shim):
    # h = 2^e with a negative l: the result lies in the binade below, where
    # the double spacing halves
    for e in (-1, -15, -30):
        for k in (1, 3, 1000, 2 ** 20):
            h = 2.0 ** e
            l = float(np.float32(-k * 2.0 ** (e - 52)))
            want = F(h) + F(l)
            got = shim.shim_join(h, l)
            assert abs(F(got) - want) <= F(2) ** (e - 54), (e, k)
            got = shim.shim_join(-h, -l)
            assert abs(F(got) + want) <= F(2) ** (e - 54), (e, k)


def test_join_of_split_round_trips(shim):
    r = np.random.default_rng(3)
    for d in list(r.uniform(-1, 1, 2000)) + list(r.standard_normal(200) * 1e-9):
        d = float(d)
        h, l = split(shim, d)
        got = shim.shim_join(h, l)
        assert abs(got - d) <= abs(d) * 2.0 ** -47


def ds_of(L, z):
    rh, rl = split_const(L, z.real)
    ih, il = split_const(L, z.imag)
    return [rh, rl, ih, il]


def cval(v):
    return (val(v[0], v[1]), val(v[2], v[3]))


def test_cmad2_cmul_butterfly_accuracy(shim):
    r = np.random.default_rng(4)
    out = (ctypes.c_float * 4)()
    for _ in range(1500):
        a, b = (complex(*r.standard_normal(2)) for _ in range(2))
        x, y = (complex(*r.standard_normal(2)) * 10.0 ** r.uniform(-6, 0) for _ in range(2))
        A, B, X, Y = (ds_of(shim, z) for z in (a, b, x, y))
        shim.shim_cmad2(arr(A), arr(X), arr(B), arr(Y), out)
        (ar, ai), (br, bi), (xr, xi), (yr, yi) = (cval(v) for v in (A, B, X, Y))
        want_r = ar * xr - ai * xi + br * yr - bi * yi
        want_i = ar * xi + ai * xr + br * yi + bi * yr
        scale = F(abs(a) * abs(x) + abs(b) * abs(y))
        assert abs(val(out[0], out[1]) - want_r) <= scale * F(2) ** -45
        assert abs(val(out[2], out[3]) - want_i) <= scale * F(2) ** -45
        # the result is normalised: |low| <= half a float ulp of the high part
        assert abs(out[1]) <= float(np.spacing(np.float32(abs(out[0])))) / 2
        shim.shim_cmul(arr(A), arr(X), out)
        assert abs(val(out[0], out[1]) - (ar * xr - ai * xi)) <= F(abs(a) * abs(x)) * F(2) ** -46
        assert abs(val(out[2], out[3]) - (ar * xi + ai * xr)) <= F(abs(a) * abs(x)) * F(2) ** -46
        px, py = arr(X), arr(Y)
        shim.shim_butterfly(px, py)
        s = F(abs(x) + abs(y))
        assert abs(val(px[0], px[1]) - (xr + yr)) <= s * F(2) ** -47
        assert abs(val(py[2], py[3]) - (xi - yi)) <= s * F(2) ** -47


def test_rmad2_real_row_accuracy(shim):
    # the row of a real 2x2 gate: a, b real; any imaginary part given is ignored
    r = np.random.default_rng(5)
    out = (ctypes.c_float * 4)()
    for _ in range(1500):
        a, b = r.standard_normal(2)
        x, y = (complex(*r.standard_normal(2)) * 10.0 ** r.uniform(-6, 0) for _ in range(2))
        junk = complex(0.0, float(r.standard_normal()))
        A, B, X, Y = (ds_of(shim, z) for z in (a + junk, b - junk, x, y))
        shim.shim_rmad2(arr(A), arr(X), arr(B), arr(Y), out)
        ar, br = val(A[0], A[1]), val(B[0], B[1])
        (xr, xi), (yr, yi) = cval(X), cval(Y)
        scale = F(abs(a) * abs(x) + abs(b) * abs(y))
        assert abs(val(out[0], out[1]) - (ar * xr + br * yr)) <= scale * F(2) ** -46
        assert abs(val(out[2], out[3]) - (ar * xi + br * yi)) <= scale * F(2) ** -46
        assert abs(out[1]) <= float(np.spacing(np.float32(abs(out[0])))) / 2
        assert abs(out[3]) <= float(np.spacing(np.float32(abs(out[2])))) / 2
    # a cancelling row: RY(pi/2) on (x, x) gives (0, sqrt(2) x) up to the error bound (the
    # low-order products are summed in order, so the cancelled row need not be exactly 0)
    c = 1 / math.sqrt(2)
    x = complex(0.3, -0.7)
    C, M, X = ds_of(shim, complex(c, 0)), ds_of(shim, complex(-c, 0)), ds_of(shim, x)
    shim.shim_rmad2(arr(C), arr(X), arr(M), arr(X), out)
    assert abs(val(out[0], out[1])) <= F(abs(x)) * F(2) ** -46
    assert abs(val(out[2], out[3])) <= F(abs(x)) * F(2) ** -46
    shim.shim_rmad2(arr(C), arr(X), arr(C), arr(X), out)
    want = 2 * val(C[0], C[1])
    assert abs(val(out[0], out[1]) - want * val(X[0], X[1])) <= F(abs(x)) * F(2) ** -46
    assert abs(val(out[2], out[3]) - want * val(X[2], X[3])) <= F(abs(x)) * F(2) ** -46


def test_scale_by_a_double_single_constant(shim):
    c = 1 / math.sqrt(2)
    ch, cl = split_const(shim, c)
    assert abs(val(ch, cl) - F(c)) <= F(c) * F(2) ** -48
    h, l = ctypes.c_float(), ctypes.c_float()
    for x in (1.0, 0.3, -2.0 ** -10):
        xh, xl = split(shim, x)
        shim.shim_mul1(xh, xl, ch, cl, ctypes.byref(h), ctypes.byref(l))
        assert abs(val(h.value, l.value) - val(xh, xl) * val(ch, cl)) <= F(abs(x)) * F(2) ** -46
