"""Double-float arithmetic (csrc/dfloat.h) compiled for the host: the
error-free transformations are exact, and every compound operation lies within
a small multiple of u^2 (u = 2^-24) of the exact result, computed in rational
arithmetic (or at 60 digits for division and square root)."""
import ctypes
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HARNESS = os.path.join(ROOT, "tests", "dfloat_harness.cpp")
U2 = 2.0 ** -48


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = tmp_path_factory.mktemp("dfloat") / "libdfloat_test.so"
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-fno-fast-math", "-ffp-contract=off", HARNESS, "-o", str(out)],
                   check=True, capture_output=True)
    L = ctypes.CDLL(str(out))
    for f, t in (("df_eft", ctypes.c_float), ("df_ops", ctypes.c_double)):
        getattr(L, f).argtypes = [ctypes.c_int, ctypes.POINTER(t), ctypes.POINTER(t),
                                  ctypes.POINTER(ctypes.c_float)]
    return L


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _F(x):
    return Fraction(float(x))


def test_error_free_transformations_are_exact(lib):
    rng = np.random.default_rng(1)
    n = 4000
    a = (rng.normal(size=n) * 10.0 ** rng.uniform(-8, 8, n)).astype(np.float32)
    b = (rng.normal(size=n) * 10.0 ** rng.uniform(-8, 8, n)).astype(np.float32)
    out = np.zeros(4 * n, np.float32)
    lib.df_eft(n, _p(a, ctypes.c_float), _p(b, ctypes.c_float), _p(out, ctypes.c_float))
    o = out.reshape(n, 4)
    for i in range(n):
        assert _F(o[i, 0]) + _F(o[i, 1]) == _F(a[i]) + _F(b[i])
        assert _F(o[i, 2]) + _F(o[i, 3]) == _F(a[i]) * _F(b[i])


def _run_ops(lib, a, b):
    n = a.size
    out = np.zeros(12 * n, np.float32)
    lib.df_ops(n, _p(a, ctypes.c_double), _p(b, ctypes.c_double), _p(out, ctypes.c_float))
    return out.reshape(n, 6, 2)


def _df(d):
    hi = np.float32(d)
    lo = np.float32(d - float(hi))
    return _F(hi) + _F(lo)


def test_compound_operations_within_their_bounds(lib):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    rng = np.random.default_rng(2)
    n = 3000
    a = rng.normal(size=n) * 10.0 ** rng.uniform(-6, 6, n)
    b = rng.normal(size=n) * 10.0 ** rng.uniform(-6, 6, n)
    # near-cancelling subtractions: b within a few ulps of a (relative to the result)
    b[:300] = a[:300] * (1 + rng.uniform(-1e-6, 1e-6, 300))
    o = _run_ops(lib, a, b)
    worst = np.zeros(6)
    for i in range(n):
        x, y = _df(a[i]), _df(b[i])
        got = [_F(o[i, k, 0]) + _F(o[i, k, 1]) for k in range(6)]
        exact = [x + y, x - y, x * y, None, None, x * _F(np.float32(b[i]))]
        for k in (0, 1, 2, 5):
            if exact[k] != 0:
                worst[k] = max(worst[k], abs(float((got[k] - exact[k]) / exact[k])))
        q = mpmath.mpf(x.numerator) / x.denominator / (mpmath.mpf(y.numerator) / y.denominator)
        worst[3] = max(worst[3], float(abs((mpmath.mpf(got[3].numerator) / got[3].denominator - q) / q)))
        ax = abs(x)
        r = mpmath.sqrt(mpmath.mpf(ax.numerator) / ax.denominator)
        worst[4] = max(worst[4], float(abs((mpmath.mpf(got[4].numerator) / got[4].denominator - r) / r)))
    bounds = np.array([3, 3, 6, 16, 8, 4]) * U2
    assert np.all(worst <= bounds), (worst / U2).round(2)
