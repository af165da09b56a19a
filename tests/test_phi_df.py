"""The fundamental solution in double-float arithmetic (csrc/phi_df.h),
compiled for the host, against 40-digit mpmath: sin/cos of angles up to
6400 rad to 1e-14 absolute, and phi_kappa (3D: e^{i kappa r}/(4 pi r); 2D:
(i/4) H0(kappa r) from the FP64 modulus/phase fits) with the body-pair phase
split to 3e-12 relative at kappa <= 40, R <= 140.  The bound follows from the
phase kappa (r - R), up to ~130 rad, carried at 2^-48 relative through a few
operations; the FP64 kernel's phase kappa r ~ 5600 carries 1e-12 as well."""
import ctypes
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HARNESS = os.path.join(ROOT, "tests", "phi_df_harness.cpp")
mp = pytest.importorskip("mpmath")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = tmp_path_factory.mktemp("phidf") / "libphidf_test.so"
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-fno-fast-math", "-ffp-contract=off", HARNESS, "-o", str(out)],
                   check=True, capture_output=True)
    L = ctypes.CDLL(str(out))
    F, I = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int)
    L.phi_df_batch.argtypes = [ctypes.c_int, ctypes.c_int, F, F, I]
    L.sincos_df_batch.argtypes = [ctypes.c_int, F, F]
    return L


def _f32(x):
    return struct.unpack("f", struct.pack("f", float(x)))[0]


def _df(x):
    x = mp.mpf(x)
    hi = _f32(x)
    return hi, _f32(x - mp.mpf(hi))


def _val(hi, lo):
    return mp.mpf(float(hi)) + mp.mpf(float(lo))


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def test_sincos_double_float(lib):
    mp.mp.dps = 40
    rng = np.random.default_rng(0)
    th = np.concatenate([rng.uniform(-6400, 6400, 600), rng.uniform(-4, 4, 200),
                         (np.arange(-40, 40) * np.pi / 2)])  # near the reduction boundaries
    n = th.size
    inp = np.array([_df(t) for t in th], np.float32).ravel()
    out = np.zeros(4 * n, np.float32)
    lib.sincos_df_batch(n, _fp(inp), _fp(out))
    err = 0
    for i in range(n):
        t = _val(inp[2 * i], inp[2 * i + 1])
        err = max(err, abs(_val(out[4 * i], out[4 * i + 1]) - mp.sin(t)),
                  abs(_val(out[4 * i + 2], out[4 * i + 3]) - mp.cos(t)))
    assert err < 1e-14, float(err)


@pytest.mark.parametrize("dim", [3, 2])
def test_phi_double_float_with_phase_split(lib, dim):
    mp.mp.dps = 40
    rng = np.random.default_rng(10 + dim)
    n = 400
    rows = []
    for _ in range(n):
        kappa, R, delta = rng.uniform(1, 40), rng.uniform(2.5, 140), rng.uniform(-3, 3)
        s = 2 * R * delta + delta * delta * rng.uniform(0.2, 1)
        kd, Rd, sd = _df(kappa), _df(R), _df(s)
        ph0 = mp.fmod(_val(*kd) * _val(*Rd) + (mp.pi / 4 if dim == 2 else 0), 2 * mp.pi)
        rows.append((kd, Rd, sd, _df(ph0)))
    inp = np.array([[a for pair in r for a in pair] for r in rows], np.float32).ravel()
    out = np.zeros(4 * n, np.float32)
    ok = np.zeros(n, np.int32)
    lib.phi_df_batch(dim, n, _fp(inp), _fp(out), ok.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    worst, nok = 0, 0
    for i in range(n):
        if not ok[i]:
            continue
        nok += 1
        kd, Rd, sd, pd = rows[i]
        k, R, s, p0 = _val(*kd), _val(*Rd), _val(*sd), _val(*pd)
        r = mp.sqrt(R * R + s)
        # the phase exactly as the split inputs define it (p0 is kappa R [+ pi/4]
        # mod 2 pi up to its own double-float rounding)
        shift = p0 - mp.fmod(k * R + (mp.pi / 4 if dim == 2 else 0), 2 * mp.pi)
        ref = (mp.exp(1j * (k * r + shift)) / (4 * mp.pi * r) if dim == 3
               else 0.25j * mp.hankel1(0, k * r) * mp.exp(1j * shift))
        got = mp.mpc(_val(out[4 * i], out[4 * i + 1]), _val(out[4 * i + 2], out[4 * i + 3]))
        worst = max(worst, abs(got - ref) / abs(ref))
    assert nok > 0.9 * n
    assert worst < 3e-12, float(worst)
