"""The double-float G_hat matvec (csrc/gdf_core.h with phi_df.h), run as a
host loop in the order a kernel takes it, against the oracle's FP64 matvec
(Sec. 1 eq. Gmtx-entries): per body pair FP64 work (centre difference, the
phase kappa |D| mod 2 pi in double-double), per point pair double-float
arithmetic (phase split, phi, compensated multiply-add).  At kappa = 40 over
a 100 x 100 box the oracle itself carries ~1e-13 against 30-digit references,
and so does this path; the bound is 5e-13 (1e-12 for the kappa-37.3 case,
whose kappa is not a float)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import mbs_inputs as mi
import oracle as orc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HARNESS = os.path.join(ROOT, "tests", "gdf_harness.cpp")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = tmp_path_factory.mktemp("gdf") / "libgdf_test.so"
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-fno-fast-math", "-ffp-contract=off", HARNESS, "-o", str(out)],
                   check=True, capture_output=True)
    L = ctypes.CDLL(str(out))
    D, I64 = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
    L.gdf_matvec.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, I64, D, D, ctypes.c_int, D, D]
    L.gdf_matvec.restype = ctypes.c_int64
    return L


def _config1_subset(kappa):
    wl = mi.config1(kappa=kappa)
    pick = np.random.default_rng(4).choice(wl.T, 24, replace=False)
    return wl.subset(pick)


CASES = {
    "2d": (lambda: mi.tiny_2d(seed=3, T=6, kappa=6.0, nrhs=3), 5e-13, False),
    "2d_small_kappa_r": (lambda: mi.tiny_2d(seed=3, T=6, kappa=1.5, nrhs=3), 5e-13, True),
    "3d": (lambda: mi.tiny_3d(), 5e-13, False),
    "2d_kappa40_box100": (lambda: _config1_subset(40.0), 5e-13, False),
    "2d_kappa37.3_box100": (lambda: _config1_subset(37.3), 1e-12, False),
}


@pytest.mark.parametrize("case", list(CASES))
def test_double_float_matvec_matches_fp64_oracle(lib, case):
    make, bound, expect_fallback = CASES[case]
    wl = make()
    lay = orc.layout(wl, orc.build_all(wl))
    xh, body, off = lay["xhat"], lay["body"], lay["offsets"].astype(np.int64)
    N, d, nr = xh.shape[0], wl.dim, 3
    cen = np.ascontiguousarray(wl.centres, dtype=np.float64)
    delta = np.zeros((N, 3))
    delta[:, :d] = xh - wl.centres[body, :d]
    rng = np.random.default_rng(7)
    q = rng.normal(size=(N, nr)) + 1j * rng.normal(size=(N, nr))
    qa = np.ascontiguousarray(q.T).view(np.float64).ravel()
    y = np.zeros_like(qa)
    P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    nfb = lib.gdf_matvec(d, wl.kappa, wl.T, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), P(cen),
                         P(np.ascontiguousarray(delta)), nr, P(qa), P(y))
    assert (nfb > 0) == expect_fallback
    ydf = y.view(np.complex128).reshape(nr, N).T
    yref = orc.G_matvec(d, wl.kappa, xh, body, q)
    err = np.max(np.abs(ydf - yref)) / np.max(np.abs(yref))
    assert err < bound, err
