"""Host logic of block GMRES (restarted GMRES of Sec. 2.4 with s right-hand
sides per block): the incremental Givens reduction of the block Hessenberg
least-squares problem and its back substitution (csrc/blsq.cpp), compiled for
the host and checked against numpy's dense least squares after every step."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2603_19113_gb300", "csrc", "blsq.cpp")
HARNESS = os.path.join(ROOT, "tests", "blsq_harness.cpp")


@pytest.fixture(scope="module")
def blsq(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = tmp_path_factory.mktemp("blsq") / "libblsq_test.so"
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", HARNESS, SRC, "-o", str(out)],
                   check=True, capture_output=True)
    lib = ctypes.CDLL(str(out))
    P = ctypes.POINTER(ctypes.c_double)
    lib.blsq_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P, P, P, P]
    lib.blsq_run.restype = ctypes.c_int
    return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _cplx(rng, *shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def _upper(rng, s):
    R = np.triu(_cplx(rng, s, s))
    R[np.diag_indices(s)] = np.abs(rng.normal(size=s)) + 0.5  # CholQR factors: positive real diagonal
    return R


def _run(lib, s, restart, H, R0, beta, nsteps):
    hc, rk = [], []
    for j in range(nsteps):
        K = (j + 1) * s
        hc.append(np.ascontiguousarray(H[:K, j * s:(j + 1) * s].T).ravel())   # column-major K x s
        rk.append(np.ascontiguousarray(H[K:K + s, j * s:(j + 1) * s].T).ravel())
    hc = np.ascontiguousarray(np.concatenate(hc)).view(np.float64)
    rk = np.ascontiguousarray(np.concatenate(rk)).view(np.float64)
    r0 = np.ascontiguousarray(R0.T).ravel().view(np.float64)
    resid = np.zeros(nsteps * s)
    Y = np.zeros(2 * nsteps * s * s)
    assert lib.blsq_run(s, restart, nsteps, _ptr(r0), _ptr(beta), _ptr(hc), _ptr(rk),
                        _ptr(resid), _ptr(Y)) == 0
    return resid.reshape(nsteps, s), Y.view(np.complex128).reshape(s, nsteps * s).T


def _block_hessenberg(rng, s, nsteps, zero_last=False):
    H = np.zeros(((nsteps + 1) * s, nsteps * s), complex)
    for j in range(nsteps):
        K = (j + 1) * s
        H[:K, j * s:(j + 1) * s] = _cplx(rng, K, s)
        H[K:K + s, j * s:(j + 1) * s] = 0.0 if (zero_last and j == nsteps - 1) else _upper(rng, s)
    return H


@pytest.mark.parametrize("s,nsteps,restart", [(1, 9, 9), (2, 7, 10), (3, 6, 6), (8, 5, 12), (16, 3, 4)])
def test_block_lsq_matches_dense_least_squares(blsq, s, nsteps, restart):
    rng = np.random.default_rng(100 * s + nsteps)
    H = _block_hessenberg(rng, s, nsteps)
    R0, beta = _upper(rng, s), rng.uniform(0.5, 2.0, s)
    G0 = np.zeros(((nsteps + 1) * s, s), complex)
    G0[:s] = R0 * beta[None, :]
    resid, Y = _run(blsq, s, restart, H, R0, beta, nsteps)
    for n in range(1, nsteps + 1):
        Hn, Gn = H[:(n + 1) * s, :n * s], G0[:(n + 1) * s]
        Yn = np.linalg.lstsq(Hn, Gn, rcond=None)[0]
        ref = np.linalg.norm(Gn - Hn @ Yn, axis=0)
        assert np.allclose(resid[n - 1], ref, rtol=1e-10, atol=1e-12 * np.linalg.norm(G0)), (n, resid[n - 1], ref)
        if n == nsteps:
            assert np.max(np.abs(Y - Yn)) < 1e-10 * np.max(np.abs(Yn))


def test_block_lsq_breakdown_block(blsq):
    """A last block with R_k = 0 (the new block adds no direction, the
    solution lies in the space): the reduction still matches least squares."""
    rng = np.random.default_rng(7)
    s, nsteps = 3, 4
    H = _block_hessenberg(rng, s, nsteps, zero_last=True)
    R0, beta = _upper(rng, s), np.ones(s)
    G0 = np.zeros(((nsteps + 1) * s, s), complex)
    G0[:s] = R0
    resid, Y = _run(blsq, s, nsteps, H, R0, beta, nsteps)
    Yn = np.linalg.lstsq(H, G0, rcond=None)[0]
    assert np.allclose(resid[-1], np.linalg.norm(G0 - H @ Yn, axis=0), atol=1e-10)
    assert np.max(np.abs(Y - Yn)) < 1e-9 * np.max(np.abs(Yn))
