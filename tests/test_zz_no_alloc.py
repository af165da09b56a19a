"""The allocation-free G_hat entry point (mbs_apply_G_noalloc) against the
context-based one (mbs_apply_G), through the C ABI.

It serves callers that must not allocate device memory while they run
(fixed memory pools handed out at start-up, allocation-free real-time
loops).  This file is collected last on purpose, and it must pass both alone
in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import mbs_inputs as mi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2603_19113_gb300 as pkg
    return pkg, torch


def _device_layout(ctx, torch):
    N, off, xyz = ctx.get_layout()
    body = np.repeat(np.arange(len(off) - 1), np.diff(off)).astype(np.int32)
    dev = torch.device("cuda")
    return (N, torch.from_numpy(off).to(dev), torch.from_numpy(body).to(dev),
            torch.from_numpy(np.ascontiguousarray(xyz.T)).to(dev))


@pytest.mark.parametrize("make,dim", [(lambda: mi.tiny_2d(seed=1, T=9, kappa=6.0), 2),
                                      (lambda: mi.tiny_3d(seed=0, T=5, nth=10, nph=14, p=141, k=70), 3)])
def test_noalloc_matches_context_call_twice(env, make, dim):
    pkg, torch = env
    wl = make()
    ctx = pkg.Context(dim, wl.kappa)
    ctx.build_scattering_matrices(wl)
    N, off, body, xw = _device_layout(ctx, torch)
    rng = np.random.default_rng(3)
    qh = rng.normal(size=(N, 3)) + 1j * rng.normal(size=(N, 3))
    q = torch.from_numpy(np.ascontiguousarray(qh.T)).cuda().T
    ref = ctx.apply_G(q, pkg.PREC_FP64).cpu().numpy()
    for _ in range(2):  # the static scratch keeps the previous call's contents
        y = torch.full((3, N), float("nan"), dtype=torch.complex128, device="cuda").T
        pkg.api.apply_G_noalloc(dim, wl.kappa, off, body, xw, q, y)
        torch.cuda.synchronize()
        out = y.cpu().numpy()
        assert np.max(np.abs(out - ref)) / np.max(np.abs(ref)) < 1e-12
    ctx.close()


def test_noalloc_rejects_sizes_beyond_the_static_scratch(env):
    pkg, torch = env
    import ctypes as C
    lib = pkg.load_library()
    t = torch.zeros(8, dtype=torch.int64, device="cuda")
    p = C.c_void_p(t.data_ptr())
    # N * nrhs above the 64 MiB limit: rejected before anything is launched
    st = lib.mbs_apply_G_noalloc(2, 1.0, 4_000_000, 1, p, p, p, 2, p, p, None)
    assert st == 1
    # sizes whose product wraps around 64 bits (N = 2^40, nrhs = 2^24) are
    # rejected too, before any pointer is looked at
    st = lib.mbs_apply_G_noalloc(2, 1.0, 1 << 40, 1, p, p, p, 1 << 24, p, p, None)
    assert st == 1
