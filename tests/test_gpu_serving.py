"""Serving (continuous batching) on the GPU: every request's result is the same
alone and in a mix of concurrently running requests, and matches a direct
solve through a context."""
import numpy as np
import pytest

import mbs_inputs as mi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2603_19113_gb300 as p
    return p


def _requests():
    trace = mi.serving_trace(seed=5, n=6, Tmin=20, Tmax=120, p2d=1.0)
    out = []
    for r in trace:
        r.kappa = 5.0 + r.kappa % 10.0  # keep the test's iteration counts small
        wl = mi.request_workload(r)
        out.append((wl, wl.boundary_data()))
    return out


def test_each_result_is_the_same_alone_and_in_the_mix(pkg):
    reqs = _requests()
    alone = []
    srv = pkg.Server(max_active=1)
    for wl, v in reqs:
        rid = srv.submit(wl, v, tol=1e-9)
        srv.drain()
        res = srv.poll(rid, want_solution=True)
        assert res["done"] == 1, res
        alone.append(res["qhat"])
    srv.close()
    srv = pkg.Server(max_active=4)
    ids = [srv.submit(wl, v, tol=1e-9) for wl, v in reqs]
    srv.drain()
    for i, rid in enumerate(ids):
        res = srv.poll(rid, want_solution=True)
        assert res["done"] == 1, res
        q = res["qhat"]
        assert np.max(np.abs(q - alone[i])) <= 1e-12 * np.max(np.abs(alone[i]))
        assert res["t_start"] >= res["t_submit"] and res["t_end"] >= res["t_start"]
    srv.close()
    # and the same as a direct solve through a context
    wl, v = reqs[0]
    ctx = pkg.Context(2, wl.kappa, precision=pkg.PREC_MIXED, tol=1e-9)
    ctx.build_scattering_matrices(wl)
    q, info = ctx.solve(ctx.rhs(v))
    assert np.max(np.abs(q - alone[0])) <= 1e-12 * np.max(np.abs(q))


def test_admission_by_memory_budget(pkg):
    """With a budget below one request's footprint, requests still finish one at
    a time (an oversized request runs alone); nothing is dropped."""
    reqs = _requests()[:3]
    srv = pkg.Server(max_active=3, hbm_budget=1 << 20)
    ids = [srv.submit(wl, v, tol=1e-8) for wl, v in reqs]
    srv.drain()
    spans = []
    for rid in ids:
        res = srv.poll(rid)
        assert res["done"] == 1
        spans.append((res["t_start"], res["t_end"]))
    spans.sort()
    for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
        assert s1 >= e0 - 1e-6  # serialised by the budget
    srv.close()
