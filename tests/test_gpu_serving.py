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


def test_fp64_requests_iteration_caps_and_device_timings(pkg):
    """A request may take the plain FP64 path (its result matches the mixed
    one to the tolerance and a direct FP64 solve exactly), an iteration cap
    ends a solve early with converged = 0 and no error, and every finished
    request reports its device interval (events on its own stream) and its
    G_hat kernel time, which lies inside that interval."""
    reqs = _requests()[:3]
    srv = pkg.Server(max_active=3)
    ids_mixed = [srv.submit(wl, v, tol=1e-10) for wl, v in reqs]
    ids_fp64 = [srv.submit(wl, v, tol=1e-10, fp64=True) for wl, v in reqs]
    id_cap = srv.submit(reqs[0][0], reqs[0][1], tol=1e-12, max_iter=3)
    srv.drain()
    for rm, rf, (wl, v) in zip(ids_mixed, ids_fp64, reqs):
        a, b = srv.poll(rm, want_solution=True), srv.poll(rf, want_solution=True)
        assert a["done"] == 1 and b["done"] == 1 and a["converged"] == 1 and b["converged"] == 1
        assert np.max(np.abs(a["qhat"] - b["qhat"])) <= 1e-8 * np.max(np.abs(b["qhat"]))
        for res in (a, b):
            assert 0.0 <= res["dev_start"] < res["dev_end"]
            assert 0.0 < res["g_busy_ms"] <= 1e3 * (res["dev_end"] - res["dev_start"]) * 1.01
    cap = srv.poll(id_cap)
    assert cap["done"] == 1 and cap["converged"] == 0 and cap["inner_iterations"] <= 3
    srv.close()
    wl, v = reqs[1]
    ctx = pkg.Context(2, wl.kappa, precision=pkg.PREC_FP64, tol=1e-10)
    ctx.build_scattering_matrices(wl)
    q, _ = ctx.solve(ctx.rhs(v))
    srv = pkg.Server(max_active=1)
    rid = srv.submit(wl, v, tol=1e-10, fp64=True)
    srv.drain()
    assert np.array_equal(srv.poll(rid, want_solution=True)["qhat"], q)
    srv.close()


def test_shortest_work_first_admission(pkg):
    """Policy 1 admits the queued request of least estimated work first: with
    one slot, a large request submitted first runs first (the queue was empty),
    and of the two queued behind it the smaller (20 bodies) runs before the
    larger (90 bodies), which was submitted earlier."""
    trace = mi.serving_trace(seed=5, n=3, Tmin=20, Tmax=120, p2d=1.0)
    # the first request runs for a while (400 bodies at kappa = 25), so the
    # other two are both queued when the slot frees
    sizes = [(400, 25.0, 8), (90, 6.0, 2), (20, 6.0, 2)]
    reqs = []
    for r, (T, kap, nr) in zip(trace, sizes):
        r.T, r.kappa, r.nrhs = T, kap, nr
        wl = mi.request_workload(r)
        reqs.append((wl, wl.boundary_data()))
    srv = pkg.Server(max_active=1)
    srv.set_policy(1)
    ids = [srv.submit(*reqs[0], tol=1e-8)]
    import time
    t0 = time.time()
    while srv.poll(ids[0])["t_start"] == 0.0 and time.time() - t0 < 60:
        time.sleep(0.001)
    ids += [srv.submit(wl, v, tol=1e-8) for wl, v in reqs[1:]]
    srv.drain()
    start = [srv.poll(i)["t_start"] for i in ids]
    assert start[0] < start[2] < start[1]
    srv.close()
