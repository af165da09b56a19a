#!/usr/bin/env python
"""Benchmark of the multibody scattering hot path on GB300.

One step = the whole path on the 2D workload of 1000 bodies (circle /
3-star / ellipse, N = 64,000 skeleton points, kappa = 40, 8 plane waves):
scattering-matrix build on the device, layout, right-hand side, the
mixed-precision solve (FP32 GMRES inside FP64 iterative refinement) to a
relative residual of 1e-11, and the scattered field at 4096 far targets.

value = G_hat pair-interactions per second over the step (one pair = one
phi evaluation with its multiply-add into all 8 right-hand sides; every
operator application and the field evaluation count).  Under torchrun each
rank runs an independent replica (the path is not sharded across GPUs).

--config 2 / 3 runs the same measurement on the two largest single-GPU
workloads (2D, 10,000 bodies, N ~ 700k, 16 waves; 3D, 2000 ellipsoids,
N = 600,000, 4 waves).  Their solves need thousands of iterations, so one
step there is the S build, the right-hand side, a capped mixed solve (a fixed
number of block-GMRES steps and its FP64 residual) and the field; the line
reports the pair-interaction rate, the kernel roofline and the S-build time,
not a time to solution.

--impl reference times the CPU oracle (numpy/scipy FP64) on a bounded
sample of the same workload with the same metric.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Ĝ pair-interactions/s; time-to-1e-9 mixed vs FP64 on GB300; served p50/p99"
UNIT = "pair-interactions/s"
WORKLOADS = {
    1: ("2D sound-soft, 1000 bodies (circle, 3-star, ellipse 1:0.6; radius 1) on a jittered "
        "32x32 lattice in a 100x100 box, random rotations, kappa=40, m=128 n=64 k=64 p=129 "
        "per body (N=64,000), 8 plane waves; mixed FP32/FP64-IR solve to rel. residual 1e-11"),
    2: ("2D sound-soft, 10,000 bodies of radius U(0.5,1.5) (circle, 3-star, ellipse) on a jittered "
        "100x100 lattice in a 400x400 box, kappa=20, k=clamp(3.5 kappa rho, 32, 128), m=2k, n=k, "
        "p=2k+1 (N=700,230), 16 plane waves; S build of 10,000 unique shapes + capped mixed solve"),
    3: ("3D sound-soft, 2000 ellipsoids (semi-axes U(0.6,1.0)) on a jittered 13^3 lattice in a "
        "40^3 box, kappa=8, m=600 n=150 k=300 p=601 per body (N=600,000), 4 plane waves; "
        "S build of 2000 unique shapes + capped mixed solve"),
}
WORKLOAD = WORKLOADS[1]
# convention: one pair = one phi plus a complex multiply-add (8 flops) into every
# right-hand side; phi = 35 flops in 2D, 15 in 3D (FFMA = 2, special function = 1)
FLOPS_PER_PAIR = {2: lambda nrhs: 35 + 8 * nrhs, 3: lambda nrhs: 15 + 8 * nrhs}
FLOPS_PER_PAIR_2D = FLOPS_PER_PAIR[2]
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x 2 flop x max SM clock
# DRAM bytes (read + write) of one launch on this workload, from one ncu capture
# of the kernel as built (profiles/g_umma_kernel_2d_1000bodies_8rhs.md); null for
# kernels not captured at their workload's full size
TRAFFIC_BYTES = {"g_umma_kernel<2,8>": 34287360 + 269312}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mbs", choices=["mbs", "reference"])
    ap.add_argument("--config", type=int, default=1, choices=[1, 2, 3],
                    help="workload: 1 the 1000-body 2D headline workload (default), 2 the 10,000-body "
                         "2D workload, 3 the 2000-ellipsoid 3D workload")
    ap.add_argument("--capped-iters", type=int, default=20,
                    help="configs 2/3: block-GMRES steps of the capped mixed solve in each step")
    ap.add_argument("--tol", type=float, default=None,
                    help="relative residual of the solve: default 1e-11 on the 1000-body workload, "
                         "1e-9 (the metric's accuracy) on the two large ones")
    ap.add_argument("--restart", type=int, default=200)
    ap.add_argument("--fp64-kernel", type=int, default=2, choices=[0, 1, 2],
                    help="FP64-accurate G_hat: 2 automatic (default: double-float on the FP32 pipe where "
                         "the solve's tolerance allows it), 1 double-float, 0 FP64 pipe")
    ap.add_argument("--inner-tol", type=float, default=1e-4,
                    help="relative tolerance of each FP32 inner solve of the mixed refinement "
                         "(1e-4 reaches 1e-11 in 3 sweeps with the fewest inner iterations)")
    ap.add_argument("--targets", type=int, default=4096)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 time-to-solution solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--e2e-steps", type=int, default=1,
                    help="steps of the end-to-end (host buffers) measurement")
    ap.add_argument("--fp64-max-iter", type=int, default=8000,
                    help="iteration cap of the measured plain-FP64 solve (config 1)")
    ap.add_argument("--serve-requests", type=int, default=64,
                    help="requests of the served trace at full size (0 = skip serving)")
    ap.add_argument("--serve-tmax", type=int, default=3000)
    ap.add_argument("--serve-max-iter", type=int, default=20,
                    help="inner-iteration cap per served request of the full-size trace")
    ap.add_argument("--serve-policy", choices=["fifo", "sjf"], default="sjf",
                    help="admission order of the server: arrival order, or shortest estimated work first")
    ap.add_argument("--serve-compare", type=int, default=8,
                    help="requests of the body-count-20..300 trace served by both the mixed and the FP64 "
                         "path (0 = skip)")
    ap.add_argument("--mac", type=int, default=0,
                    help="FP32 G_hat kernel (mac_path option): 0 auto (tcgen05), 1 FP32 pipe, "
                         "2 mma.sync tensor-core multiply-add, 3 tcgen05 tensor-core multiply-add")
    ap.add_argument("--kernel", choices=["g32", "g64"], default=None,
                    help="only apply G_hat (FP32 or FP64) to nrhs random vectors, steps times "
                         "(for profiling the dominant kernel); prints per-launch times")
    ap.add_argument("--bodies", type=int, default=0,
                    help="with --kernel: the first B bodies of the workload only (small profiling case)")
    ap.add_argument("--solve-only", action="store_true",
                    help="build S and run one solve of the workload with the bench's solver options "
                         "(for profiling the Krylov kernels); prints its time and counts, not a bench line")
    return ap.parse_args()


def _serve_trace(pkg, mi, trace, tol, slots, policy=0, fp64=False, max_iter=0, log=None):
    """Replay requests against the continuous-batching server at their arrival
    times; latency = completion - arrival (submission)."""
    import numpy as np
    work = [(r, mi.request_workload(r)) for r in trace]
    data = [(r, wl, wl.boundary_data()) for r, wl in work]
    srv = pkg.Server(max_active=slots)
    srv.set_policy(policy)
    t0 = time.perf_counter()
    ids = []
    for r, wl, v in data:
        delay = r.arrival - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        ids.append((r, srv.submit(wl, v, tol=tol, fp64=fp64, max_iter=max_iter)))
    srv.drain()
    res = [(r, srv.poll(rid)) for r, rid in ids]
    srv.close()
    ok = [(r, x) for r, x in res if x["done"] == 1]
    lat = np.array([x["t_end"] - x["t_submit"] for _, x in ok])
    waits = np.array([x["t_start"] - x["t_submit"] for _, x in ok])
    serv = np.array([x["t_end"] - x["t_start"] for _, x in ok])
    for r, x in ok:
        if log is not None:
            print(f"{log}: rid={r.rid} dim={r.dim} T={r.T} N={x['N']} nrhs={r.nrhs} kappa={r.kappa:.1f} "
                  f"iterations={x['inner_iterations']} converged={x['converged']} "
                  f"wait_s={x['t_start'] - x['t_submit']:.2f} service_s={x['t_end'] - x['t_start']:.2f}",
                  file=sys.stderr)
    # device-side overlap: the requests' device intervals (events on their own
    # streams) and their G_hat kernel time
    iv = sorted((x["dev_start"], x["dev_end"]) for _, x in ok if x["dev_end"] > x["dev_start"])
    edges = sorted([(s0, 1) for s0, _ in iv] + [(e0, -1) for _, e0 in iv])
    union = multi = 0.0
    depth, last = 0, None
    for t, d in edges:
        if last is not None and depth >= 1:
            union += t - last
            if depth >= 2:
                multi += t - last
        depth += d
        last = t
    busy = sum(x["g_busy_ms"] for _, x in ok) / 1e3
    first = min(x["t_submit"] for _, x in res) if res else 0.0
    done_t = [x["t_end"] for _, x in ok]
    return {"requests": len(res), "failed": len(res) - len(ok),
            "converged": int(sum(x["converged"] for _, x in ok)),
            "mean_wait_s": float(waits.mean()) if len(ok) else None,
            "mean_service_s": float(serv.mean()) if len(ok) else None,
            "p50_s": float(np.percentile(lat, 50)) if len(ok) else None,
            "p99_s": float(np.percentile(lat, 99)) if len(ok) else None,
            "solves_per_s": len(done_t) / (max(done_t) - first) if done_t else None,
            "overlap_fraction": multi / union if union > 0 else 0.0,
            "g_busy_over_device_union": busy / union if union > 0 else None}


def run_serving(a, pkg, mi):
    """The serving trace (exponential arrivals at 20/s, T ~ U{20..3000}, 2D/3D
    mix 70/30, kappa ~ U(5, 50), 1..32 right-hand sides): the first
    serve_requests requests at full size under an inner-iteration cap, and,
    on the same trace with body counts 20..300 so that both paths converge,
    the mixed and the plain FP64 path to 1e-9."""
    slots = 4
    policy = {"fifo": 0, "sjf": 1}[a.serve_policy]
    trace = mi.serving_trace(seed=0, n=a.serve_requests, Tmin=20, Tmax=a.serve_tmax)
    full = _serve_trace(pkg, mi, trace, 1e-9, slots, policy=policy, max_iter=a.serve_max_iter,
                        log="served")
    full["trace"] = (f"first {len(trace)} requests of the seed-0 trace: arrivals at 20/s, T ~ U{{20..{a.serve_tmax}}}, "
                     f"2D/3D 70/30, kappa ~ U(5,50), nrhs ~ U{{1..32}}; mixed precision to rel. residual 1e-9 "
                     f"with at most {a.serve_max_iter} inner iterations per request (time-to-solution capped: "
                     f"the full trace is hours of GPU work); {slots} slots, admission "
                     f"{'shortest estimated work first' if policy else 'in arrival order'}")
    out = {"full_shape": full}
    if a.serve_compare > 0:
        small = mi.serving_trace(seed=0, n=a.serve_compare, Tmin=20, Tmax=300)
        cmp = {}
        for name, fp64 in (("mixed", False), ("fp64", True)):
            cmp[name] = _serve_trace(pkg, mi, small, 1e-9, slots, policy=policy, fp64=fp64,
                                     log=f"served_{name}")
        out["mixed_vs_fp64"] = {
            "trace": f"first {len(small)} requests of the seed-0 trace with T ~ U{{20..300}}, solved to 1e-9 "
                     f"(no cap), {slots} slots, the same arrivals for both paths",
            "p50_mixed_s": cmp["mixed"]["p50_s"], "p99_mixed_s": cmp["mixed"]["p99_s"],
            "p50_fp64_s": cmp["fp64"]["p50_s"], "p99_fp64_s": cmp["fp64"]["p99_s"],
            "mixed": cmp["mixed"], "fp64": cmp["fp64"]}
    out["p50_s"], out["p99_s"] = full["p50_s"], full["p99_s"]
    out["overlap_fraction"] = full["overlap_fraction"]
    return out


def run_solve_only(a):
    import numpy as np
    import torch

    import mbs_inputs as mi
    import __graft_entry__
    __graft_entry__.build()
    import paper_2603_19113_gb300 as pkg

    wl = {1: mi.config1, 2: mi.config2, 3: mi.config3}[a.config]()
    stream = torch.cuda.current_stream()
    ctx = pkg.Context(wl.dim, wl.kappa, precision=pkg.PREC_MIXED, tol=a.tol, inner_tol=a.inner_tol,
                      restart=a.restart, fp64_kernel=a.fp64_kernel, max_iter=50000, max_sweeps=12,
                      stream=stream.cuda_stream, mac_path=a.mac)
    ctx.build_scattering_matrices(wl)
    v = torch.from_numpy(np.ascontiguousarray(wl.boundary_data().T)).cuda().T
    b = ctx.rhs(v)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, info = ctx.solve(b)
    torch.cuda.synchronize()
    out = {"solve_only": True, "config": a.config, "restart": a.restart, "tol": a.tol,
           "solve_s": time.perf_counter() - t0}
    out.update(info)
    print(json.dumps(out), flush=True)
    ctx.close()


def run_kernel_only(a):
    import numpy as np
    import torch

    import mbs_inputs as mi
    import __graft_entry__
    __graft_entry__.build()
    import paper_2603_19113_gb300 as pkg

    wl = {1: mi.config1, 2: mi.config2, 3: mi.config3}[a.config]()
    if a.bodies:
        wl = wl.subset(range(a.bodies))
    stream = torch.cuda.current_stream()
    ctx = pkg.Context(wl.dim, wl.kappa, stream=stream.cuda_stream, mac_path=a.mac, fp64_kernel=a.fp64_kernel)
    ctx.build_scattering_matrices(wl)
    q = torch.randn(wl.nrhs, ctx.N, dtype=torch.complex128, device="cuda").T
    prec = pkg.PREC_FP32 if a.kernel == "g32" else pkg.PREC_FP64
    for _ in range(a.warmup):
        ctx.apply_G(q, prec)
    ctx.profile(True)
    ctx.kernel_times()
    for _ in range(a.steps):
        ctx.apply_G(q, prec)
    kt = ctx.kernel_times()
    _, off, _ = ctx.get_layout()
    pairs = ctx.N * ctx.N - int(np.sum(np.diff(off).astype(np.int64) ** 2))
    ms = kt["g32_ms"] / max(1, kt["g32_launches"]) if a.kernel == "g32" else kt["g64_ms"] / max(1, kt["g64_launches"])
    print(json.dumps({"kernel": a.kernel, "config": a.config, "bodies": wl.T, "mac_path": a.mac,
                      "fp64_kernel": a.fp64_kernel, "N": ctx.N, "nrhs": wl.nrhs, "pairs_per_launch": pairs,
                      "ms_per_launch": ms, "pairs_per_s": pairs / (ms / 1e3), **kt}), flush=True)


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl"
        try:
            import torch
            if not torch.cuda.is_available():
                backend = "gloo"
        except Exception:
            backend = "gloo"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x, ws, device=None):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x, ws, device=None):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def _oracle_rows(args):
    import oracle as orc
    xyz, body, q, rows, kappa, dim = args
    t0 = time.perf_counter()
    orc.G_rows(dim, kappa, xyz, body, q, rows)
    return time.perf_counter() - t0


def oracle_sample_setup(seed=0, config=1):
    """Skeleton layout of the workload for timing the oracle's G_hat rows.  The
    1000-body workload takes the oracle's own skeletons; for the two large ones
    (10,000 and 2000 unique shapes) every other collocation point stands in for
    the skeleton, which leaves the number of pairs per row unchanged."""
    import numpy as np
    import mbs_inputs as mi
    import oracle as orc
    wl = {1: mi.config1, 2: mi.config2, 3: mi.config3}[config](seed=seed)
    if config == 1:
        sdata = orc.build_all(wl)
    else:
        sdata = [{"skel": np.arange(0, 2 * sh.k, 2)} for sh in wl.shapes]
    lay = orc.layout(wl, sdata)
    rng = np.random.default_rng(1)
    N = lay["xhat"].shape[0]
    q = rng.normal(size=(N, wl.nrhs)) + 1j * rng.normal(size=(N, wl.nrhs))
    return wl, lay, q


def oracle_pairs_per_s(pool, nproc, wl, lay, q, rows_total, seed=2):
    """Time the oracle's G_hat rows on a random sample of target rows, spread
    over a process pool; returns (pairs/s, seconds, rows)."""
    import numpy as np
    N = lay["xhat"].shape[0]
    rows = np.sort(np.random.default_rng(seed).choice(N, rows_total, replace=False))
    chunks = np.array_split(rows, nproc * 2)
    t0 = time.perf_counter()
    list(pool.map(_oracle_rows, [(lay["xhat"], lay["body"], q, c, wl.kappa, wl.dim) for c in chunks]))
    dt = time.perf_counter() - t0
    counts = np.bincount(lay["body"])
    pairs = int(np.sum(N - counts[lay["body"][rows]]))
    return pairs / dt, dt, rows_total


def make_pool():
    import multiprocessing as mp
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    ctx = mp.get_context("spawn")
    return ctx.Pool(n), n


# ---------------------------------------------------------------------------
# reference arm
# ---------------------------------------------------------------------------
def run_reference(a, ws, rank):
    if rank != 0:
        return
    pool, nproc = make_pool()
    wl, lay, q = oracle_sample_setup(config=a.config)
    N = lay["xhat"].shape[0]
    # rows of the large workloads hold ~10x the sources: fewer rows per step
    rows = max(64, 16 * nproc) if a.config == 1 else max(32, 2 * nproc)
    for _ in range(a.warmup):
        oracle_pairs_per_s(pool, nproc, wl, lay, q, rows, seed=10)
    t0 = time.perf_counter()
    rates = []
    for s in range(a.steps):
        r, dt, _ = oracle_pairs_per_s(pool, nproc, wl, lay, q, rows, seed=20 + s)
        rates.append(r)
    total = time.perf_counter() - t0
    pool.close()
    value = statistics.mean(rates)
    sample = f"oracle G_hat rows: {rows} random target rows x {N:,} sources x {wl.nrhs} RHS per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * total / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOADS[a.config], "reference": "CPU oracle (numpy/scipy)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nproc, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_mbs(a, ws, rank, local):
    pool = None
    nproc = 0
    if rank == 0 and not a.no_cpu:
        pool, nproc = make_pool()  # spawn before any CUDA work
    import numpy as np
    import torch

    import mbs_inputs as mi
    import __graft_entry__
    __graft_entry__.build()
    import paper_2603_19113_gb300 as pkg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    cfg = a.config
    capped = cfg != 1
    wl = {1: mi.config1, 2: mi.config2, 3: mi.config3}[cfg](seed=rank)
    dim = wl.dim
    v_host = wl.boundary_data()
    tg_host = mi.far_targets(wl, a.targets, mode="ring")
    M = tg_host.shape[0]
    nrhs = wl.nrhs
    # device-resident inputs (column-major (rows, nrhs) complex128; targets (M, dim))
    v_dev = torch.from_numpy(np.ascontiguousarray(v_host.T)).to(dev).T
    tg_dev = torch.from_numpy(np.ascontiguousarray(tg_host.T)).to(dev).T
    # pinned host inputs for the end-to-end measurement
    v_pin = torch.from_numpy(np.ascontiguousarray(v_host.T)).pin_memory().T
    tg_pin = torch.from_numpy(np.ascontiguousarray(tg_host.T)).pin_memory().T
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    opts = dict(precision=pkg.PREC_MIXED, tol=a.tol, inner_tol=a.inner_tol, restart=a.restart,
                fp64_kernel=a.fp64_kernel, max_iter=50000, max_sweeps=12, stream=stream.cuda_stream,
                mac_path=a.mac)
    if capped:
        # a fixed amount of solve work per step: capped_iters block-GMRES steps in
        # one refinement sweep, then its FP64 residual
        opts.update(max_iter=a.capped_iters, max_sweeps=1, restart=max(a.capped_iters, 1))
    ctx = pkg.Context(dim, wl.kappa, **opts)
    build_s = []

    def step(v, tg):
        t0 = time.perf_counter()
        ctx.build_scattering_matrices(wl)  # returns after the device work
        build_s.append(time.perf_counter() - t0)
        b = ctx.rhs(v)
        q, info = ctx.solve(b, raise_on_noconv=not capped)
        u = ctx.evaluate_field(tg, q)
        return info, u

    ctx.build_scattering_matrices(wl)
    N = ctx.N
    _, off, _ = ctx.get_layout()
    kb = np.diff(off)
    pairs_mv = N * N - int(np.sum(kb.astype(np.int64) ** 2))
    for _ in range(a.warmup):
        flush.zero_()
        info, _ = step(v_dev, tg_dev)
    build_s.clear()

    # ---- timed region: device-resident inputs ----
    sampler = ClockSampler(local)
    ctx.profile(True)
    ctx.kernel_times()
    torch.cuda.synchronize(dev)
    barrier(ws)
    sampler.start()
    l0 = pkg.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    pairs = 0
    infos = []
    u_mixed = None
    for _ in range(a.steps):
        flush.zero_()
        info, u_mixed = step(v_dev, tg_dev)
        infos.append(info)
        pairs += (info["matvecs_fp32"] + info["matvecs_fp64"]) * pairs_mv + M * N
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(ws)
    launches = pkg.launch_count() - l0
    clocks = sampler.stop()
    kt = ctx.kernel_times()
    ctx.profile(False)
    ms = e0.elapsed_time(e1)
    ms_max = reduce_max(ms, ws, dev)
    pairs_all = reduce_sum(pairs, ws, dev)
    value = pairs_all / (ms_max / 1e3)

    # ---- end to end through the C ABI with pinned host buffers ----
    barrier(ws)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e_pairs = 0
    h2d = d2h = 0
    e_steps = min(a.steps, a.e2e_steps)
    for _ in range(e_steps):
        flush.zero_()
        ctx.build_scattering_matrices(wl)
        b = ctx.rhs(v_pin)                 # H2D v, D2H b
        q, info = ctx.solve(b, raise_on_noconv=not capped)  # H2D b (and x0), D2H q
        u = ctx.evaluate_field(tg_pin, q)  # H2D targets and q, D2H u
        e_pairs += (info["matvecs_fp32"] + info["matvecs_fp64"]) * pairs_mv + M * N
        h2d += v_pin.numel() * 16 + 2 * b.numel() * 16 + q.numel() * 16 + tg_pin.numel() * 8
        d2h += b.numel() * 16 + q.numel() * 16 + u.numel() * 16
    torch.cuda.synchronize(dev)
    e_dt = reduce_max(time.perf_counter() - t0, ws, dev)
    e_value = reduce_sum(e_pairs, ws, dev) / e_dt

    t2s = {"mixed_s": statistics.mean(i["seconds"] for i in infos),
           "mixed_inner_iterations": infos[-1]["inner_iterations"],
           "mixed_sweeps": infos[-1]["sweeps"], "mixed_rel_residual": infos[-1]["rel_residual"],
           "mixed_fp64_kernel": "double-float" if infos[-1]["fp64_kernel"] else "FP64 pipe",
           "tol": a.tol}
    if capped:
        t2s = {"capped_solve_s": t2s["mixed_s"], "block_gmres_steps": infos[-1]["inner_iterations"],
               "rel_residual_after_cap": infos[-1]["rel_residual"],
               "fp64_kernel": t2s["mixed_fp64_kernel"],
               "note": "time to solution not measured on this workload: thousands of iterations"}
    if cfg == 1 and not a.no_fp64 and rank == 0:
        # ---- the plain FP64 path to the same tolerance, measured (one solve) ----
        ctx64 = pkg.Context(2, wl.kappa, precision=pkg.PREC_FP64, tol=a.tol, restart=a.restart,
                            fp64_kernel=a.fp64_kernel, max_iter=a.fp64_max_iter, stream=stream.cuda_stream)
        ctx64.build_scattering_matrices(wl)
        b64 = ctx64.rhs(v_dev)
        q64, i64 = ctx64.solve(b64, raise_on_noconv=False)
        u64 = ctx64.evaluate_field(tg_dev, q64)
        ctx64.close()
        t2s.update({"fp64_s": i64["seconds"], "fp64_iterations": i64["inner_iterations"],
                    "fp64_rel_residual": i64["rel_residual"], "fp64_converged": bool(i64["converged"]),
                    "fp64_kernel": "double-float" if i64["fp64_kernel"] else "FP64 pipe",
                    "fp64_over_mixed": i64["seconds"] / t2s["mixed_s"],
                    "field_rel_err_vs_fp64": float((u_mixed - u64).abs().max() / u64.abs().max()),
                    "field_targets": M})
        # both paths to convergence on the 10-body workload as well
        wl0 = mi.config0()
        v0 = torch.from_numpy(np.ascontiguousarray(wl0.boundary_data().T)).to(dev).T
        tg0 = torch.from_numpy(np.ascontiguousarray(mi.far_targets(wl0, 256).T)).to(dev).T
        res0 = {}
        for name, prec in (("fp64", pkg.PREC_FP64), ("mixed", pkg.PREC_MIXED)):
            c0 = pkg.Context(2, wl0.kappa, precision=prec, tol=a.tol, restart=a.restart,
                             stream=stream.cuda_stream)
            c0.build_scattering_matrices(wl0)
            q0, i0 = c0.solve(c0.rhs(v0))
            res0[name] = (i0, c0.evaluate_field(tg0, q0))
            c0.close()
        u64, umx = res0["fp64"][1], res0["mixed"][1]
        t2s["config0"] = {"fp64_s": res0["fp64"][0]["seconds"], "mixed_s": res0["mixed"][0]["seconds"],
                          "fp64_iterations": res0["fp64"][0]["inner_iterations"],
                          "mixed_inner_iterations": res0["mixed"][0]["inner_iterations"],
                          "mixed_vs_fp64_field_rel_err":
                              float((u64 - umx).abs().max() / u64.abs().max())}

    # ---- roofline of the dominant kernel (FP32 G_hat) ----
    flops_launch = pairs_mv * FLOPS_PER_PAIR[dim](nrhs)
    avg_ms = kt["g32_ms"] / max(1, kt["g32_launches"])
    achieved = flops_launch / (avg_ms / 1e3) / 1e12
    nr = 16 if nrhs >= 16 else 8
    kname = {1: f"g_f32_kernel<{dim},{min(nrhs, 8)},2>", 2: f"g_tc_kernel<{dim},1>",
             3: f"g_umma_kernel<{dim},{nr}>"}.get(kt["g32_path"], "unknown")
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved,
                "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                "traffic": TRAFFIC_BYTES.get(kname) if cfg == 1 else None, "avg_launch_ms": avg_ms,
                "launches": kt["g32_launches"], "nsplit": kt["g32_nsplit"],
                "flops_per_launch": flops_launch,
                "pairs_per_s": pairs_mv / (avg_ms / 1e3),
                "peak_note": "FP32 SIMT peak from unit counts: 152 SMs x 128 lanes x 2 x 2070 MHz; the "
                             "convention counts the complex multiply-add (8 flops per RHS) against it, "
                             "though in g_umma_kernel that part runs on the tensor cores, so with many "
                             "RHS the fraction can exceed 1"}
    share = kt["g32_ms"] / ms if ms > 0 else None
    g64_share = kt["g64_ms"] / ms if ms > 0 else None

    served = None
    if rank == 0 and a.serve_requests > 0 and cfg == 1:
        served = run_serving(a, pkg, mi)

    cpu = None
    if pool is not None:
        import oracle  # noqa: F401  (test infrastructure: CPU baseline leg only)
        wlo, lay, qo = oracle_sample_setup(config=cfg)
        rows = max(64, 32 * nproc) if cfg == 1 else max(32, 4 * nproc)
        # one untimed pass first: the spawned workers import numpy, scipy and the oracle
        oracle_pairs_per_s(pool, nproc, wlo, lay, qo, 2 * nproc, seed=3)
        rate, dt, _ = oracle_pairs_per_s(pool, nproc, wlo, lay, qo, rows)
        pool.close()
        cpu = {"value": rate, "unit": UNIT, "cores": nproc, "kind": "oracle",
               "sample": f"oracle G_hat rows: {rows} random target rows x {N:,} sources x {nrhs} RHS "
                         f"({dt:.1f} s wall on {nproc} processes)"}

    if rank == 0:
        config = {"workload": WORKLOADS[cfg], "N": N, "pairs_per_matvec": pairs_mv, "nrhs": nrhs,
                  "field_targets": M, "restart": opts["restart"], "inner_tol": a.inner_tol,
                  "fp64_kernel": {0: "FP64 pipe", 1: "double-float on the FP32 pipe",
                                  2: "automatic (double-float where the tolerance allows)"}[a.fp64_kernel],
                  "l2": "256 MiB buffer written before every step",
                  "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"}
        if capped:
            config["capped_solve"] = f"{a.capped_iters} block-GMRES steps + 1 FP64 residual per step"
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": config,
            "e2e": {"value": e_value, "unit": UNIT, "h2d_bytes_per_step": h2d // max(1, e_steps),
                    "d2h_bytes_per_step": d2h // max(1, e_steps), "steps": e_steps},
            "roofline": roofline,
            "g32_time_share": share,
            "g64_time_share": g64_share,
            "s_build_s": statistics.mean(build_s) if build_s else None,
            "time_to_solution": t2s,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": launches,
            "served": served,
        }
        print(json.dumps(line), flush=True)
    ctx.close()


def main():
    a = parse()
    if a.tol is None:
        a.tol = 1e-11 if a.config == 1 else 1e-9
    ws, rank, local = dist_setup()
    if a.kernel:
        run_kernel_only(a)
    elif a.solve_only:
        run_solve_only(a)
    elif a.impl == "reference":
        run_reference(a, ws, rank)
    else:
        run_mbs(a, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
