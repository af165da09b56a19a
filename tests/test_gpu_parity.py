"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (derivations in the design notes):
  * FP64 kernels: 1e-12 relative to the largest output entry (rounding of sums
    of N terms with entries accurate to ~1e-15);
  * FP32 G_hat: 2e-5 norm-wise (per-entry phi error <= ~1e-6 from the phase
    split, the fitted modulus/phase and the hardware sine/cosine, with a
    cancellation allowance for the multi-body sum), and element-wise
    |y_i - ref_i| <= 2e-5 (|G| |q|)_i: every output entry within 2e-5 of the
    sum of the magnitudes of its terms.  Per term the FP32 error is <= ~1e-6
    relative (phi) plus the FP32 accumulation (16-source chunks, split partial
    sums: a random walk of ~sqrt(N) roundings of 6e-8, ~3e-6 for N = 2000);
    a wrong block of one body pair puts an error of the order of that block's
    share of the sum (>= 1e-2 here) on its rows;
  * solves: relative scattered-field error <= 1e-9 against the oracle (FP64
    and mixed precision), <= 1e-10 for FP64 with injected scattering data.
"""
import math

import numpy as np
import pytest

import geometries as geo
import mbs_inputs as mi
import oracle as orc

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


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _nrel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _erel(a, ref, absref):
    """Largest entry-wise error relative to the sum of term magnitudes."""
    return float(np.max(np.abs(a - ref) / absref))


def _abs_terms(G, q):
    return np.abs(G) @ np.abs(q)


def _abs_terms_rows(dim, kappa, xhat, body, q, rows, chunk=16):
    """(|G| |q|)[rows], G_hat's rows evaluated by the oracle's kernel (same-body
    entries, the zero diagonal blocks, set to zero)."""
    out = []
    aq = np.abs(q)
    for a in range(0, len(rows), chunk):
        r = np.asarray(rows[a:a + chunk])
        with np.errstate(all="ignore"):
            K = np.abs(orc.kernel_matrix(dim, kappa, xhat[r], xhat))
        K[body[r][:, None] == body[None, :]] = 0.0
        out.append(K @ aq)
    return np.concatenate(out)


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def _ctx_with_oracle_S(pkg, wl, **kw):
    sdata = orc.build_all(wl)
    ctx = pkg.Context(wl.dim, wl.kappa, **kw)
    ctx.build_scattering_matrices(wl)
    for s, sd in enumerate(sdata):
        if sd is not None:
            ctx.inject_scattering(s, sd["skel"], sd["S"], sd["W"])
    lay = orc.layout(wl, sdata)
    return ctx, sdata, lay


# --------------------------------------------------------------------------
# G_hat matvec (several tiles and a ragged tail; nrhs chunking)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("fp64_kernel", [0, 1])
@pytest.mark.parametrize("nrhs", [1, 3, 8, 17])
def test_G_2d_fp64_and_fp32(pkg, nrhs, fp64_kernel):
    """Both FP64-accurate kernels (FP64 pipe, double-float) and the FP32 one."""
    wl = mi.tiny_2d(seed=1, T=9, kappa=6.0, ks=(24, 37, 50))
    ctx, sdata, lay = _ctx_with_oracle_S(pkg, wl, fp64_kernel=fp64_kernel)
    assert ctx.N > 256 and ctx.N % 256 != 0
    q = _rand((ctx.N, nrhs), nrhs)
    G = orc.G_dense(2, wl.kappa, lay["xhat"], lay["body"])
    ref = G @ q
    y64 = ctx.apply_G(q, pkg.PREC_FP64)
    y32 = ctx.apply_G(q, pkg.PREC_FP32)
    assert _rel(y64, ref) < 1e-12
    assert _nrel(y32, ref) < 2e-5
    assert _erel(y32, ref, _abs_terms(G, q)) < 2e-5


@pytest.mark.parametrize("mac_path", [1, 2, 3])
@pytest.mark.parametrize("dim,nrhs,kappa", [(2, 8, 6.0), (2, 5, 6.0), (2, 16, 6.0), (2, 1, 6.0), (2, 8, 30.0),
                                            (2, 16, 30.0), (3, 8, 3.0), (3, 11, 3.0), (3, 2, 3.0)])
def test_G_fp32_multiply_add_paths(pkg, mac_path, dim, nrhs, kappa):
    """Every FP32 G_hat kernel (FP32 pipe; mma.sync and tcgen05 tensor-core
    multiply-add with the 3xTF32 split) against the oracle, with right-hand-side
    counts that fill, pad and span two blocks of right-hand sides (fewer than 4
    right-hand sides take the FP32 pipe on every path).  At kappa = 30 the
    nearest body pairs come to kappa r ~ 30 (the x >= 8 fit of H0) and the
    others stay beyond kappa r = 64 (the x >= 64 fit)."""
    wl = (mi.tiny_2d(seed=4, T=9, kappa=kappa, ks=(24, 37, 50)) if dim == 2
          else mi.tiny_3d(seed=1, T=5, kappa=kappa, nth=10, nph=14, p=141, k=70))
    ctx, sdata, lay = _ctx_with_oracle_S(pkg, wl, mac_path=mac_path)
    if kappa == 30.0:  # both fits occur
        cen, rho = wl.centres[:, :2], np.array([wl.shapes[s].bound_radius for s in wl.body_shape])
        gap = kappa * (np.linalg.norm(cen[:, None] - cen[None], axis=2) - rho[:, None] - rho[None])
        off = ~np.eye(wl.T, dtype=bool)
        assert gap[off].min() < 64.0 < gap[off].max()
    q = _rand((ctx.N, nrhs), 13)
    G = orc.G_dense(dim, wl.kappa, lay["xhat"], lay["body"])
    ref = G @ q
    y32 = ctx.apply_G(q, pkg.PREC_FP32)
    assert _nrel(y32, ref) < 2e-5
    assert _erel(y32, ref, _abs_terms(G, q)) < 2e-5


@pytest.mark.parametrize("mac_path", [1, 3])
def test_G_2d_small_arguments(pkg, mac_path):
    """Neighbouring bodies at low kappa put kappa r below 3 and between 3 and
    16: every branch of the H0 evaluation is exercised."""
    wl = mi.tiny_2d(seed=2, T=9, kappa=2.0, ks=(30, 41), spacing=2.9)
    ctx, sdata, lay = _ctx_with_oracle_S(pkg, wl, mac_path=mac_path)
    x = wl.kappa * np.linalg.norm(lay["xhat"][:, None] - lay["xhat"][None], axis=2)
    other = lay["body"][:, None] != lay["body"][None, :]
    assert x[other].min() < 3.0 and x[other].max() > 16.0
    q = _rand((ctx.N, 5), 7)
    G = orc.G_dense(2, wl.kappa, lay["xhat"], lay["body"])
    ref = G @ q
    assert _rel(ctx.apply_G(q, pkg.PREC_FP64), ref) < 1e-12
    y32 = ctx.apply_G(q, pkg.PREC_FP32)
    assert _nrel(y32, ref) < 2e-5
    assert _erel(y32, ref, _abs_terms(G, q)) < 2e-5


@pytest.mark.parametrize("fp64_kernel", [0, 1])
@pytest.mark.parametrize("nrhs", [1, 4])
def test_G_3d_fp64_and_fp32(pkg, nrhs, fp64_kernel):
    wl = mi.tiny_3d(seed=0, T=5, kappa=3.0, nth=10, nph=14, p=141, k=70)
    ctx, sdata, lay = _ctx_with_oracle_S(pkg, wl, fp64_kernel=fp64_kernel)
    q = _rand((ctx.N, nrhs), 11)
    G = orc.G_dense(3, wl.kappa, lay["xhat"], lay["body"])
    ref = G @ q
    assert _rel(ctx.apply_G(q, pkg.PREC_FP64), ref) < 1e-12
    y32 = ctx.apply_G(q, pkg.PREC_FP32)
    assert _nrel(y32, ref) < 2e-5
    assert _erel(y32, ref, _abs_terms(G, q)) < 2e-5


_DF_CASES = {
    "2d": lambda: mi.tiny_2d(seed=1, T=9, kappa=6.0, ks=(24, 37, 50)),
    "2d_small_kappa_r": lambda: mi.tiny_2d(seed=2, T=9, kappa=2.0, ks=(30, 41), spacing=2.9),
    "3d": lambda: mi.tiny_3d(seed=0, T=5, kappa=3.0, nth=10, nph=14, p=141, k=70),
}


@pytest.mark.parametrize("case,nrhs", [(c, 5) for c in _DF_CASES] + [("2d", 9), ("3d", 16)])
def test_G_fp64_double_float_kernel(pkg, case, nrhs):
    """The FP64-accurate G_hat in double-float arithmetic on the FP32 pipe
    (fp64_kernel = 1) against the oracle at the FP64-pipe kernel's bound: 2D in
    the fitted range and below it (the FP64 series), 3D; N not a multiple of
    the 128-target tile; 5 right-hand sides (one pass of 8), 9 (a second pass
    with one right-hand side) and 16 (two full passes)."""
    wl = _DF_CASES[case]()
    ctx, sdata, lay = _ctx_with_oracle_S(pkg, wl, fp64_kernel=1)
    q = _rand((ctx.N, nrhs), 21)
    ref = orc.G_dense(wl.dim, wl.kappa, lay["xhat"], lay["body"]) @ q
    assert _rel(ctx.apply_G(q, pkg.PREC_FP64), ref) < 1e-12


def test_mixed_solve_with_double_float_residuals(pkg):
    """Iterative refinement whose FP64 residuals come from the double-float
    kernel converges to the oracle's solution."""
    wl = mi.config0()
    ref = orc.solve_workload(wl)
    tg = mi.far_targets(wl, 128, mode="ring")
    u_ref = orc.field(2, wl.kappa, tg, ref["layout"]["xhat"], ref["q"])
    ctx, sdata, lay = _ctx_with_oracle_S(pkg, wl, precision=pkg.PREC_MIXED, tol=1e-11, fp64_kernel=1)
    q, info = ctx.solve(ref["b"])
    assert info["converged"] == 1
    assert _rel(ctx.evaluate_field(tg, q), u_ref) < 1e-9


def test_apply_operator_matches_oracle(pkg):
    wl = mi.config0()
    ctx, sdata, lay = _ctx_with_oracle_S(pkg, wl)
    q = _rand((ctx.N, 1), 3)
    ref = orc.apply_operator(wl, sdata, lay, q)
    assert _rel(ctx.apply_operator(q), ref) < 1e-12
    ctx.set_options(precision=pkg.PREC_FP32)
    assert _nrel(ctx.apply_operator(q), ref) < 2e-5


@pytest.mark.parametrize("mac_path,fp64_kernel", [(0, 0), (3, 1)])
def test_G_full_size_config1_sampled_rows(pkg, mac_path, fp64_kernel):
    """The bench workload (1000 bodies, N = 64,000, 8 right-hand sides, kappa = 40)
    in the bench's launch configuration: 256 sampled rows against the oracle.
    The skeleton is the oracle's (injected), so no oracle input comes from the
    GPU."""
    wl = mi.config1()
    ctx, sdata, lay = _ctx_with_oracle_S(pkg, wl, mac_path=mac_path, fp64_kernel=fp64_kernel)
    N = ctx.N
    assert N == 64000
    q = _rand((N, 8), 5)
    y64 = ctx.apply_G(q, pkg.PREC_FP64)
    y32 = ctx.apply_G(q, pkg.PREC_FP32)
    rows = np.random.default_rng(0).choice(N, 256, replace=False)
    ref = orc.G_rows(2, wl.kappa, lay["xhat"], lay["body"], q, rows)
    assert _rel(y64[rows], ref) < 1e-12
    assert _nrel(y32[rows], ref) < 2e-5
    absref = _abs_terms_rows(2, wl.kappa, lay["xhat"], lay["body"], q, rows)
    assert _erel(y32[rows], ref, absref) < 2e-5


# --------------------------------------------------------------------------
# right-hand side, solve, field
# --------------------------------------------------------------------------
def _inject_every_other_point(ctx, wl):
    """Skeleton = every other collocation point of each shape, S = 0.  The
    G_hat layout is then fixed by the inputs alone, so the oracle computes its
    own skeleton coordinates and takes nothing from the GPU."""
    sdata = []
    for s, sh in enumerate(wl.shapes):
        skel = np.arange(0, 2 * sh.k, 2, dtype=np.int32)
        assert skel[-1] < sh.m
        ctx.inject_scattering(s, skel, np.zeros((sh.k, sh.k), np.complex128))
        sdata.append({"skel": skel})
    return orc.layout(wl, sdata)


@pytest.mark.parametrize("name,rows", [("config2", 24), ("config3", 96)])
def test_G_full_size_sampled_rows_fp32(pkg, name, rows):
    """The two largest workloads at full size in their launch configuration:
    2D, 10,000 bodies of 35-105 skeleton points (ragged 16-point chunks),
    N ~ 700k, 16 right-hand sides (one 16-column tcgen05 block); 3D, 2000
    ellipsoids, N = 600,000, 4 right-hand sides (a padded 8-column block, or
    the FP32 pipe where the autotuner finds it faster).  Sampled rows of the
    FP32 G_hat against the oracle."""
    wl = getattr(mi, name)()
    ctx = pkg.Context(wl.dim, wl.kappa)
    ctx.build_scattering_matrices(wl)
    lay = _inject_every_other_point(ctx, wl)
    N = ctx.N
    assert N == lay["xhat"].shape[0] and N > 500_000
    q = _rand((N, wl.nrhs), 9)
    y32 = ctx.apply_G(q, pkg.PREC_FP32)
    sel = np.random.default_rng(1).choice(N, rows, replace=False)
    ref = orc.G_rows(wl.dim, wl.kappa, lay["xhat"], lay["body"], q, sel)
    assert _nrel(y32[sel], ref) < 2e-5
    absref = _abs_terms_rows(wl.dim, wl.kappa, lay["xhat"], lay["body"], q, sel)
    assert _erel(y32[sel], ref, absref) < 2e-5
    ctx.close()


def test_injected_solve_fp64_and_mixed_config0(pkg):
    wl = mi.config0()
    ref = orc.solve_workload(wl)
    tg = mi.far_targets(wl, 128, mode="ring")
    u_ref = orc.field(2, wl.kappa, tg, ref["layout"]["xhat"], ref["q"])
    for prec, tol in ((pkg.PREC_FP64, 1e-10), (pkg.PREC_MIXED, 1e-9)):
        ctx, sdata, lay = _ctx_with_oracle_S(pkg, wl, precision=prec, tol=1e-12)
        b = ctx.rhs(ref["v"])
        b_ref = orc.rhs(wl, sdata, lay, ref["v"], explicit_W=True)
        assert _rel(b, b_ref) < 1e-12
        q, info = ctx.solve(ref["b"])
        assert info["converged"] == 1
        assert _nrel(q, ref["q"]) < tol
        u = ctx.evaluate_field(tg, q)
        assert _rel(u, u_ref) < tol


@pytest.mark.parametrize("nrhs", [1, 2, 5, 8])
def test_mixed_solve_through_the_fp32_gram_schmidt_rings(pkg, nrhs):
    """Mixed solves whose FP32 block Gram-Schmidt runs on the tensor-copy ring
    kernels (even N, block width <= 8) at the shapes their boxes cut: N not a
    multiple of the 64-row stage, block widths 1-8, basis widths of 6 to 48
    columns (restart 6: below and across the 16- and 32-column boxes) and up
    to 320 (restart 40), against the oracle's dense solve with the same S."""
    wl = mi.tiny_2d(seed=2, T=9, kappa=6.0, nrhs=nrhs, ks=(24, 38, 50))
    ref = orc.solve_workload(wl)
    for restart in (6, 40):
        ctx, sdata, lay = _ctx_with_oracle_S(pkg, wl, precision=pkg.PREC_MIXED, tol=1e-12, restart=restart)
        assert ctx.N % 2 == 0 and ctx.N % 64 != 0
        q, info = ctx.solve(ref["b"])
        assert info["converged"] == 1
        assert _nrel(q, ref["q"]) < 1e-9
        ctx.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_block_gmres_graph_replay_matches_direct(pkg, prec):
    """Block GMRES steps replayed from captured CUDA graphs give bitwise the
    result of the same steps launched directly (short restart, so step graphs
    are reused across restart cycles and refinement sweeps)."""
    wl = mi.tiny_2d(seed=3, T=9, kappa=6.0, nrhs=3)
    p = pkg.PREC_MIXED if prec == "mixed" else pkg.PREC_FP64
    out = []
    for graphs in (1, 0):
        ctx = pkg.Context(2, wl.kappa, precision=p, tol=1e-10, restart=4, cuda_graphs=graphs)
        ctx.build_scattering_matrices(wl)
        b = ctx.rhs(wl.boundary_data())
        ctx.profile(True)  # G_hat timing events inside the step graphs
        q, info = ctx.solve(b)
        kt = ctx.kernel_times()
        assert info["converged"] == 1 and info["inner_iterations"] > 8
        assert kt["g32_launches"] + kt["g64_launches"] == info["matvecs_fp32"] + info["matvecs_fp64"]
        assert kt["g32_ms"] + kt["g64_ms"] > 0
        out.append(q)
        ctx.close()
    assert np.array_equal(out[0], out[1])


def test_evaluate_field_matches_oracle(pkg):
    wl = mi.tiny_2d(seed=3, T=7, kappa=5.0)
    ctx, sdata, lay = _ctx_with_oracle_S(pkg, wl)
    q = _rand((ctx.N, 3), 9)
    tg = mi.far_targets(wl, 300, mode="gaps", seed=4)
    ref = orc.field(2, wl.kappa, tg, lay["xhat"], q)
    assert _rel(ctx.evaluate_field(tg, q), ref) < 1e-12


def test_gpu_built_S_single_circle_closed_form(pkg):
    """GPU S build (pivoted QR, ID, least squares) for one circle: the field
    matches the separation-of-variables solution and the oracle."""
    from closed_forms import circle_scattered
    kappa = 10.0
    wl = mi.circle_single(kappa, m=128, eps=1e-12, proxy_factor=2.0)
    ctx = pkg.Context(2, kappa, tol=1e-13)
    ctx.build_scattering_matrices(wl)
    info = ctx.get_shape(0)
    sd = orc.build_all(wl)[0]
    assert np.array_equal(info["skel"], sd["skel"])
    v = wl.boundary_data()
    q = ctx.rhs(v)
    a = np.linspace(0, 2 * np.pi, 120, endpoint=False) + 0.1
    tg = 2.7 * np.stack([np.cos(a), np.sin(a)], axis=1)
    u = ctx.evaluate_field(tg, q)[:, 0]
    assert _rel(u, circle_scattered(kappa, 1.0, 0.0, tg)) < 1e-9
    # S itself: the outgoing field of S v_hat outside the proxy
    qs = info["S"] @ v[info["skel"], 0]
    us = orc.field(2, kappa, tg, wl.shapes[0].x[info["skel"]], qs)
    assert _rel(us, circle_scattered(kappa, 1.0, 0.0, tg)) < 1e-9


def test_gpu_built_pipeline_three_bodies(pkg):
    """Full GPU pipeline (S build, right-hand side, FP64 and mixed solves, field)
    against the oracle on three resolved bodies.  ||S|| reaches 1.2e5 (ID to
    1e-12 on 192 points), so an FP64 evaluation of the operator rounds to
    ~u ||S|| ~ 1.3e-11 relative: solved to 5e-11."""
    shapes = [mi.shape_2d("star3n", 192, 96, 193, 1.8, eps=1e-12),
              mi.shape_2d("ellipse", 192, 96, 193, 1.8, eps=1e-12)]
    centres = np.array([[0.0, 0.0, 0], [4.1, 0.6, 0], [1.2, 4.3, 0]])
    rots = np.stack([mi.rot2(0.3), mi.rot2(1.9), mi.rot2(-0.8)])
    dirs = np.array([[1.0, 0, 0], [math.cos(2.0), math.sin(2.0), 0]])
    wl = mi.Workload("three", 2, 5.0, shapes, np.array([0, 1, 0], np.int32), centres, rots, dirs)
    ref = orc.solve_workload(wl)
    tg = mi.far_targets(wl, 128, mode="ring")
    u_ref = orc.field(2, wl.kappa, tg, ref["layout"]["xhat"], ref["q"])
    for s in range(2):
        assert np.array_equal(ref["sdata"][s]["skel"], orc.cpqr_id(ref["sdata"][s]["B"], eps=1e-12)[0])
    for prec in (pkg.PREC_FP64, pkg.PREC_MIXED):
        ctx = pkg.Context(2, wl.kappa, precision=prec, tol=5e-11)
        ctx.build_scattering_matrices(wl)
        _check_build_matches_oracle(ctx, wl, ref)
        b = ctx.rhs(ref["v"])
        q, info = ctx.solve(b)
        assert info["converged"] == 1 and info["rel_residual"] <= 5e-11
        u = ctx.evaluate_field(tg, q)
        assert _rel(u, u_ref) < 1e-9, prec


def _near_targets(wl, per_body=48, seed=7):
    """Targets inside every proxy: on Gamma between collocation points (where
    u + u_inc = 0 must hold) and in the annulus between Gamma and the proxy."""
    from mbs_inputs.workloads import _BOUND, _curve
    rng = np.random.default_rng(seed)
    pts, on_gamma = [], []
    for t in range(wl.T):
        sh = wl.shapes[int(wl.body_shape[t])]
        th = 2 * np.pi * (np.arange(sh.m) + 0.5) / sh.m
        on = _curve(sh.name, th, sh.bound_radius / _BOUND[sh.name])[::max(1, sh.m // per_body)]
        ang = rng.uniform(0, 2 * np.pi, per_body)
        rad = rng.uniform(sh.bound_radius * 1.05, sh.proxy_radius * 0.98, per_body)
        ring = np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)
        for loc, flag in ((on, True), (ring, False)):
            pts.append(wl.centres[t, :2] + loc @ wl.rots[t, :2, :2].T)
            on_gamma.append(np.full(len(loc), flag))
    return np.concatenate(pts, axis=0), np.concatenate(on_gamma)


def test_near_field_reconstruction_matches_oracle(pkg):
    """Sec. 4.6 on the GPU: q_mfs = A^+ (v - U G_hat q_hat) from the GPU-built
    factors and the near field (MFS sources of the body whose proxy holds the
    target, skeleton sums of the others) against the oracle's, on Gamma and in
    the annuli between Gamma and the proxies; the GPU's own field also meets
    the sound-soft condition on Gamma.  Far targets give exactly what
    mbs_evaluate_field gives."""
    wl = mi.tiny_2d(seed=0, T=4, kappa=6.0, nrhs=2, ks=(0, 0, 0), eps=1e-12)
    for i, a in enumerate((1.0, 0.8, 0.9)):  # circles of three radii (resolved at m = 160)
        wl.shapes[i] = mi.shape_2d("circle", 160, 80, 161, 1.3, scale=a, k=0, eps=1e-12)
    ref = orc.solve_workload(wl)
    qm_ref = orc.reconstruct_mfs(wl, ref["sdata"], ref["layout"], ref["q"], ref["v"])
    tg, on_gamma = _near_targets(wl)
    assert np.all(orc.proxy_body(wl, tg) >= 0)
    u_ref = orc.field_near(wl, ref["sdata"], ref["layout"], ref["q"], qm_ref, tg)
    far = mi.far_targets(wl, 64, mode="ring")
    for prec in (pkg.PREC_FP64, pkg.PREC_MIXED):
        ctx = pkg.Context(2, wl.kappa, precision=prec, tol=1e-11)
        ctx.build_scattering_matrices(wl)
        _check_build_matches_oracle(ctx, wl, ref)
        q, info = ctx.solve(ctx.rhs(ref["v"]))
        assert info["rel_residual"] <= 1e-11, prec
        qm = ctx.reconstruct(ref["v"], q)
        assert qm.shape == (ctx.Nm, 2)
        u = ctx.evaluate_field_near(tg, q, qm)
        assert _rel(u, u_ref) < 1e-8, prec
        on = tg[on_gamma]
        u_on = u[on_gamma]
        assert np.max(np.abs(u_on + wl.incident(on))) < 1e-8, prec
        assert np.array_equal(ctx.evaluate_field_near(far, q, qm), ctx.evaluate_field(far, q))
        with pytest.raises(pkg.MbsError):
            ctx.evaluate_field(tg[:4], q)  # near targets need the reconstruction
        ctx.close()


def _oracle_rank_a(wl, s):
    """Singular values of the shape's MFS matrix A kept by the oracle's
    truncated SVD (relative 1e-14)."""
    sh = wl.shapes[s]
    sv = np.linalg.svd(orc.kernel_matrix(wl.dim, wl.kappa, sh.x, sh.y), compute_uv=False)
    return int(np.sum(sv > 1e-14 * sv[0]))


def _check_build_matches_oracle(ctx, wl, ref):
    """The GPU build picks the oracle's skeleton and keeps the same singular
    values of A (up to one at the cutoff)."""
    for s in range(len(wl.shapes)):
        if ref["sdata"][s] is None:  # shape used by no body: not built
            continue
        g = ctx.get_shape(s)
        assert np.array_equal(np.sort(g["skel"]), np.sort(ref["sdata"][s]["skel"])), s
        assert abs(ctx.get_shape_stats(s)["rank_a"] - _oracle_rank_a(wl, s)) <= 1, s


def test_near_field_reconstruction_3d(pkg):
    """The same in 3D: three spheres resolved to a boundary residual of ~1e-4
    (kappa = 1, 16 x 32 collocation grid, MFS surface at half the radius, proxy
    at 1.6 radii), targets between each surface and its proxy sphere, GPU-built
    S against the oracle.  Relative 1e-15 perturbations of the oracle's point
    sets move its own fields by up to 6.7e-10 (far) and 2.4e-10 (near): the
    bounds are 1e-9 far (measured 5.1e-10) and 2e-9 near (measured 2.3e-10),
    within 10x of that rounding sensitivity."""
    wl = geo.spheres()
    ref = orc.solve_workload(wl)
    qm_ref = orc.reconstruct_mfs(wl, ref["sdata"], ref["layout"], ref["q"], ref["v"])
    tg = geo.spheres_near_targets(wl)
    assert np.all(orc.proxy_body(wl, tg) >= 0)
    u_ref = orc.field_near(wl, ref["sdata"], ref["layout"], ref["q"], qm_ref, tg)
    far = mi.far_targets(wl, 96, mode="ring")
    u_far = orc.field(3, wl.kappa, far, ref["layout"]["xhat"], ref["q"])
    ctx = pkg.Context(3, wl.kappa, precision=pkg.PREC_FP64, tol=1e-11, max_iter=400)
    ctx.build_scattering_matrices(wl)
    _check_build_matches_oracle(ctx, wl, ref)
    q, info = ctx.solve(ctx.rhs(ref["v"]))
    assert info["rel_residual"] <= 1e-11
    assert _rel(ctx.evaluate_field(far, q), u_far) < 1e-9
    u = ctx.evaluate_field_near(tg, q, ctx.reconstruct(ref["v"], q))
    assert _rel(u, u_ref) < 2e-9
    ctx.close()


def test_gpu_built_ellipsoids_far_field_3d(pkg):
    """3D far-field parity of the GPU-built S on resolved ellipsoids: three
    shapes (semi-axes up to 0.9), four bodies, kappa = 2, 16 x 32 collocation
    grid, MFS surface at 0.7 scale, proxy at 1.5 times the largest semi-axis,
    ID to 1e-10 (k ~ 480 of m = 512).  FP64 and mixed-precision solves to a
    relative residual of 1e-11, scattered field at a far ring against the
    oracle at 1e-9 (measured 1.2e-10; the oracle's own field moves by ~6e-11
    under relative 1e-15 perturbations of its point sets)."""
    wl = geo.ellipsoids()
    ref = orc.solve_workload(wl)
    far = mi.far_targets(wl, 96, mode="ring")
    u_far = orc.field(3, wl.kappa, far, ref["layout"]["xhat"], ref["q"])
    for prec in (pkg.PREC_FP64, pkg.PREC_MIXED):
        ctx = pkg.Context(3, wl.kappa, precision=prec, tol=1e-11, max_iter=400)
        ctx.build_scattering_matrices(wl)
        _check_build_matches_oracle(ctx, wl, ref)
        q, info = ctx.solve(ctx.rhs(ref["v"]))
        assert info["rel_residual"] <= 1e-11, prec
        assert _rel(ctx.evaluate_field(far, q), u_far) < 1e-9, prec
        ctx.close()


def test_gpu_built_teardrops_with_corner_refinement(pkg):
    """Non-smooth bodies (Sec. 3.3): three teardrops on Gauss-Legendre panels
    with 12 dyadic refinements at the corner (m = 640, sources down to ~1e-5
    from the corner), S built on the GPU, FP64 and mixed solves, far field and
    near field against the oracle.

    The corner-refined MFS matrix A has condition ~1e17; S (norm ~1.5e7) then
    fixes the FP64 residual to ~u ||S|| (measured 1.4e-9 FP64, 1.7e-9 mixed),
    the floor of any FP64 evaluation of this operator.  Relative 1e-15
    perturbations of the oracle's point sets move its own far field by 5.3e-10
    and its field on Gamma next to the corner by 3.8e-8: the bounds are 1e-9
    far (measured 6.7e-10) and 1e-7 near (measured 1.8e-8)."""
    wl = geo.teardrops()
    ref = orc.solve_workload(wl)
    qm_ref = orc.reconstruct_mfs(wl, ref["sdata"], ref["layout"], ref["q"], ref["v"])
    far = mi.far_targets(wl, 96, mode="ring")
    near = geo.panel_near_targets(wl)
    u_far = orc.field(2, wl.kappa, far, ref["layout"]["xhat"], ref["q"])
    u_near = orc.field_near(wl, ref["sdata"], ref["layout"], ref["q"], qm_ref, near)
    for prec in (pkg.PREC_FP64, pkg.PREC_MIXED):
        ctx = pkg.Context(2, wl.kappa, precision=prec, tol=1e-12, max_iter=600)
        ctx.build_scattering_matrices(wl)
        _check_build_matches_oracle(ctx, wl, ref)
        q, info = ctx.solve(ctx.rhs(ref["v"]), raise_on_noconv=False)
        assert info["rel_residual"] < 3e-9, prec
        assert _rel(ctx.evaluate_field(far, q), u_far) < 1e-9, prec
        u = ctx.evaluate_field_near(near, q, ctx.reconstruct(ref["v"], q))
        assert _rel(u, u_near) < 1e-7, prec
        ctx.close()


def test_gpu_built_cshapes_and_rods(pkg):
    """The other non-smooth families of Sec. 5.1: two C-shapes (arcs joined by
    semicircular caps) and two rods (rectangles with semicircular caps) on
    Gauss-Legendre panels refined 4 times at every joint, S built on the GPU,
    FP64 and mixed solves, far field and near field on Gamma against the
    oracle.  ||S|| ~ 1.7e5 puts the FP64 residual floor near 1.5e-11.  The
    oracle's own fields move by 5.6e-11 (far) and 1.8e-9 (on Gamma next to the
    joints) under relative 1e-15 perturbations of its point sets: the bounds
    are 5e-10 far (measured 2.3e-10) and 1.5e-8 near (measured 7.9e-9)."""
    wl = geo.cshapes_rods()
    ref = orc.solve_workload(wl)
    qm_ref = orc.reconstruct_mfs(wl, ref["sdata"], ref["layout"], ref["q"], ref["v"])
    far = mi.far_targets(wl, 96, mode="ring")
    near = geo.panel_near_targets(wl)
    u_far = orc.field(2, wl.kappa, far, ref["layout"]["xhat"], ref["q"])
    u_near = orc.field_near(wl, ref["sdata"], ref["layout"], ref["q"], qm_ref, near)
    for prec in (pkg.PREC_FP64, pkg.PREC_MIXED):
        ctx = pkg.Context(2, wl.kappa, precision=prec, tol=1e-12, max_iter=600)
        ctx.build_scattering_matrices(wl)
        _check_build_matches_oracle(ctx, wl, ref)
        q, info = ctx.solve(ctx.rhs(ref["v"]), raise_on_noconv=False)
        assert info["rel_residual"] < 5e-11, (prec, info)
        assert _rel(ctx.evaluate_field(far, q), u_far) < 5e-10, prec
        u = ctx.evaluate_field_near(near, q, ctx.reconstruct(ref["v"], q))
        assert _rel(u, u_near) < 1.5e-8, prec
        ctx.close()


def test_reconstruction_refuses_injected_data(pkg):
    wl = mi.config0()
    ctx, sdata, lay = _ctx_with_oracle_S(pkg, wl)
    q = _rand((ctx.N, 1), 2)
    with pytest.raises(pkg.MbsError):
        ctx.reconstruct(wl.boundary_data(), q)
    ctx.close()


# --------------------------------------------------------------------------
# errors and degenerate cases
# --------------------------------------------------------------------------
def test_error_paths(pkg):
    wl = mi.config0()
    ctx = pkg.Context(2, wl.kappa)
    with pytest.raises(pkg.MbsError) as e:
        ctx.apply_operator(np.zeros((10, 1)))  # before build
    assert e.value.status == 8
    ctx.build_scattering_matrices(wl)
    with pytest.raises(pkg.MbsError) as e:
        ctx.evaluate_field(np.array([[0.1, 0.2]]), np.zeros((ctx.N, 1)))
    assert e.value.status == 7
    bad = mi.config0()
    bad.centres[1, :2] = bad.centres[0, :2] + 1.0  # body 1 inside body 0's proxy
    with pytest.raises(pkg.MbsError) as e:
        pkg.Context(2, wl.kappa).build_scattering_matrices(bad)
    assert e.value.status == 2


def test_single_body_has_no_coupling(pkg):
    wl = mi.circle_single(3.0, m=96, eps=1e-10, proxy_factor=2.0)
    ctx = pkg.Context(2, wl.kappa)
    ctx.build_scattering_matrices(wl)
    q = _rand((ctx.N, 2), 1)
    assert np.all(ctx.apply_G(q) == 0)
    b = ctx.rhs(wl.boundary_data())
    x, info = ctx.solve(b)
    assert _rel(x, b) < 1e-14


def test_bench_workload_solution_residual_against_oracle_rows(pkg):
    """The bench's headline solve (1000 bodies, N = 64,000, 8 plane waves, mixed
    precision to 1e-11, GPU-built S) checked independently of the GPU's own
    operator: for four sampled bodies, the oracle's G_hat rows applied to the
    GPU's q_hat, then each body's S (as built), give the residual
    b - (q + S G q) on those 256 rows.  Bound: 1e-9 relative to |b| on the
    sampled rows (the solve reached 6e-12 with the GPU operator; the oracle's
    FP64 rows differ from the GPU's double-float ones by ~1e-13 relative,
    times ||S|| ~ 25)."""
    wl = mi.config1()
    ctx = pkg.Context(2, wl.kappa, precision=pkg.PREC_MIXED, tol=1e-11, restart=200, inner_tol=1e-4,
                      max_iter=50000, max_sweeps=12)
    ctx.build_scattering_matrices(wl)
    b = ctx.rhs(wl.boundary_data())
    q, info = ctx.solve(b)
    assert info["rel_residual"] <= 1e-11
    N, off, xyz = ctx.get_layout()
    body = np.repeat(np.arange(wl.T), np.diff(off))
    rng = np.random.default_rng(7)
    for t in rng.choice(wl.T, 4, replace=False):
        rows = np.arange(off[t], off[t + 1])
        Gq = orc.G_rows(2, wl.kappa, xyz, body, q, rows)
        S = ctx.get_shape(int(wl.body_shape[t]))["S"]
        r = b[rows] - q[rows] - S @ Gq
        assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm(b[rows]), t
    ctx.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_gpu_randomized_id_matches_oracle_sketch(pkg, dim):
    """Randomized ID (id_sketch): the GPU generates the same Gaussian sketch as
    the oracle (Philox4x32-10 keyed by seed and shape, Box-Muller), takes the
    skeleton from the pivoted QR of Omega B, and builds S from it.  The
    skeleton equals the oracle's sketch skeleton (and differs from the
    deterministic one, so the option is in effect); FP64 and mixed solves
    match the oracle's sketched pipeline in the far field to 1e-9.  2D: the
    10-body workload (B 129 x 128, k = 64, 74-row sketch); 3D: five
    ellipsoids (B 141 x 140, k = 70, 80-row sketch)."""
    wl = mi.config0() if dim == 2 else mi.tiny_3d(seed=0, T=5, kappa=3.0, nth=10, nph=14, p=141, k=70)
    ref = orc.solve_workload(wl, sketch=(7, 10))
    det = orc.build_all(wl)
    tg = mi.far_targets(wl, 96, mode="ring")
    u_ref = orc.field(dim, wl.kappa, tg, ref["layout"]["xhat"], ref["q"])
    differs = False
    for prec in (pkg.PREC_FP64, pkg.PREC_MIXED):
        ctx = pkg.Context(dim, wl.kappa, precision=prec, tol=1e-12, id_sketch=10, id_seed=7)
        ctx.build_scattering_matrices(wl)
        for s, sd in enumerate(ref["sdata"]):
            if sd is None:
                continue
            g = np.sort(ctx.get_shape(s)["skel"])
            assert np.array_equal(g, np.sort(sd["skel"])), s
            differs = differs or not np.array_equal(g, np.sort(det[s]["skel"]))
        q, info = ctx.solve(ctx.rhs(ref["v"]))
        assert _rel(ctx.evaluate_field(tg, q), u_ref) < 1e-9, prec
        ctx.close()
    assert differs
