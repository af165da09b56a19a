"""The seeded synthetic workloads match their stated recipe: sizes, skeleton
counts, pairs per matvec, incident fields, determinism, and the geometric
guarantees the method needs (bounding circles/spheres apart by the stated gap,
no body reaching into another body's proxy surface; Sec. 4.1 requires the
sources of every other body to lie outside each proxy)."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import mbs_inputs as mi


def _min_pair_margin(wl, need):
    """min over body pairs of |c_t - c_s| - need(t, s), with need a function of
    the two bodies (checked on the 12 nearest neighbours of every body)."""
    d = wl.dim
    c = wl.centres[:, :d]
    dist, idx = cKDTree(c).query(c, k=min(13, wl.T))
    worst = np.inf
    for t in range(wl.T):
        for dd, s in zip(dist[t, 1:], idx[t, 1:]):
            worst = min(worst, dd - need(t, s))
    return worst


def _rotations_ok(wl):
    d = wl.dim
    R = wl.rots[:, :d, :d]
    eye = np.einsum("tij,tkj->tik", R, R)
    return np.allclose(eye, np.eye(d)[None], atol=1e-12) and np.allclose(np.linalg.det(R), 1.0)


def test_config0_recipe():
    wl = mi.config0()
    sh = wl.shapes[0]
    assert (wl.T, sh.m, sh.n, sh.p, sh.k, wl.kappa, wl.nrhs) == (10, 128, 64, 129, 64, 10.0, 1)
    assert sh.proxy_radius == 1.5 and sh.bound_radius == pytest.approx(1.2)
    assert np.allclose(wl.directions[0], [1.0, 0.0, 0.0])
    assert _min_pair_margin(wl, lambda t, s: 1.2 + 1.2 + 0.6) >= -1e-12  # gap 0.6


def test_config1_recipe():
    wl = mi.config1()
    ks = np.array([wl.shapes[s].k for s in wl.body_shape])
    N = int(ks.sum())
    assert (wl.T, N, wl.kappa, wl.nrhs, len(wl.shapes)) == (1000, 64000, 40.0, 8, 3)
    assert N * N - int(np.sum(ks ** 2)) == 4_091_904_000
    for sh in wl.shapes:
        assert (sh.m, sh.n, sh.p, sh.k, sh.proxy_radius) == (128, 64, 129, 64, 1.25)
        assert np.max(np.linalg.norm(sh.x, axis=1)) <= 1.0 + 1e-12
    ang = np.arctan2(wl.directions[:, 1], wl.directions[:, 0]) % (2 * np.pi)
    assert np.allclose(np.sort(ang), 2 * np.pi * np.arange(8) / 8)
    assert np.all(np.abs(wl.centres[:, :2] - 50.0) <= 50.0)
    assert _rotations_ok(wl)
    assert _min_pair_margin(wl, lambda t, s: 2.5) >= -1e-12          # bounding gap >= 0.5
    assert _min_pair_margin(wl, lambda t, s: 1.25 + 1.0) > 0          # outside every proxy
    assert np.array_equal(mi.config1().centres, wl.centres)           # seeded
    assert not np.array_equal(mi.config1(seed=1).centres, wl.centres)


def test_config2_recipe():
    wl = mi.config2()
    rho = np.array([sh.bound_radius for sh in wl.shapes])
    ks = np.array([sh.k for sh in wl.shapes])
    assert (wl.T, wl.kappa, wl.nrhs) == (10000, 20.0, 16)
    assert np.all((rho >= 0.5) & (rho <= 1.5))
    assert np.array_equal(ks, np.clip(np.round(3.5 * 20.0 * rho), 32, 128).astype(int))
    assert ks.min() >= 35 and ks.max() <= 105
    for sh, k, r in zip(wl.shapes[:200], ks[:200], rho[:200]):
        assert (sh.m, sh.n, sh.p) == (2 * k, k, 2 * k + 1) and sh.proxy_radius == pytest.approx(r + 0.25)
    assert _min_pair_margin(wl, lambda t, s: rho[t] + rho[s] + 0.5) >= -1e-9
    assert _min_pair_margin(wl, lambda t, s: rho[t] + 0.25 + rho[s]) > 0


def test_config3_recipe():
    wl = mi.config3()
    assert (wl.T, wl.dim, wl.kappa, wl.nrhs) == (2000, 3, 8.0, 4)
    sh0 = wl.shapes[0]
    assert (sh0.m, sh0.n, sh0.p, sh0.k) == (600, 150, 601, 300)
    N = sum(sh.k for sh in wl.shapes)
    assert N == 600_000 and N * N - 2000 * 300 ** 2 == 359_820_000_000
    amax = np.array([sh.bound_radius for sh in wl.shapes])
    assert np.all((amax >= 0.6) & (amax <= 1.0))
    assert np.allclose(np.linalg.norm(wl.directions, axis=1), 1.0)
    assert _rotations_ok(wl)
    assert _min_pair_margin(wl, lambda t, s: amax[t] + 0.25 + amax[s]) > 0


def test_serving_trace_recipe():
    tr = mi.serving_trace()
    assert len(tr) == 512
    arr = np.array([r.arrival for r in tr])
    assert np.all(np.diff(arr) > 0)
    assert abs(np.mean(np.diff(arr)) - 1 / 20) < 0.15 / 20
    T = np.array([r.T for r in tr])
    assert T.min() >= 20 and T.max() <= 3000
    frac2d = np.mean([r.dim == 2 for r in tr])
    assert abs(frac2d - 0.7) < 0.07
    assert all(5 <= r.kappa <= 50 and 1 <= r.nrhs <= 32 for r in tr)
    assert [(r.T, r.dim, r.nrhs) for r in mi.serving_trace()] == [(r.T, r.dim, r.nrhs) for r in tr]


def test_incident_field_and_boundary_data():
    wl = mi.config0()
    X = wl.collocation_world()
    assert X.shape == (1280, 2)
    v = wl.boundary_data()
    assert np.allclose(v[:, 0], -np.exp(1j * 10.0 * X[:, 0]))


@pytest.mark.parametrize("kind,m_base,nref", [("teardrop", 16, 12), ("cshape", 40, 4), ("rod", 44, 4)])
def test_panel_shapes_refine_at_corners_and_keep_sources_inside(kind, m_base, nref):
    """Sec. 3.3: the panels touching every corner (or curvature joint) are
    halved n_refine times towards it, so the smallest panels there have
    length h / 2^n_refine; every MFS source lies strictly inside the curve
    (winding number 1), as the method of fundamental solutions requires."""
    from mbs_inputs import workloads as w
    sh = mi.shape_panels_2d(kind, m_base, nref, 0.3 if kind == "teardrop" else 0.1, 1.6)
    h = 2 * np.pi / m_base
    br = sh.panels
    lengths = np.diff(br)
    for c in w._CORNERS[kind]:
        for side in (+1, -1):
            # the panel that ends (side -1) or starts (side +1) at the corner
            t = c % (2 * np.pi)
            if side > 0:
                i = int(np.argmin(np.abs(br[:-1] - t)))
                if t == 0.0:
                    i = 0
            else:
                i = int(np.argmin(np.abs(br[1:] - (t if t > 0 else 2 * np.pi))))
            assert lengths[i] == pytest.approx(h / 2 ** nref, rel=1e-9), (kind, c, side)
    poly = w._curve(kind, np.linspace(0, 2 * np.pi, 20001)[:-1], 1.0)
    assert np.all(_winding_number(poly, sh.y) == 1)
    assert np.all(_winding_number(poly, 1.7 * sh.z / np.linalg.norm(sh.z, axis=1, keepdims=True)) == 0)


def _winding_number(poly, pts):
    """Winding number of a closed polygon (M, 2) around each point (K, 2)."""
    a = poly[None, :, :] - pts[:, None, :]
    b = np.roll(poly, -1, axis=0)[None, :, :] - pts[:, None, :]
    ang = np.arctan2(a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0], np.sum(a * b, axis=-1))
    return np.rint(ang.sum(axis=1) / (2 * np.pi)).astype(int)


def test_serving_requests_materialise_as_stated():
    """A 2D request is the config1 construction at its own T, kappa and nrhs
    (box side scaled with sqrt(T / 1000)); a 3D request is the config3
    construction with nrhs unit directions."""
    tr = mi.serving_trace()
    r2 = next(r for r in tr if r.dim == 2 and r.T < 400)
    r3 = next(r for r in tr if r.dim == 3 and r.T < 400)
    w2, w3 = mi.request_workload(r2), mi.request_workload(r3)
    assert (w2.dim, w2.T, w2.kappa, w2.nrhs) == (2, r2.T, r2.kappa, r2.nrhs)
    assert all(sh.k == 64 and sh.m == 128 for sh in w2.shapes)
    side = np.ptp(w2.centres[:, :2], axis=0).max()
    assert side <= 100 * math.sqrt(r2.T / 1000) * 1.1 + 3.2
    assert (w3.dim, w3.T, w3.kappa, w3.nrhs) == (3, r3.T, r3.kappa, r3.nrhs)
    assert all(sh.k == 300 and sh.m == 600 for sh in w3.shapes)
    assert np.allclose(np.linalg.norm(w3.directions, axis=1), 1.0)
