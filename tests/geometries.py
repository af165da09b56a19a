"""Small multibody geometries shared by the GPU parity tests and by
oracle_sensitivity.py (inputs only: no solver arithmetic)."""
import math

import numpy as np

import mbs_inputs as mi


def teardrops():
    """Three teardrops (Sec. 5.1 Ex. 3) on 16 Gauss-Legendre panels with 12
    dyadic refinements at the corner, kappa = 5, two plane waves."""
    sh = mi.shape_panels_2d("teardrop", 16, 12, 0.3, 1.6, eps=1e-12)
    centres = np.array([[0.0, 0.0, 0], [3.6, 0.5, 0], [0.9, 3.7, 0]])
    rots = np.stack([mi.rot2(0.3), mi.rot2(1.9), mi.rot2(-0.8)])
    return mi.Workload("teardrops", 2, 5.0, [sh], np.zeros(3, np.int32), centres, rots,
                       np.array([[1.0, 0, 0], [math.cos(2.0), math.sin(2.0), 0]]))


def cshapes_rods():
    """Two C-shapes and two rods (Sec. 5.1 Ex. 2/4), joints refined 4 times."""
    shc = mi.shape_panels_2d("cshape", 40, 4, 0.1, 1.6, eps=1e-12)
    shr = mi.shape_panels_2d("rod", 44, 4, 0.1, 1.6, eps=1e-12)
    centres = np.array([[0.0, 0.0, 0], [3.4, 0.3, 0], [0.2, 3.5, 0], [3.6, 3.6, 0]])
    rots = np.stack([mi.rot2(0.4), mi.rot2(2.1), mi.rot2(-1.0), mi.rot2(0.9)])
    return mi.Workload("cshapes+rods", 2, 5.0, [shc, shr], np.array([0, 1, 1, 0], np.int32), centres,
                       rots, np.array([[1.0, 0, 0], [math.cos(2.0), math.sin(2.0), 0]]))


def spheres():
    """Three spheres, kappa = 1, 16 x 32 collocation grid, MFS surface at half
    the radius, proxy at 1.6 radii."""
    rng = np.random.default_rng(2)
    radii = (0.8, 0.7, 0.75)
    shapes = [mi.shape_ellipsoid(a, a, a, nth=16, nph=32, p=601, proxy_radius=1.6 * a, eps=1e-10,
                                 mfs_scale=0.5) for a in radii]
    centres = np.array([[0, 0, 0], [3.6, 0.4, 0.2], [0.5, 3.5, -0.3]], float)
    rots = np.stack([mi.rot_quat(rng.normal(size=4)) for _ in radii])
    return mi.Workload("spheres", 3, 1.0, shapes, np.arange(3, dtype=np.int32), centres, rots,
                       np.array([[1.0, 0, 0], [0, 0.6, 0.8]]))


def spheres_near_targets(wl, seed=2):
    """40 targets per sphere between its surface and its proxy sphere."""
    rng = np.random.default_rng(seed)
    for _ in wl.body_shape:  # the rotations drew four normals each
        rng.normal(size=4)
    pts = []
    for t in range(wl.T):
        sh = wl.shapes[int(wl.body_shape[t])]
        a, rp = sh.bound_radius, sh.proxy_radius
        d = rng.normal(size=(40, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        pts.append(wl.centres[t] + d * rng.uniform(1.1 * a, 0.97 * rp, 40)[:, None])
    return np.concatenate(pts)


def ellipsoids():
    """Four resolved ellipsoids of three shapes (semi-axes up to 0.9), kappa =
    2, 16 x 32 collocation grid, MFS surface at 0.7 scale, proxy at 1.5 times
    the largest semi-axis."""
    rng = np.random.default_rng(5)
    axes = [(0.9, 0.7, 0.6), (0.8, 0.8, 0.6), (0.7, 0.6, 0.9)]
    shapes = [mi.shape_ellipsoid(a, b, c, nth=16, nph=32, p=601, proxy_radius=1.5 * max(a, b, c),
                                 eps=1e-10, mfs_scale=0.7) for a, b, c in axes]
    centres = np.array([[0, 0, 0], [3.4, 0.4, 0.2], [0.5, 3.5, -0.3], [3.6, 3.4, 0.4]], float)
    rots = np.stack([mi.rot_quat(rng.normal(size=4)) for _ in range(4)])
    return mi.Workload("ellipsoids", 3, 2.0, shapes, np.array([0, 1, 2, 0], np.int32), centres, rots,
                       np.array([[1.0, 0, 0], [0, 0.6, 0.8]]))


def panel_near_targets(wl):
    """Points on Gamma between collocation nodes (every fifth check point)."""
    return np.concatenate([wl.centres[t, :2] + mi.panel_check_points(wl.shapes[int(wl.body_shape[t])])[::5]
                           @ wl.rots[t, :2, :2].T for t in range(wl.T)])
