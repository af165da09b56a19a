"""Seeded synthetic workloads for the multibody scattering solve.

This module produces *inputs only*: point sets on each body's boundary
(collocation points x), inside it (MFS sources y) and on its proxy surface
(proxy points z), body placements (centre + rotation), incident plane waves
sampled at the collocation points, and evaluation targets.  It holds none of
the solver's arithmetic (no kernel, no factorisation, no solve), so the CPU
oracle and the CUDA path can both draw from it without sharing method code.

Geometry readings (the paper leaves them open; see DESIGN notes):
  * smooth 2D bodies: points equispaced in the curve parameter (Sec. 3.2),
    MFS sources on the body scaled by 0.7 about its centre,
  * proxy surface: a circle (2D) or sphere (3D) about the body centre,
    p points equispaced (2D) or on a spherical Fibonacci lattice (3D),
  * 3D ellipsoids: tensor grid in (theta, phi) with the 2:1 ratio per
    parameter between collocation and MFS grids (Sec. 3.4),
  * non-smooth 2D bodies: Gauss-Legendre panels with dyadic refinement
    towards corners, MFS distance scaled with the local panel size (Sec. 3.3),
  * incident field u_inc = exp(i kappa d.x); the boundary data is
    v = -u_inc (sound-soft, Sec. 2.1 footnote).
"""
from .workloads import (  # noqa: F401
    Shape,
    Workload,
    shape_2d,
    shape_panels_2d,
    panel_breaks,
    panel_check_points,
    shape_ellipsoid,
    config0,
    config1,
    config2,
    config3,
    tiny_2d,
    tiny_3d,
    circle_single,
    sphere_single,
    serving_trace,
    request_workload,
    Request,
    fibonacci_sphere,
    far_targets,
    rot2,
    rot_quat,
)
