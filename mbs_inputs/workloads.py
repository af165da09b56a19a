"""Seeded synthetic geometries and incident fields (inputs only, no solver math).

Every generator draws from ``numpy.random.default_rng(seed)`` (PCG64) in a
fixed call order, so a (generator, seed) pair always yields the same bytes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * math.pi


# ----------------------------------------------------------------------------
# data containers
# ----------------------------------------------------------------------------
@dataclass
class Shape:
    """Point sets of one body shape in its local frame (centre at origin).

    x: (m, d) collocation points on the boundary Gamma (Sec. 3.1),
    y: (n, d) MFS sources on the interior curve/surface (Sec. 3.1),
    z: (p, d) proxy points on the proxy surface Psi (Sec. 4.2),
    k: fixed skeleton count (0 means: stop the pivoted QR at eps),
    eps: relative stopping tolerance of the pivoted QR when k == 0.
    """

    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    k: int = 0
    eps: float = 0.0
    proxy_radius: float = 0.0
    bound_radius: float = 0.0
    name: str = ""
    panels: np.ndarray | None = None  # panel end points in the curve parameter (panel shapes)

    @property
    def dim(self) -> int:
        return self.x.shape[1]

    @property
    def m(self) -> int:
        return self.x.shape[0]

    @property
    def n(self) -> int:
        return self.y.shape[0]

    @property
    def p(self) -> int:
        return self.z.shape[0]


@dataclass
class Workload:
    """T bodies, each a rigid placement x_world = c + R x_local of a shape."""

    name: str
    dim: int
    kappa: float
    shapes: list
    body_shape: np.ndarray  # (T,) int32
    centres: np.ndarray  # (T, 3) float64 (z = 0 in 2D)
    rots: np.ndarray  # (T, 3, 3) float64 (2D: upper-left 2x2 block used)
    directions: np.ndarray  # (nrhs, 3) unit propagation directions
    meta: dict = field(default_factory=dict)

    @property
    def T(self) -> int:
        return int(self.body_shape.shape[0])

    @property
    def nrhs(self) -> int:
        return int(self.directions.shape[0])

    def m_of_body(self) -> np.ndarray:
        return np.array([self.shapes[s].m for s in self.body_shape], dtype=np.int64)

    def body_points(self, tau: int, which: str = "x") -> np.ndarray:
        """World coordinates of one body's point set ('x', 'y' or 'z')."""
        sh = self.shapes[int(self.body_shape[tau])]
        loc = getattr(sh, which)
        d = self.dim
        return self.centres[tau, :d] + loc @ self.rots[tau, :d, :d].T

    def collocation_world(self) -> np.ndarray:
        """All collocation points, body after body: (sum m_tau, d)."""
        return np.concatenate([self.body_points(t, "x") for t in range(self.T)], axis=0)

    def incident(self, pts: np.ndarray) -> np.ndarray:
        """u_inc(x) = exp(i kappa d.x) for every direction: (M, nrhs) complex128."""
        d = self.dim
        phase = pts @ self.directions[:, :d].T
        return np.exp(1j * self.kappa * phase)

    def boundary_data(self) -> np.ndarray:
        """v = -u_inc at every collocation point (sound-soft data): (sum m, nrhs)."""
        return -self.incident(self.collocation_world())

    def proxy_radius_of_body(self) -> np.ndarray:
        return np.array([self.shapes[s].proxy_radius for s in self.body_shape])

    def bound_radius_of_body(self) -> np.ndarray:
        return np.array([self.shapes[s].bound_radius for s in self.body_shape])

    def subset(self, bodies) -> "Workload":
        """Workload restricted to the listed bodies (shapes kept as they are)."""
        bodies = np.asarray(bodies, dtype=np.int64)
        return Workload(
            name=self.name + f"[{len(bodies)} bodies]",
            dim=self.dim,
            kappa=self.kappa,
            shapes=self.shapes,
            body_shape=self.body_shape[bodies].copy(),
            centres=self.centres[bodies].copy(),
            rots=self.rots[bodies].copy(),
            directions=self.directions.copy(),
            meta=dict(self.meta),
        )


# ----------------------------------------------------------------------------
# rotations
# ----------------------------------------------------------------------------
def rot2(angle: float) -> np.ndarray:
    c, s = math.cos(angle), math.sin(angle)
    R = np.eye(3)
    R[0, 0], R[0, 1], R[1, 0], R[1, 1] = c, -s, s, c
    return R


def rot_quat(q: np.ndarray) -> np.ndarray:
    """Rotation matrix of a (not necessarily unit) quaternion (w, x, y, z)."""
    w, x, y, z = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    return np.array(
        [
            [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
            [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
            [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
        ]
    )


# ----------------------------------------------------------------------------
# shapes
# ----------------------------------------------------------------------------
# Piecewise curves of Sec. 5.1 (C-shapes and rods): segments of circular arcs
# and straight lines, each a fixed fraction of the parameter range [0, 2 pi)
# (the footnoted panel fractions, so that equal panels in t put those shares
# of the base panels on each segment); the joints are refined like corners.
_C_ALPHA = math.pi / 4  # half opening angle of the C-shape's cavity
_ROD_A, _ROD_B = 0.8, 0.2  # rod: straight half length, cap radius (width 0.4)


def _arc(cx, cy, r, a0, a1):
    return ("arc", cx, cy, r, a0, a1)


def _line(x0, y0, x1, y1):
    return ("line", x0, y0, x1, y1)


_PIECES = {
    # outer arc (2/5), cap at -alpha (3/20), inner arc backwards (3/10), cap at +alpha (3/20)
    "cshape": [(0.4, _arc(0.0, 0.0, 1.0, _C_ALPHA, TWO_PI - _C_ALPHA)),
               (0.15, _arc(0.8 * math.cos(_C_ALPHA), -0.8 * math.sin(_C_ALPHA), 0.2,
                           -_C_ALPHA, math.pi - _C_ALPHA)),
               (0.3, _arc(0.0, 0.0, 0.6, TWO_PI - _C_ALPHA, _C_ALPHA)),
               (0.15, _arc(0.8 * math.cos(_C_ALPHA), 0.8 * math.sin(_C_ALPHA), 0.2,
                           math.pi + _C_ALPHA, TWO_PI + _C_ALPHA))],
    # bottom side (4/11), right cap (3/22), top side (4/11), left cap (3/22)
    "rod": [(4 / 11, _line(-_ROD_A, -_ROD_B, _ROD_A, -_ROD_B)),
            (3 / 22, _arc(_ROD_A, 0.0, _ROD_B, -math.pi / 2, math.pi / 2)),
            (4 / 11, _line(_ROD_A, _ROD_B, -_ROD_A, _ROD_B)),
            (3 / 22, _arc(-_ROD_A, 0.0, _ROD_B, math.pi / 2, 1.5 * math.pi))],
}


def _piece_starts(kind: str) -> np.ndarray:
    return TWO_PI * np.concatenate([[0.0], np.cumsum([f for f, _ in _PIECES[kind]])])


def _piecewise(kind: str, t: np.ndarray, deriv: bool) -> np.ndarray:
    """Point (or d/dt) of a piecewise curve at parameters t in [0, 2 pi)."""
    t = np.mod(np.asarray(t, dtype=np.float64), TWO_PI)
    st = _piece_starts(kind)
    idx = np.clip(np.searchsorted(st, t, side="right") - 1, 0, len(_PIECES[kind]) - 1)
    out = np.empty((t.size, 2))
    for i, (frac, seg) in enumerate(_PIECES[kind]):
        sel = idx == i
        u = (t[sel] - st[i]) / (TWO_PI * frac)
        du = 1.0 / (TWO_PI * frac)
        if seg[0] == "arc":
            _, cx, cy, r, a0, a1 = seg
            a = a0 + (a1 - a0) * u
            if deriv:
                out[sel] = (r * (a1 - a0) * du) * np.stack([-np.sin(a), np.cos(a)], axis=1)
            else:
                out[sel] = np.stack([cx + r * np.cos(a), cy + r * np.sin(a)], axis=1)
        else:
            _, x0, y0, x1, y1 = seg
            if deriv:
                out[sel] = np.array([(x1 - x0) * du, (y1 - y0) * du])
            else:
                out[sel] = np.stack([x0 + (x1 - x0) * u, y0 + (y1 - y0) * u], axis=1)
    return out


def _curve(kind: str, t: np.ndarray, scale: float) -> np.ndarray:
    if kind in _PIECES:
        return scale * _piecewise(kind, t, False)
    if kind == "circle":
        r = np.ones_like(t)
        return scale * np.stack([r * np.cos(t), r * np.sin(t)], axis=1)
    if kind == "star3":  # r(t) = 1 + 0.2 cos 3t   (rho = 1.2)
        r = 1.0 + 0.2 * np.cos(3 * t)
        return scale * np.stack([r * np.cos(t), r * np.sin(t)], axis=1)
    if kind == "star3n":  # the same curve normalised to unit bounding radius
        r = (1.0 + 0.2 * np.cos(3 * t)) / 1.2
        return scale * np.stack([r * np.cos(t), r * np.sin(t)], axis=1)
    if kind == "ellipse":  # semi-axes 1 and 0.6
        return scale * np.stack([np.cos(t), 0.6 * np.sin(t)], axis=1)
    if kind == "teardrop":  # one corner at t = 0 (Sec. 5.1, Example 3)
        x1 = 2.0 / np.pi ** 2 * t ** 2 - 4.0 / np.pi * t + 1.0
        x2 = 2.0 / np.pi ** 3 * t ** 3 - 6.0 / np.pi ** 2 * t ** 2 + 4.0 / np.pi * t
        return scale * np.stack([x1, x2], axis=1)
    if kind == "starfish5":  # f(t) = 81/101 - 20/101 cos 5t  (Sec. 5.1, Example 1)
        r = 81.0 / 101.0 - 20.0 / 101.0 * np.cos(5 * t)
        return scale * np.stack([r * np.cos(t), r * np.sin(t)], axis=1)
    raise ValueError(kind)


_BOUND = {"circle": 1.0, "star3": 1.2, "star3n": 1.0, "ellipse": 1.0, "starfish5": 1.0,
          "teardrop": 1.0, "cshape": 1.0, "rod": _ROD_A + _ROD_B}
# curve parameters of corners and of joints where the curvature jumps (all
# curves run over [0, 2 pi))
_CORNERS = {"teardrop": (0.0,),
            "cshape": tuple(_piece_starts("cshape")[:-1]),
            "rod": tuple(_piece_starts("rod")[:-1])}


def _tangent(kind: str, t: np.ndarray, scale: float, h: float = 1e-6) -> np.ndarray:
    """d x / d t: exact on piecewise curves (a difference would straddle a
    joint next to a deeply refined one), else a central difference of the
    parametrisation (inputs only)."""
    if kind in _PIECES:
        return scale * _piecewise(kind, t, True)
    return (_curve(kind, t + h, scale) - _curve(kind, t - h, scale)) / (2.0 * h)


def panel_breaks(kind: str, m_base: int, n_refine: int) -> np.ndarray:
    """Panel end points in [0, 2 pi]: m_base equal panels, the two panels
    touching each corner halved n_refine times towards it (dyadic refinement,
    Sec. 3.3)."""
    h = TWO_PI / m_base
    br = set(np.round(np.arange(m_base + 1) * h, 15))
    for c in _CORNERS.get(kind, ()):
        for j in range(1, n_refine + 1):
            br.add(round((c + h / 2 ** j) % TWO_PI, 15))
            br.add(round((c - h / 2 ** j) % TWO_PI, 15))
    return np.array(sorted(br))


def shape_panels_2d(kind: str, m_base: int, n_refine: int, d: float, proxy_radius: float,
                    q: int = 16, scale: float = 1.0, k: int = 0, eps: float = 0.0) -> Shape:
    """Non-smooth 2D body on Gauss-Legendre panels (Sec. 3.3): q nodes per
    panel for the collocation points, q / 2 per panel for the MFS sources
    (n = m / 2), each source moved into the body along the normal by d times
    the panel's length relative to a base panel, so the distance shrinks with
    the dyadic refinement at corners; p = m + 1 proxy points on a circle."""
    if kind in _PIECES:
        for f, _ in _PIECES[kind]:
            if abs(f * m_base - round(f * m_base)) > 1e-9:
                raise ValueError(f"{kind}: m_base = {m_base} does not put whole panels on every segment")
    br = panel_breaks(kind, m_base, n_refine)
    h = TWO_PI / m_base
    gx, _ = np.polynomial.legendre.leggauss(q)
    gy, _ = np.polynomial.legendre.leggauss(q // 2)
    tx, ty, dy = [], [], []
    for a, b in zip(br[:-1], br[1:]):
        tx.append(a + (b - a) * (gx + 1.0) / 2.0)
        ty.append(a + (b - a) * (gy + 1.0) / 2.0)
        dy.append(np.full(q // 2, d * (b - a) / h))
    tx, ty, dy = np.concatenate(tx), np.concatenate(ty), np.concatenate(dy)
    x = _curve(kind, tx, scale)
    tan = _tangent(kind, ty, scale)
    inward = np.stack([-tan[:, 1], tan[:, 0]], axis=1) / np.linalg.norm(tan, axis=1)[:, None]
    y = _curve(kind, ty, scale) + scale * dy[:, None] * inward  # counter-clockwise curves: left = inside
    m = x.shape[0]
    tz = TWO_PI * np.arange(m + 1) / (m + 1)
    z = proxy_radius * np.stack([np.cos(tz), np.sin(tz)], axis=1)
    return Shape(x=x, y=y, z=z, k=k, eps=eps, proxy_radius=proxy_radius,
                 bound_radius=_BOUND[kind] * scale, name=kind, panels=br)


def panel_check_points(sh: Shape, q: int = 7, scale: float = 1.0) -> np.ndarray:
    """Points of a panel shape's boundary between its collocation points
    (q-point Gauss-Legendre nodes on every panel)."""
    g, _ = np.polynomial.legendre.leggauss(q)
    br = sh.panels
    t = np.concatenate([a + (b - a) * (g + 1.0) / 2.0 for a, b in zip(br[:-1], br[1:])])
    return _curve(sh.name, t, scale)


def shape_2d(kind: str, m: int, n: int, p: int, proxy_radius: float, scale: float = 1.0,
             k: int = 0, eps: float = 0.0, mfs_scale: float = 0.7) -> Shape:
    """Smooth 2D body: m collocation and n MFS points equispaced in the curve
    parameter, MFS curve = body curve scaled by ``mfs_scale``, p proxy points
    equispaced on a circle of radius ``proxy_radius``."""
    tx = TWO_PI * np.arange(m) / m
    ty = TWO_PI * np.arange(n) / n
    tz = TWO_PI * np.arange(p) / p
    x = _curve(kind, tx, scale)
    y = _curve(kind, ty, scale * mfs_scale)
    z = proxy_radius * np.stack([np.cos(tz), np.sin(tz)], axis=1)
    return Shape(x=x, y=y, z=z, k=k, eps=eps, proxy_radius=proxy_radius,
                 bound_radius=_BOUND[kind] * scale, name=kind)


def fibonacci_sphere(p: int, radius: float) -> np.ndarray:
    """p points of the spherical Fibonacci lattice (Gonzalez 2010) on a sphere."""
    i = np.arange(p) + 0.5
    zc = 1.0 - 2.0 * i / p
    rr = np.sqrt(np.maximum(0.0, 1.0 - zc * zc))
    ga = math.pi * (3.0 - math.sqrt(5.0))
    ph = ga * np.arange(p)
    return radius * np.stack([rr * np.cos(ph), rr * np.sin(ph), zc], axis=1)


def _ellipsoid_grid(a, b, c, nth, nph, scale=1.0):
    th = math.pi * (np.arange(nth) + 0.5) / nth
    ph = TWO_PI * np.arange(nph) / nph
    T, P = np.meshgrid(th, ph, indexing="ij")
    pts = np.stack([a * np.sin(T) * np.cos(P), b * np.sin(T) * np.sin(P), c * np.cos(T)], axis=-1)
    return scale * pts.reshape(-1, 3)


def shape_ellipsoid(a: float, b: float, c: float, nth: int = 20, nph: int = 30, p: int = 601,
                    proxy_radius: float | None = None, k: int = 0, eps: float = 0.0,
                    mfs_scale: float = 0.7) -> Shape:
    """Ellipsoid with semi-axes (a, b, c): collocation on an nth x nph grid in
    (theta, phi), MFS sources on an (nth/2) x (nph/2) grid of the ellipsoid
    scaled by ``mfs_scale`` (ratio 2 per parameter, Sec. 3.4), proxy points on a
    Fibonacci sphere."""
    amax = max(a, b, c)
    if proxy_radius is None:
        proxy_radius = amax + 0.25
    x = _ellipsoid_grid(a, b, c, nth, nph)
    y = _ellipsoid_grid(a, b, c, nth // 2, nph // 2, mfs_scale)
    z = fibonacci_sphere(p, proxy_radius)
    return Shape(x=x, y=y, z=z, k=k, eps=eps, proxy_radius=proxy_radius, bound_radius=amax,
                 name=f"ellipsoid({a:.3f},{b:.3f},{c:.3f})")


def _dirs_2d(nrhs: int) -> np.ndarray:
    ang = TWO_PI * np.arange(nrhs) / nrhs
    return np.stack([np.cos(ang), np.sin(ang), np.zeros(nrhs)], axis=1)


# ----------------------------------------------------------------------------
# the five workload families
# ----------------------------------------------------------------------------
def config0() -> Workload:
    """10 copies of r = 1 + 0.2 cos 3t on a 5 x 2 grid of spacing 3, kappa = 10,
    m = 128, n = 64 (at 0.7 r), k = 64, p = 129, proxy radius 1.5, one plane
    wave along +x1."""
    sh = shape_2d("star3", 128, 64, 129, 1.5, k=64)
    T = 10
    centres = np.zeros((T, 3))
    for t in range(T):
        i, j = t // 2, t % 2
        centres[t, 0], centres[t, 1] = 3.0 * i, 3.0 * j
    rots = np.repeat(np.eye(3)[None], T, axis=0)
    return Workload("config0", 2, 10.0, [sh], np.zeros(T, np.int32), centres, rots,
                    _dirs_2d(1), meta={"seed": None})


def _lattice_2d(rng, T, nside, spacing, jitter):
    sites = rng.permutation(nside * nside)[:T]
    ix, iy = sites % nside, sites // nside
    jit = rng.uniform(-jitter, jitter, size=(T, 2))
    c = np.zeros((T, 3))
    c[:, 0] = (ix + 0.5) * spacing + jit[:, 0]
    c[:, 1] = (iy + 0.5) * spacing + jit[:, 1]
    return c


def config1(seed: int = 0, T: int = 1000, kappa: float = 40.0, nrhs: int = 8,
            k: int = 64) -> Workload:
    """1000 bodies (circle, 3-star, ellipse 1:0.6, unit bounding radius) on a
    jittered 32 x 32 lattice of spacing 3.125 in a 100 x 100 box (gap >= 0.5),
    random rotations, kappa = 40, m = 128, n = 64, k = 64, p = 129, proxy 1.25,
    8 plane waves at angles 2 pi j / 8.  Smaller T keeps the same density."""
    rng = np.random.default_rng(seed)
    nside = 32 if T == 1000 else max(1, math.ceil(math.sqrt(T * 1024 / 1000)))
    centres = _lattice_2d(rng, T, nside, 3.125, 0.3125)
    sid = rng.integers(3, size=T).astype(np.int32)
    ang = rng.uniform(0.0, TWO_PI, size=T)
    shapes = [shape_2d(kind, 128, 64, 129, 1.25, k=k) for kind in ("circle", "star3n", "ellipse")]
    rots = np.stack([rot2(a) for a in ang])
    return Workload(f"config1(T={T})", 2, kappa, shapes, sid, centres, rots, _dirs_2d(nrhs),
                    meta={"seed": seed})


def config2(seed: int = 0, T: int = 10000, kappa: float = 20.0, nrhs: int = 16) -> Workload:
    """10,000 bodies of radius rho ~ U(0.5, 1.5) on a jittered 100 x 100 lattice
    of spacing 4 (jitter 0.25), shapes as config1 scaled by rho, random
    rotation, k = clamp(round(3.5 kappa rho), 32, 128), m = 2k, n = k,
    p = 2k + 1, proxy rho + 0.25, kappa = 20, 16 plane waves; every body is its
    own shape."""
    rng = np.random.default_rng(seed)
    nside = 100 if T == 10000 else max(1, math.ceil(math.sqrt(T)))
    centres = _lattice_2d(rng, T, nside, 4.0, 0.25)
    rho = rng.uniform(0.5, 1.5, size=T)
    kind_id = rng.integers(3, size=T)
    ang = rng.uniform(0.0, TWO_PI, size=T)
    kinds = ("circle", "star3n", "ellipse")
    shapes = []
    for t in range(T):
        k = int(min(128, max(32, round(3.5 * kappa * rho[t]))))
        shapes.append(shape_2d(kinds[kind_id[t]], 2 * k, k, 2 * k + 1, rho[t] + 0.25,
                               scale=rho[t], k=k))
    rots = np.stack([rot2(a) for a in ang])
    return Workload(f"config2(T={T})", 2, kappa, shapes, np.arange(T, dtype=np.int32), centres,
                    rots, _dirs_2d(nrhs), meta={"seed": seed})


def config3(seed: int = 0, T: int = 2000, kappa: float = 8.0, nth: int = 20, nph: int = 30,
            p: int = 601, k: int = 300) -> Workload:
    """2000 ellipsoids (semi-axes ~ U(0.6, 1.0)) on a jittered 13^3 lattice of
    spacing 40/13 (jitter 0.288), uniform random rotations, kappa = 8,
    m = 600 (20 x 30), n = 150 (10 x 15, scale 0.7), k = 300, p = 601,
    proxy a_max + 0.25, plane waves along x, y, z and (1,1,1)/sqrt(3)."""
    rng = np.random.default_rng(seed)
    nside = 13 if T == 2000 else max(1, math.ceil(T ** (1.0 / 3.0) * (2197 / 2000) ** (1 / 3)))
    sp = 40.0 / 13.0
    sites = rng.permutation(nside ** 3)[:T]
    ix, iy, iz = sites % nside, (sites // nside) % nside, sites // (nside * nside)
    jit = rng.uniform(-0.288, 0.288, size=(T, 3))
    centres = np.stack([(ix + 0.5) * sp, (iy + 0.5) * sp, (iz + 0.5) * sp], axis=1) + jit
    axes = rng.uniform(0.6, 1.0, size=(T, 3))
    quats = rng.normal(size=(T, 4))
    shapes = [shape_ellipsoid(*axes[t], nth=nth, nph=nph, p=p, k=k) for t in range(T)]
    rots = np.stack([rot_quat(q) for q in quats])
    s3 = 1.0 / math.sqrt(3.0)
    dirs = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0], [s3, s3, s3]])
    return Workload(f"config3(T={T})", 3, kappa, shapes, np.arange(T, dtype=np.int32), centres,
                    rots, dirs, meta={"seed": seed})


# ----------------------------------------------------------------------------
# small cases for tests
# ----------------------------------------------------------------------------
def tiny_2d(seed: int = 0, T: int = 5, kappa: float = 6.0, nrhs: int = 3,
            ks=(24, 37, 50), m_per_k: int = 2, spacing: float = 3.2, eps: float = 0.0) -> Workload:
    """A few 2D bodies with uneven skeleton counts (one shape per k value)."""
    rng = np.random.default_rng(seed)
    kinds = ("star3n", "ellipse", "circle")
    shapes = []
    for i, k in enumerate(ks):
        m = m_per_k * k if k else 96
        shapes.append(shape_2d(kinds[i % 3], m, m // 2, m + 1, 1.3, k=k, eps=eps))
    nside = max(2, math.ceil(math.sqrt(T)))
    centres = _lattice_2d(rng, T, nside, spacing, 0.2)
    sid = rng.integers(len(shapes), size=T).astype(np.int32)
    ang = rng.uniform(0.0, TWO_PI, size=T)
    rots = np.stack([rot2(a) for a in ang])
    return Workload(f"tiny_2d(T={T})", 2, kappa, shapes, sid, centres, rots, _dirs_2d(nrhs),
                    meta={"seed": seed})


def tiny_3d(seed: int = 0, T: int = 4, kappa: float = 3.0, nrhs: int = 2, nth: int = 12,
            nph: int = 16, p: int = 193, k: int = 90, eps: float = 0.0) -> Workload:
    """A few small ellipsoids (coarse grids) for 3D tests."""
    rng = np.random.default_rng(seed)
    nside = max(2, math.ceil(T ** (1 / 3)))
    sp = 3.0
    sites = rng.permutation(nside ** 3)[:T]
    ix, iy, iz = sites % nside, (sites // nside) % nside, sites // (nside * nside)
    centres = np.stack([(ix + 0.5) * sp, (iy + 0.5) * sp, (iz + 0.5) * sp], axis=1)
    centres += rng.uniform(-0.2, 0.2, size=(T, 3))
    axes = rng.uniform(0.6, 1.0, size=(T, 3))
    quats = rng.normal(size=(T, 4))
    shapes = [shape_ellipsoid(*axes[t], nth=nth, nph=nph, p=p, k=k, eps=eps) for t in range(T)]
    rots = np.stack([rot_quat(q) for q in quats])
    dirs = np.array([[1.0, 0, 0], [0, 0.6, 0.8]])[:nrhs]
    return Workload(f"tiny_3d(T={T})", 3, kappa, shapes, np.arange(T, dtype=np.int32), centres,
                    rots, dirs, meta={"seed": seed})


def circle_single(kappa: float, m: int = 256, radius: float = 1.0, proxy_factor: float = 1.5,
                  eps: float = 1e-12, k: int = 0, nrhs_angles=(0.0,)) -> Workload:
    """One sound-soft circle of the given radius at the origin."""
    sh = shape_2d("circle", m, m // 2, m + 1, proxy_factor * radius, scale=radius, k=k, eps=eps)
    ang = np.asarray(nrhs_angles, dtype=np.float64)
    dirs = np.stack([np.cos(ang), np.sin(ang), np.zeros_like(ang)], axis=1)
    return Workload("circle", 2, kappa, [sh], np.zeros(1, np.int32), np.zeros((1, 3)),
                    np.eye(3)[None].copy(), dirs)


def sphere_single(kappa: float, nth: int = 30, nph: int = 60, radius: float = 1.0,
                  proxy_factor: float = 1.5, p: int | None = None, eps: float = 1e-10,
                  k: int = 0) -> Workload:
    """One sound-soft sphere at the origin, plane wave along +x3."""
    p = p if p is not None else nth * nph + 1
    sh = shape_ellipsoid(radius, radius, radius, nth=nth, nph=nph, p=p,
                         proxy_radius=proxy_factor * radius, k=k, eps=eps)
    return Workload("sphere", 3, kappa, [sh], np.zeros(1, np.int32), np.zeros((1, 3)),
                    np.eye(3)[None].copy(), np.array([[0.0, 0.0, 1.0]]))


# ----------------------------------------------------------------------------
# evaluation targets and the serving trace
# ----------------------------------------------------------------------------
def far_targets(wl: Workload, M: int, seed: int = 1, mode: str = "ring") -> np.ndarray:
    """Targets outside every proxy surface.

    mode 'ring': M points on a circle/sphere enclosing every proxy with margin 1;
    mode 'gaps': M points drawn uniformly in the bounding box and kept only if
    they lie outside every proxy (rejection sampling)."""
    rng = np.random.default_rng(seed)
    d = wl.dim
    c = wl.centres[:, :d]
    pr = wl.proxy_radius_of_body()
    if mode == "ring":
        mid = 0.5 * (c.min(axis=0) + c.max(axis=0))
        R = float(np.max(np.linalg.norm(c - mid, axis=1) + pr)) + 1.0
        if d == 2:
            a = TWO_PI * (np.arange(M) + rng.uniform()) / M
            return mid + R * np.stack([np.cos(a), np.sin(a)], axis=1)
        return mid + fibonacci_sphere(M, R)
    lo = c.min(axis=0) - pr.max()
    hi = c.max(axis=0) + pr.max()
    out = []
    got = 0
    while got < M:
        cand = rng.uniform(lo, hi, size=(4 * M, d))
        dist = np.linalg.norm(cand[:, None, :] - c[None, :, :], axis=2) if len(c) * 4 * M < 4e7 else None
        if dist is None:
            ok = np.ones(len(cand), bool)
            for t in range(len(c)):
                ok &= np.linalg.norm(cand - c[t], axis=1) > pr[t] * 1.02
        else:
            ok = np.all(dist > pr[None, :] * 1.02, axis=1)
        sel = cand[ok][: M - got]
        out.append(sel)
        got += len(sel)
    return np.concatenate(out, axis=0)


@dataclass
class Request:
    rid: int
    arrival: float
    dim: int
    T: int
    kappa: float
    nrhs: int
    seed: int


def serving_trace(seed: int = 0, n: int = 512, rate: float = 20.0, Tmin: int = 20,
                  Tmax: int = 3000, p2d: float = 0.7) -> list:
    """Request stream: exponential inter-arrival times of mean 1/rate, body
    counts T ~ U{Tmin..Tmax}, 2D with probability p2d else 3D,
    kappa ~ U(5, 50), nrhs ~ U{1..32}."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n)
    arr = np.cumsum(gaps)
    Ts = rng.integers(Tmin, Tmax + 1, size=n)
    is2d = rng.uniform(size=n) < p2d
    kap = rng.uniform(5.0, 50.0, size=n)
    nr = rng.integers(1, 33, size=n)
    seeds = rng.integers(0, 2 ** 31 - 1, size=n)
    return [Request(i, float(arr[i]), 2 if is2d[i] else 3, int(Ts[i]), float(kap[i]), int(nr[i]),
                    int(seeds[i])) for i in range(n)]


def request_workload(req: Request, k2d: int = 64, k3d: int = 300, nth: int = 20, nph: int = 30,
                     p3d: int = 601) -> Workload:
    """Materialise one request: config1 construction (2D, box side scaled with
    sqrt(T/1000)) or config3 construction (3D)."""
    if req.dim == 2:
        wl = config1(seed=req.seed, T=req.T, kappa=req.kappa, nrhs=req.nrhs, k=k2d)
    else:
        wl = config3(seed=req.seed, T=req.T, kappa=req.kappa, nth=nth, nph=nph, p=p3d, k=k3d)
        ang = TWO_PI * np.arange(req.nrhs) / max(1, req.nrhs)
        wl.directions = np.stack([np.cos(ang) * 0.6, np.sin(ang) * 0.6,
                                  np.full_like(ang, 0.8)], axis=1)
    wl.name = f"request{req.rid}"
    return wl
