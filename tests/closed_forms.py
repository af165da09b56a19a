"""Textbook separation-of-variables solutions used to pin the oracle.

Sound-soft scattering of a plane wave u_inc = exp(i kappa d.x) by one circle
or one sphere of radius a centred at the origin; the scattered field u
satisfies u = -u_inc on the boundary and the radiation condition.  These are
the classical series (e.g. Colton & Kress, "Inverse Acoustic and
Electromagnetic Scattering Theory", Sec. 3.4 / 2D analogue): they use nothing
from the oracle.
"""
import numpy as np
from scipy.special import eval_legendre, hankel1, jv, spherical_jn, spherical_yn


def circle_scattered(kappa, a, alpha, pts, nmax=None):
    """u(r, theta) = -sum_n i^n J_n(ka)/H_n(ka) H_n(kr) e^{i n (theta - alpha)}."""
    r = np.hypot(pts[:, 0], pts[:, 1])
    th = np.arctan2(pts[:, 1], pts[:, 0])
    ka = kappa * a
    nmax = nmax or int(ka + 40 + 4 * ka ** (1 / 3))
    u = np.zeros(len(r), dtype=np.complex128)
    for n in range(-nmax, nmax + 1):
        coef = (1j ** n) * jv(n, ka) / hankel1(n, ka)
        u -= coef * hankel1(n, kappa * r) * np.exp(1j * n * (th - alpha))
    return u


def sphere_scattered(kappa, a, d, pts, nmax=None):
    """u = -sum_n i^n (2n+1) j_n(ka)/h_n(ka) h_n(kr) P_n(cos gamma), gamma = angle(x, d)."""
    r = np.linalg.norm(pts, axis=1)
    cg = (pts @ np.asarray(d)) / r
    ka = kappa * a
    nmax = nmax or int(ka + 40 + 4 * ka ** (1 / 3))
    u = np.zeros(len(r), dtype=np.complex128)
    for n in range(nmax + 1):
        ha = spherical_jn(n, ka) + 1j * spherical_yn(n, ka)
        hr = spherical_jn(n, kappa * r) + 1j * spherical_yn(n, kappa * r)
        u -= (1j ** n) * (2 * n + 1) * spherical_jn(n, ka) / ha * hr * eval_legendre(n, cg)
    return u
