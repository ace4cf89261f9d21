"""Closed forms on the unit sphere that pin the oracle (test infrastructure).

Convention: n = normal into the body (n = -nu with nu the outward radial
unit vector on the unit sphere), alpha = i/k, G = e^{ikr}/(4 pi r), as in
the paper's Eq. cbie / eq_bm.

Mie series (rigid unit sphere, incident e^{ik d.x}): the total field on the
surface is
    u(theta) = (i/k^2) sum_n (2n+1) i^n P_n(cos theta) / h_n'(k),
theta the angle between x and d, h_n = spherical Hankel function of the
first kind (Wronskian j_n y_n' - j_n' y_n = 1/x^2).

Sphere eigenvalues of the discretised operator's continuous counterpart
A = 1/2 + D + alpha H (D double layer with n, H hypersingular):
    A[P_n] = lambda_n P_n,
    lambda_n = 1/2 - (i k^2/2)(j_n' h_n + j_n h_n') - k^2 j_n' h_n',
from the addition theorem (the double layer's principal value is the mean
of its two one-sided limits; H is continuous across the sphere).
"""
from __future__ import annotations

import numpy as np
from scipy import special


def _h1(n, x, derivative=False):
    return (special.spherical_jn(n, x, derivative=derivative)
            + 1j * special.spherical_yn(n, x, derivative=derivative))


def mie_nmax(k: float) -> int:
    return int(np.ceil(k + 10.0 * k ** (1.0 / 3.0) + 10.0))


def mie_surface_field(k: float, cos_theta, nmax: int | None = None):
    """Total surface field of the rigid unit sphere for a plane wave e^{ik d.x}."""
    ct = np.asarray(cos_theta, dtype=np.float64)
    nmax = mie_nmax(k) if nmax is None else nmax
    u = np.zeros(ct.shape, dtype=np.complex128)
    for n in range(nmax + 1):
        coef = (2 * n + 1) * (1j ** n) * (1j / (k * k)) / _h1(n, k, derivative=True)
        u += coef * special.eval_legendre(n, ct)
    return u


def sphere_eigenvalue(n: int, k: float, alpha_sign: float = 1.0) -> complex:
    """lambda_n for alpha = alpha_sign i/k: 1/2 + D + alpha H with
    D[Y_n] = -(i k^2/2)(j_n' h_n + j_n h_n') Y_n and H[Y_n] = i k^3 j_n' h_n' Y_n."""
    jn = special.spherical_jn(n, k)
    jd = special.spherical_jn(n, k, derivative=True)
    hn = _h1(n, k)
    hd = _h1(n, k, derivative=True)
    alpha = alpha_sign * 1j / k
    return 0.5 - 0.5j * k * k * (jd * hn + jn * hd) + alpha * 1j * k ** 3 * jd * hd


def legendre_on_mesh(centroids, n: int, axis=(0.0, 0.0, 1.0)):
    """P_n(cos theta_i) at the radial projection of each centroid."""
    c = np.asarray(centroids, dtype=np.float64)
    u = c / np.linalg.norm(c, axis=1, keepdims=True)
    return special.eval_legendre(n, u @ np.asarray(axis, dtype=np.float64))
