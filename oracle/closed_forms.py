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

Right-hand side's layers of Eq. eq_bm acting on q = du/dn,
B = -alpha/2 + S + alpha K' (S single layer, K' its normal derivative in n,
direct value): B[P_n] = beta_n P_n,
    beta_n = -alpha/2 + i k j_n h_n - alpha (i k^2/2)(j_n h_n' + j_n' h_n),
since S[Y_n] = i k j_n h_n Y_n on the unit sphere and the radial derivative
of the single-layer potential is i k^2 j_n h_n' outside and i k^2 j_n' h_n
inside (their mean is the direct value in nu; n = -nu flips its sign).

Point source at x_s, |x_s| = r_s > 1, outside the rigid unit sphere (the
comparison of Sec. 5.2): with the addition theorem
G(x, x_s) = (ik/4pi) sum_n (2n+1) j_n(k r) h_n(k r_s) P_n(cos gamma), a
scattered field sum_n a_n h_n(k r) P_n with zero total radial derivative at
r = 1 and the Wronskian leave on the surface
    u(gamma) = -(1/(4 pi k)) sum_n (2n+1) h_n(k r_s) P_n(cos gamma) / h_n'(k),
gamma the angle between x and x_s.

Pulsating unit sphere (Sec. 5.1), du/dn = 1 with n into the body: the
radiating solution u = A e^{ikr}/r gives u = 1/(1 - ik) on the surface
(beta_0 / lambda_0 equals it for either sign of alpha).
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


def sphere_eigenvalue(n: int, k: float, alpha_sign: float = -1.0) -> complex:
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


def sphere_rhs_eigenvalue(n: int, k: float, alpha_sign: float = -1.0) -> complex:
    """beta_n for alpha = alpha_sign i/k: -alpha/2 + S + alpha K' on P_n."""
    jn = special.spherical_jn(n, k)
    jd = special.spherical_jn(n, k, derivative=True)
    hn = _h1(n, k)
    hd = _h1(n, k, derivative=True)
    alpha = alpha_sign * 1j / k
    return -0.5 * alpha + 1j * k * jn * hn - alpha * 0.5j * k * k * (jn * hd + jd * hn)


def pulsating_sphere_potential(k: float) -> complex:
    """Surface potential of the unit sphere pulsating with du/dn = 1 (n into the body)."""
    return 1.0 / (1.0 - 1j * k)


def point_source_surface_field(k: float, rs: float, cos_gamma, nmax: int | None = None):
    """Total surface field of the rigid unit sphere for u_inc = G(x, x_s), |x_s| = rs."""
    ct = np.asarray(cos_gamma, dtype=np.float64)
    nmax = mie_nmax(k) + int(np.ceil(10.0 / np.log(rs))) if nmax is None else nmax
    u = np.zeros(ct.shape, dtype=np.complex128)
    for n in range(nmax + 1):
        u += (-(2 * n + 1) / (4 * np.pi * k)) * _h1(n, k * rs) / _h1(n, k, derivative=True) * \
            special.eval_legendre(n, ct)
    return u


def mie_scattered_field(k: float, r, cos_theta, nmax: int | None = None):
    """Scattered field of the rigid unit sphere for e^{ik d.x} at radius r >= 1:
    sum_n a_n h_n(k r) P_n(cos theta), a_n = -(2n+1) i^n j_n'(k)/h_n'(k)."""
    ct = np.asarray(cos_theta, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    nmax = mie_nmax(k) if nmax is None else nmax
    u = np.zeros(np.broadcast(ct, r).shape, dtype=np.complex128)
    for n in range(nmax + 1):
        an = -(2 * n + 1) * (1j ** n) * special.spherical_jn(n, k, derivative=True) / _h1(n, k, derivative=True)
        u += an * _h1(n, k * r) * special.eval_legendre(n, ct)
    return u


def mie_far_field(k: float, cos_theta, nmax: int | None = None):
    """Far-field pattern of the rigid unit sphere, u_sc ~ e^{ikr}/r F:
    F = (i/k) sum_n (2n+1) j_n'(k)/h_n'(k) P_n(cos theta) (h_n(x) ~ (-i)^{n+1} e^{ix}/x)."""
    ct = np.asarray(cos_theta, dtype=np.float64)
    nmax = mie_nmax(k) if nmax is None else nmax
    f = np.zeros(ct.shape, dtype=np.complex128)
    for n in range(nmax + 1):
        f += (2 * n + 1) * special.spherical_jn(n, k, derivative=True) / _h1(n, k, derivative=True) * \
            special.eval_legendre(n, ct)
    return (1j / k) * f
