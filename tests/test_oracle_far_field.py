"""Pins of the oracle's fields off the surface (Green's representation of
Eq. cbie with c = 1 in the acoustic domain) and far-field pattern, for the
rigid unit sphere and a plane wave: both reached from the oracle's own
dense solution against the Mie series, the pattern as the large-radius
limit of the field, and reciprocity F(a; d) = F(-d; -a)."""
import numpy as np

import oracle
from inputs import icosphere, ellipsoid_from_icosphere, fibonacci_directions

K = 5.0


def _solve(v, f, k, d):
    a = oracle.assemble(v, f, k)
    return oracle.lu_solve(a, oracle.rhs_plane_wave(v, f, k, [d])[0])


def test_far_field_and_scattered_field_converge_to_mie():
    dirs = fibonacci_directions(40)
    pts = np.array([[0, 0, 1.5], [0, 2.0, 0.5], [-2.5, 0.3, 0.2], [0, 0, -3.0]])
    r = np.linalg.norm(pts, axis=1)
    ef, es = [], []
    for L in (2, 3, 4):
        v, f = icosphere(L)
        u = _solve(v, f, K, [0.0, 0.0, 1.0])
        F = oracle.far_field(v, f, K, u, dirs)
        ef.append(np.linalg.norm(F - oracle.mie_far_field(K, dirs[:, 2])) / np.linalg.norm(F))
        us = oracle.scattered_field(v, f, K, u, pts)
        um = oracle.mie_scattered_field(K, r, pts[:, 2] / r)
        es.append(np.linalg.norm(us - um) / np.linalg.norm(um))
    assert ef[2] < ef[1] / 3 < ef[0] / 9 and ef[2] < 1e-2
    assert es[2] < es[1] / 3 < es[0] / 9 and es[2] < 5e-3


def test_far_field_is_the_large_radius_limit():
    v, f = icosphere(3)
    u = _solve(v, f, K, [0.0, 0.0, 1.0])
    dirs = fibonacci_directions(12)
    F = oracle.far_field(v, f, K, u, dirs)
    gaps = []
    for R in (1e3, 1e4):
        us = oracle.scattered_field(v, f, K, u, dirs * R)
        gaps.append(np.linalg.norm(us * R / np.exp(1j * K * R) - F) / np.linalg.norm(F))
    assert gaps[1] < gaps[0] / 5 and gaps[1] < 1e-3


def test_reciprocity_on_an_ellipsoid():
    """F(a; d) = F(-d; -a) for the exact scattering; the discrete solutions
    keep it to discretisation accuracy."""
    d = np.array([0.0, 0.0, 1.0])
    a = np.array([0.6, 0.0, 0.8])
    gaps = []
    for L in (3, 4):
        v, f = ellipsoid_from_icosphere(L)
        f1 = oracle.far_field(v, f, 3.0, _solve(v, f, 3.0, d), [a])[0]
        f2 = oracle.far_field(v, f, 3.0, _solve(v, f, 3.0, -a), [-d])[0]
        gaps.append(abs(f1 - f2) / abs(f1))
    # first order in h (1.8e-2, 9.0e-3)
    assert gaps[1] < gaps[0] / 1.6 and gaps[1] < 1.5e-2
