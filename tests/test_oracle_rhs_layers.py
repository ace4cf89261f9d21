"""Pins of the oracle's right-hand-side layers of Eq. eq_bm acting on given
Neumann data q = du/dn (a radiating body):

    (B q)_i = -alpha q_i / 2 + sum_j int_{tri_j} [G + alpha dG/dn_x](x_i, y) dy q_j

against what the mathematics and the paper fix: the weakly singular self
integral by a Duffy-transformed brute force and a closed form, the
potential of a uniform layer on the sphere, the sphere eigenvalues beta_n,
and the pulsating-sphere errors printed in Table tab_usphpls (Sec. 5.1).
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle
from inputs import icosphere, octasphere

HERE = os.path.dirname(os.path.abspath(__file__))


def _duffy_single_layer(v, k):
    """int_tri e^{ikR}/(4 pi R) dA from the centroid x: the triangle split at
    x into three, each mapped by y = x + u ((a - x) + w (b - a)) on the unit
    square, where the 1/R singularity cancels against the Jacobian u."""
    x = v.mean(axis=0)
    tot = 0.0 + 0.0j
    for e in range(3):
        a, b = v[e], v[(e + 1) % 3]
        J = np.linalg.norm(np.cross(a - x, b - a))

        def f(u, w, part):
            rho = np.linalg.norm((a - x) + w * (b - a))
            val = np.exp(1j * k * u * rho) * J / (4 * np.pi * rho)
            return val.real if part == 0 else val.imag

        re = integrate.dblquad(f, 0, 1, 0, 1, args=(0,), epsabs=1e-13, epsrel=1e-12)[0]
        im = integrate.dblquad(f, 0, 1, 0, 1, args=(1,), epsabs=1e-13, epsrel=1e-12)[0]
        tot += re + 1j * im
    return tot


@pytest.mark.parametrize("k", [1e-3, 2.0, 30.0])
def test_self_single_layer_against_duffy_brute_force(k):
    v = np.array([[0.0, 0.0, 0.0], [0.13, 0.01, 0.02], [0.03, 0.11, -0.01]])
    f = np.array([[0, 1, 2]], dtype=np.int32)
    got = oracle.self_single_layer(v, f, 0, k)
    ref = _duffy_single_layer(v, k)
    assert abs(got - ref) < 1e-9 * abs(ref), (got, ref)


def test_self_single_layer_equilateral_closed_form():
    """k -> 0, equilateral triangle of inradius r: int 1/(4 pi R) dA from the
    centroid = 6 r ln(2 + sqrt 3)/(4 pi); the next term is i k area/(4 pi)."""
    s, k = 0.1, 1e-4
    v = np.array([[0, 0, 0], [s, 0, 0], [s / 2, s * math.sqrt(3) / 2, 0]], dtype=np.float64)
    f = np.array([[0, 1, 2]], dtype=np.int32)
    r = s / (2 * math.sqrt(3))
    got = oracle.self_single_layer(v, f, 0, k)
    assert abs(got.real - 6 * r * math.log(2 + math.sqrt(3)) / (4 * math.pi)) < 1e-9 * got.real
    # imaginary part int sin(kR)/(4 pi R) dA = k area/(4 pi) (1 + O(k^2 R^2)); at
    # k = 1e-2 (1 - cos(k rho))/k keeps nine digits
    k = 1e-2
    area = s * s * math.sqrt(3) / 4
    got = oracle.self_single_layer(v, f, 0, k)
    assert abs(got.imag - k * area / (4 * math.pi)) < 1e-5 * k * area / (4 * math.pi)


def test_rhs_self_entry_is_jump_plus_single_layer():
    """B_ii = -alpha/2 + int G (the adjoint double layer vanishes on a flat
    triangle); B_ij for a distant pair is the six-point rule of G + alpha dG/dn_x."""
    v, f = icosphere(2)
    k = 4.0
    for s_ in (1.0, -1.0):
        got = oracle.rhs_layers_entry(v, f, k, 7, 7, alpha_sign=s_)
        want = -0.5 * s_ * 1j / k + oracle.self_single_layer(v, f, 7, k)
        assert abs(got - want) < 1e-14 * abs(want)
    c, n, area, _ = oracle.geometry(v, f)
    i, j = 0, int(np.argmax(np.linalg.norm(c - c[0], axis=1)))
    pts, w = oracle.rule6()
    P = v[f[j]]
    ref = 0.0
    for (b1, b2), wq in zip(pts, w):
        y = P[0] + b1 * (P[1] - P[0]) + b2 * (P[2] - P[0])
        r = c[i] - y
        R = np.linalg.norm(r)
        g = np.exp(1j * k * R) / (4 * np.pi * R)
        dgdnx = -np.exp(1j * k * R) * (1 - 1j * k * R) * (r @ n[i]) / (4 * np.pi * R ** 3)
        ref += wq * area[j] * (g + (1j / k) * dgdnx)
    assert abs(oracle.rhs_layers_entry(v, f, k, i, j, alpha_sign=1.0) - ref) < 1e-13 * abs(ref)


def test_uniform_single_layer_potential_on_sphere():
    """k -> 0 and no coupling (alpha = 0): sum_j B_ij = S[1] = 1 on the unit
    sphere (a uniform unit layer's potential at its surface), converging
    under refinement."""
    errs = []
    for L in (2, 3, 4):
        v, f = icosphere(L)
        s1 = oracle.rhs_layers_matvec(v, f, 1e-4, np.ones(len(f)), alpha_sign=0.0)
        errs.append(np.abs(s1.real - 1.0).max())
    assert errs[2] < errs[1] / 2 < errs[0] / 4
    assert errs[2] < 5e-3


@pytest.mark.parametrize("alpha_sign", [1.0, -1.0])
def test_rhs_layer_eigenvalues_converge(alpha_sign):
    """B P_n ~ beta_n P_n on the unit sphere: the Rayleigh quotient converges
    to the closed form as the mesh is refined.  A dropped term (the jump, the
    adjoint double layer or the single layer) or a wrong sign moves beta_n by
    O(1) and fails here."""
    k = 3.0
    errs = {}
    for L in (2, 3, 4):
        v, f = icosphere(L)
        c, *_ = oracle.geometry(v, f)
        for n in (0, 1, 2, 4):
            x = oracle.legendre_on_mesh(c, n)
            y = oracle.rhs_layers_matvec(v, f, k, x, alpha_sign=alpha_sign)
            beta = np.vdot(x, y) / np.vdot(x, x)
            ref = oracle.sphere_rhs_eigenvalue(n, k, alpha_sign)
            errs[(L, n)] = abs(beta - ref) / abs(ref)
    # first order in h (flat facets, constant elements), pre-asymptotic at level 2
    for n in (0, 1, 2, 4):
        assert errs[(4, n)] < errs[(3, n)] and errs[(4, n)] < errs[(2, n)] / 2.5
        assert errs[(4, n)] < 2e-2


def test_closed_forms_consistent():
    """beta_0 / lambda_0 is the pulsating-sphere potential 1/(1 - ik) for
    either sign of the coupling."""
    for k in (0.5, math.pi, 7.3):
        for s_ in (1.0, -1.0):
            r = oracle.sphere_rhs_eigenvalue(0, k, s_) / oracle.sphere_eigenvalue(0, k, s_)
            assert abs(r - oracle.pulsating_sphere_potential(k)) < 1e-12


def _paper_table():
    rows = []
    for line in open(os.path.join(HERE, "golden", "pulsating_sphere_table.txt")):
        if line.strip() and not line.startswith("#"):
            n, kp, eps, it, err = line.split()
            rows.append((int(n), float(kp), float(eps), int(it), float(err)))
    return rows


def test_pulsating_sphere_matches_paper_table():
    """Dense LU of A u = B 1 on the paper's sphere family (N = 512, 2048 with
    k = pi, 2 pi): the relative L2 error against 1/(1 - ik) is within 10% of
    the errors printed in Table tab_usphpls (there dominated by the
    discretisation), and it halves when N quadruples and k doubles."""
    paper = {(n, kp): err for n, kp, eps, it, err in _paper_table() if eps == 1e-3}
    errs = []
    for level, kp in ((3, 1.0), (4, 2.0)):
        v, f = octasphere(level)
        k = kp * math.pi
        a = oracle.assemble(v, f, k)
        b = oracle.rhs_layers_assemble(v, f, k) @ np.ones(len(f))
        u = oracle.lu_solve(a, b)
        ue = oracle.pulsating_sphere_potential(k)
        err = np.linalg.norm(u - ue) / (abs(ue) * math.sqrt(len(f)))
        errs.append(err)
        assert abs(err - paper[(len(f), kp)]) < 0.1 * paper[(len(f), kp)], (len(f), err)
    assert 1.6 < errs[0] / errs[1] < 2.4


def _brute_single_layer(x, nx, p, k):
    """adaptive 2-D quadrature of G + alpha dG/dn_x over triangle p"""
    p = np.asarray(p)
    e1, e2 = p[1] - p[0], p[2] - p[0]
    jac = np.linalg.norm(np.cross(e1, e2))
    alpha = 1j / k

    def f(t, s, part):
        y = p[0] + s * e1 + t * e2
        g = oracle.kernels(x, nx, y, nx, k)
        v = (g[0] + alpha * g[2]) * jac
        return v.real if part == 0 else v.imag

    re = integrate.dblquad(f, 0, 1, 0, lambda s: 1 - s, args=(0,), epsabs=1e-12, epsrel=1e-11)[0]
    im = integrate.dblquad(f, 0, 1, 0, lambda s: 1 - s, args=(1,), epsabs=1e-12, epsrel=1e-11)[0]
    return re + 1j * im


@pytest.mark.parametrize("case", ["edge_neighbour", "vertex_neighbour", "far"])
def test_rhs_element_rules_against_brute_force(case):
    """The right-hand side's layers through the same element rules: near
    pairs (subdivided rule) and far pairs (six-point rule) against adaptive
    quadrature of G + alpha dG/dn_x."""
    v, f = icosphere(2)
    c, n, a, h2 = oracle.geometry(v, f)
    i = 0
    shared = [len(set(f[i]) & set(f[j])) for j in range(len(f))]
    if case == "edge_neighbour":
        j = next(j for j in range(len(f)) if shared[j] == 2)
    elif case == "vertex_neighbour":
        j = next(j for j in range(len(f)) if shared[j] == 1)
    else:
        j = int(np.argmax(np.linalg.norm(c - c[i], axis=1)))
    k = 5.0
    got = oracle.rhs_layers_entry(v, f, k, i, j, alpha_sign=1.0)
    ref = _brute_single_layer(c[i], n[i], v[f[j]], k)
    tol = 1e-4 if case != "far" else 1e-6
    assert abs(got - ref) < tol * abs(ref), (got, ref)
