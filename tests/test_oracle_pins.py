"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: finite
differences of G, exact polynomial integrals, brute-force adaptive
quadrature, Hadamard finite parts by disk exclusion, the k -> 0 Gauss
identity, the sphere eigenvalues, the Mie series (itself pinned by mpmath
and the Rayleigh limit), icosahedral symmetry, and LU vs GMRES.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from inputs import icosphere, icosahedral_rotations

K = 3.0


# ---------------------------------------------------------------- kernels
def _g(x, y, k):
    r = np.linalg.norm(np.asarray(x) - np.asarray(y))
    return np.exp(1j * k * r) / (4 * np.pi * r)


@pytest.mark.parametrize("k", [0.7, 5.0, 40.0])
def test_kernel_derivatives_match_finite_differences(k):
    """dG/dn_y, dG/dn_x and d2G/dn_x dn_y (Eq. eq_bm's layer kernels) agree
    with central differences of G = e^{ikr}/(4 pi r)."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        x = rng.normal(size=3)
        y = x + rng.normal(size=3) * 0.3 + 0.2
        nx = rng.normal(size=3); nx /= np.linalg.norm(nx)
        ny = rng.normal(size=3); ny /= np.linalg.norm(ny)
        G, dny, dnx, d2 = oracle.kernels(x, nx, y, ny, k)
        h = 1e-5
        assert abs(G - _g(x, y, k)) < 1e-14 * abs(G) + 1e-300
        fd_ny = (_g(x, y + h * ny, k) - _g(x, y - h * ny, k)) / (2 * h)
        fd_nx = (_g(x + h * nx, y, k) - _g(x - h * nx, y, k)) / (2 * h)
        h2 = 1e-4
        fd_2 = (_g(x + h2 * nx, y + h2 * ny, k) - _g(x + h2 * nx, y - h2 * ny, k)
                - _g(x - h2 * nx, y + h2 * ny, k) + _g(x - h2 * nx, y - h2 * ny, k)) / (4 * h2 * h2)
        assert abs(dny - fd_ny) < 1e-7 * (abs(dny) + abs(G))
        assert abs(dnx - fd_nx) < 1e-7 * (abs(dnx) + abs(G))
        assert abs(d2 - fd_2) < 1e-5 * (abs(d2) + abs(G))


def test_kernel_symmetries():
    """G(x,y) = G(y,x); d2G is invariant under (x, n_x) <-> (y, n_y);
    dG/dn_y(x,y) = dG/dn_x(y,x) with the normals swapped."""
    rng = np.random.default_rng(5)
    x, y = rng.normal(size=3), rng.normal(size=3)
    nx = rng.normal(size=3); nx /= np.linalg.norm(nx)
    ny = rng.normal(size=3); ny /= np.linalg.norm(ny)
    a = oracle.kernels(x, nx, y, ny, 4.0)
    b = oracle.kernels(y, ny, x, nx, 4.0)
    assert abs(a[0] - b[0]) < 1e-15 * abs(a[0])
    assert abs(a[3] - b[3]) < 1e-13 * abs(a[3])
    assert abs(a[1] - b[2]) < 1e-13 * abs(a[1])


# ---------------------------------------------------------------- quadrature
def test_regular_rule_is_exact_to_degree_4():
    """The six-point rule integrates every monomial x^a y^b, a + b <= 4,
    exactly over the reference triangle (exact value a! b! / (a+b+2)!), and
    misses some degree-5 monomial."""
    pts, w = oracle.rule6()
    assert abs(w.sum() - 1.0) < 1e-15
    area = 0.5
    for a in range(5):
        for b in range(5 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            got = area * np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b)
            assert abs(got - exact) < 1e-15, (a, b)
    miss = [abs(area * np.sum(w * pts[:, 0] ** a * pts[:, 1] ** (5 - a))
                - math.factorial(a) * math.factorial(5 - a) / math.factorial(7)) for a in range(6)]
    assert max(miss) > 1e-6


def test_gauss_legendre_nodes():
    xs, ws = oracle.gauss_legendre(16)
    rx, rw = np.polynomial.legendre.leggauss(16)
    assert np.allclose(xs, rx, atol=1e-14) and np.allclose(ws, rw, atol=1e-14)


def _brute_triangle(x, nx, p, ny, k):
    """adaptive 2-D quadrature of the Burton-Miller kernel over triangle p"""
    p = np.asarray(p)
    e1, e2 = p[1] - p[0], p[2] - p[0]
    jac = np.linalg.norm(np.cross(e1, e2))
    alpha = 1j / k

    def f(t, s, part):
        y = p[0] + s * e1 + t * e2
        g = oracle.kernels(x, nx, y, ny, k)
        v = (g[1] + alpha * g[3]) * jac
        return v.real if part == 0 else v.imag

    re = integrate.dblquad(f, 0, 1, 0, lambda s: 1 - s, args=(0,), epsabs=1e-11, epsrel=1e-10)[0]
    im = integrate.dblquad(f, 0, 1, 0, lambda s: 1 - s, args=(1,), epsabs=1e-11, epsrel=1e-10)[0]
    return re + 1j * im


@pytest.mark.parametrize("case", ["edge_neighbour", "vertex_neighbour", "far"])
def test_element_rules_against_brute_force(case):
    """Near pairs: the subdivided rule (4^3 sub-triangles x 6 points) and far
    pairs: the plain six-point rule, against adaptive quadrature."""
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
    near = oracle.is_near_pair(v, f, i, j)
    assert near == (case != "far")
    k = 5.0
    got = oracle.entry(v, f, k, i, j, alpha_sign=1.0)
    ref = _brute_triangle(c[i], n[i], v[f[j]], n[j], k)
    tol = 2e-4 if case != "far" else 1e-6
    assert abs(got - ref) < tol * abs(ref), (got, ref)


def _fp_disk_exclusion(verts, k, eps):
    """Hadamard finite part of int e^{ikR}(1-ikR)/(4 pi R^3) over a flat
    triangle about its centroid, by excluding a disk of radius eps: the
    regular integral over the rest (adaptive polar quadrature) plus the
    finite part of the disk, (1/2)(ik - e^{ik eps}/eps)."""
    p = np.asarray(verts)
    c = p.mean(axis=0)
    e1 = p[1] - p[0]; e1 /= np.linalg.norm(e1)
    nrm = np.cross(p[1] - p[0], p[2] - p[0]); nrm /= np.linalg.norm(nrm)
    e2 = np.cross(nrm, e1)
    q = np.stack([(p - c) @ e1, (p - c) @ e2], axis=1)

    def rho(t):
        d = np.array([math.cos(t), math.sin(t)])
        best = np.inf
        for a in range(3):
            a0, a1 = q[a], q[(a + 1) % 3]
            m = np.array([[d[0], a0[0] - a1[0]], [d[1], a0[1] - a1[1]]])
            if abs(np.linalg.det(m)) < 1e-14:
                continue
            s, u = np.linalg.solve(m, a0)
            if s > 0 and -1e-12 <= u <= 1 + 1e-12:
                best = min(best, s)
        return best

    def radial(t, part):
        r1 = rho(t)
        g = lambda r: (np.exp(1j * k * r) * (1 - 1j * k * r) / (4 * np.pi * r ** 2))
        fn = (lambda r: g(r).real) if part == 0 else (lambda r: g(r).imag)
        return integrate.quad(fn, eps, r1, epsabs=1e-13, epsrel=1e-12, limit=200)[0]

    corners = sorted(math.atan2(qq[1], qq[0]) % (2 * math.pi) for qq in q)
    pts = corners
    re = integrate.quad(radial, 0, 2 * math.pi, args=(0,), points=pts, epsabs=1e-11, epsrel=1e-11, limit=200)[0]
    im = integrate.quad(radial, 0, 2 * math.pi, args=(1,), points=pts, epsabs=1e-11, epsrel=1e-11, limit=200)[0]
    return re + 1j * im + 0.5 * (1j * k - np.exp(1j * k * eps) / eps)


@pytest.mark.parametrize("k", [1e-6, 2.0, 30.0])
def test_self_term_finite_part(k):
    """Self element: the oracle's finite part equals the disk-exclusion
    definition for an irregular triangle; at k -> 0 the equilateral case
    has the closed form -(1/(4 pi)) * 3 sqrt(3)/d (d = inradius)."""
    v = np.array([[0.0, 0.0, 0.0], [0.13, 0.01, 0.02], [0.03, 0.11, -0.01]])
    f = np.array([[0, 1, 2]], dtype=np.int32)
    got = oracle.self_hypersingular(v, f, 0, k)
    ref = _fp_disk_exclusion(v, k, 1e-3)
    assert abs(got - ref) < 1e-7 * abs(ref), (got, ref)
    s = 0.1
    ve = np.array([[0, 0, 0], [s, 0, 0], [s / 2, s * math.sqrt(3) / 2, 0]], dtype=np.float64)
    d = s / (2 * math.sqrt(3))
    got_e = oracle.self_hypersingular(ve, f, 0, 1e-9)
    assert abs(got_e - (-(3 * math.sqrt(3) / d) / (4 * np.pi))) < 1e-10 * abs(got_e)


# ---------------------------------------------------------------- operator
def test_gauss_identity_and_hypersingular_of_constant():
    """k -> 0: 1/2 + sum_j D_ij = 1 (solid angle of a closed surface, normal
    into the body) and sum_j H_ij = 0 (the hypersingular operator kills
    constants), both relative to the entry scale 1/h."""
    v, f = icosphere(3)
    d = oracle.layer_rowsum(v, f, 1e-8, 1)
    h = oracle.layer_rowsum(v, f, 1e-8, 2)
    _, _, _, h2 = oracle.geometry(v, f)
    assert np.abs(d - 1.0).max() < 1e-5
    assert np.abs(h).max() * np.sqrt(h2.mean()) < 1e-5


@pytest.mark.parametrize("alpha_sign", [1.0, -1.0])
def test_sphere_eigenvalues_converge(alpha_sign):
    """A P_n ~ lambda_n P_n on the unit sphere: the Rayleigh quotient
    converges to lambda_n (closed form) as the mesh is refined, for both
    signs of the coupling alpha = +-i/k."""
    errs = {}
    for L in (2, 3, 4):
        v, f = icosphere(L)
        c, *_ = oracle.geometry(v, f)
        for n in (0, 1, 2, 4):
            x = oracle.legendre_on_mesh(c, n)
            y = oracle.matvec(v, f, K, x, alpha_sign=alpha_sign)
            lam = np.vdot(x, y) / np.vdot(x, x)
            ref = oracle.sphere_eigenvalue(n, K, alpha_sign)
            errs[(L, n)] = abs(lam - ref) / abs(ref)
    for n in (0, 1, 2, 4):
        assert errs[(4, n)] < errs[(3, n)] / 2.5 < errs[(2, n)] / 5
        assert errs[(4, n)] < 8e-3


def test_icosahedral_symmetry_commutes():
    """Rotating the mesh by an icosahedral rotation permutes its elements;
    the operator commutes with that permutation."""
    v, f = icosphere(2)
    c, *_ = oracle.geometry(v, f)
    rots = icosahedral_rotations()
    x = np.random.default_rng(1).normal(size=len(f)) + 1j * np.random.default_rng(2).normal(size=len(f))
    y = oracle.matvec(v, f, 4.0, x)
    for r in rots[1:6]:
        rc = c @ r.T
        perm = np.array([int(np.argmin(np.linalg.norm(c - p, axis=1))) for p in rc])
        assert np.allclose(c[perm], rc, atol=1e-12)
        # element e maps to perm[e]: (P x)[perm[e]] = x[e]
        px = np.empty_like(x); px[perm] = x
        py = np.empty_like(y); py[perm] = y
        assert np.linalg.norm(oracle.matvec(v, f, 4.0, px) - py) < 1e-11 * np.linalg.norm(y)


# ---------------------------------------------------------------- closed forms
def test_mie_series_against_mpmath_and_rayleigh():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    k = 3.7
    cts = np.array([-0.9, -0.2, 0.35, 1.0])

    def h1p(n, x):
        x = mp.mpf(x)
        j = lambda m: mp.sqrt(mp.pi / (2 * x)) * mp.besselj(m + mp.mpf(1) / 2, x)
        y = lambda m: mp.sqrt(mp.pi / (2 * x)) * mp.bessely(m + mp.mpf(1) / 2, x)
        h = lambda m: j(m) + 1j * y(m)
        return h(n - 1) - (n + 1) / x * h(n) if n > 0 else -h(1)

    ref = []
    for ct in cts:
        s = mp.mpc(0)
        for n in range(0, 40):
            s += (2 * n + 1) * (1j ** n) * (1j / (k * k)) / h1p(n, k) * mp.legendre(n, ct)
        ref.append(complex(s))
    got = oracle.mie_surface_field(k, cts)
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-12)
    # Rayleigh limit: u = 1 + (3/2) i k cos(theta) + O(k^2)
    ks = 1e-3
    u = oracle.mie_surface_field(ks, cts)
    assert np.allclose(u, 1 + 1.5j * ks * cts, atol=5e-6)


@pytest.mark.parametrize("alpha_sign", [1.0, -1.0])
def test_eigenvalues_consistent_with_mie(alpha_sign):
    """lambda_n (i/k^2)/h_n'(k) = j_n(k) - s i j_n'(k) for alpha = s i/k: the
    operator's eigenvalue applied to the Mie coefficient reproduces the
    plane-wave right-hand side's expansion coefficient (u_inc + alpha
    du_inc/dn with n = -r on the unit sphere)."""
    from scipy import special
    for k in (0.5, 5.0, 25.0):
        for n in range(0, 12):
            hd = special.spherical_jn(n, k, True) + 1j * special.spherical_yn(n, k, True)
            lhs = oracle.sphere_eigenvalue(n, k, alpha_sign) * (1j / k ** 2) / hd
            rhs = special.spherical_jn(n, k) - alpha_sign * 1j * special.spherical_jn(n, k, True)
            assert abs(lhs - rhs) < 1e-10 * (abs(rhs) + 1e-30)


# ---------------------------------------------------------------- solve
def test_conjugate_coupling_same_solution_right_half_plane():
    """Both couplings solve the same scattering problem (their LU solutions
    agree with each other and with the Mie series to discretisation error);
    with the normal into the body, alpha = -i/k keeps every sphere eigenvalue
    in the right half-plane while alpha = +i/k spreads them around 0, which is
    why GMRES needs more iterations for +i/k."""
    k = 5.0
    v, f = icosphere(3)
    c, *_ = oracle.geometry(v, f)
    ct = (c / np.linalg.norm(c, axis=1, keepdims=True))[:, 2]
    um = oracle.mie_surface_field(k, ct)
    sols = {}
    for s_ in (1.0, -1.0):
        a = oracle.assemble(v, f, k, alpha_sign=s_)
        b = oracle.rhs_plane_wave(v, f, k, [[0.0, 0.0, 1.0]], alpha_sign=s_)[0]
        sols[s_] = oracle.lu_solve(a, b)
        assert np.linalg.norm(sols[s_] - um) / np.linalg.norm(um) < 2e-2
    assert np.linalg.norm(sols[1.0] - sols[-1.0]) / np.linalg.norm(sols[1.0]) < 2e-2
    lam_p = np.array([oracle.sphere_eigenvalue(n, 20.0, 1.0) for n in range(60)])
    lam_m = np.array([oracle.sphere_eigenvalue(n, 20.0, -1.0) for n in range(60)])
    assert lam_m.real.min() > 0.4 and lam_p.real.min() < -0.5
    # where it shows (kD = 40): fewer GMRES iterations for -i/k
    iters = {}
    for s_ in (1.0, -1.0):
        a = oracle.assemble(v, f, 20.0, alpha_sign=s_)
        b = oracle.rhs_plane_wave(v, f, 20.0, [[0.0, 0.0, 1.0]], alpha_sign=s_)[0]
        _, iters[s_], _ = oracle.gmres(lambda z: a @ z, b, tol=1e-6, restart=400)
    assert iters[-1.0] < 0.8 * iters[1.0]


def test_solution_converges_to_mie_and_gmres_matches_lu():
    """Rigid sphere, plane wave e^{ikz}, k = 5: the dense-LU solution's error
    against the Mie series decays under refinement, and GMRES at tol 1e-9
    reproduces LU."""
    k = 5.0
    errs = []
    for L in (2, 3, 4):
        v, f = icosphere(L)
        c, *_ = oracle.geometry(v, f)
        a = oracle.assemble(v, f, k)
        b = oracle.rhs_plane_wave(v, f, k, [[0.0, 0.0, 1.0]])[0]
        u = oracle.lu_solve(a, b)
        ct = (c / np.linalg.norm(c, axis=1, keepdims=True))[:, 2]
        um = oracle.mie_surface_field(k, ct)
        errs.append(np.linalg.norm(u - um) / np.linalg.norm(um))
        if L == 3:
            x, it, hist = oracle.gmres(lambda z: a @ z, b, tol=1e-9, restart=60)
            assert hist[-1] <= 1e-9
            assert np.linalg.norm(x - u) < 1e-7 * np.linalg.norm(u)
    assert errs[2] < errs[1] / 2 < errs[0] / 4
    assert errs[2] < 1e-2
