"""Fields off the surface (fda_scattered_field) and far-field pattern
(fda_far_field) against the FP64 oracle on the same surface data (only the
summation order differs: <= 1e-12), and end to end from a GPU solution
against the Mie series and reciprocity."""
import numpy as np
import pytest

import oracle
from inputs import icosphere, ellipsoid_from_icosphere, complex_normal, fibonacci_directions

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_4747_gb300 import build
    build.build()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


def test_field_kernels_match_oracle():
    from paper_1403_4747_gb300 import FDAProblem
    v, f = ellipsoid_from_icosphere(3)
    k = 7.0
    P = FDAProblem(v, f, k)
    u = complex_normal(len(f), seed=31)
    q = complex_normal(len(f), seed=32)
    dirs = fibonacci_directions(37)  # not a multiple of the block's four targets
    pts = np.random.default_rng(3).normal(size=(23, 3))
    pts *= (1.5 + np.random.default_rng(4).random(23))[:, None] / np.linalg.norm(pts, axis=1, keepdims=True)
    for qq in (None, q):
        F = P.far_field(_dev(u), dirs, None if qq is None else _dev(qq)).cpu().numpy()
        assert _rel(F, oracle.far_field(v, f, k, u, dirs, q=qq)) < 1e-12
        us = P.scattered_field(_dev(u), pts, None if qq is None else _dev(qq)).cpu().numpy()
        assert _rel(us, oracle.scattered_field(v, f, k, u, pts, q=qq)) < 1e-12
    P.close()


def test_far_field_of_gpu_solution_against_mie():
    from paper_1403_4747_gb300 import FDAProblem
    k = 5.0
    v, f = icosphere(5)
    P = FDAProblem(v, f, k, precision=1)
    u, info = P.solve(P.rhs_plane_wave([0.0, 0.0, 1.0]), 1e-6)
    dirs = fibonacci_directions(60)
    F = P.far_field(u, dirs).cpu().numpy()
    assert _rel(F, oracle.mie_far_field(k, dirs[:, 2])) < 3e-3
    pts = dirs[:10] * 2.0
    us = P.scattered_field(u, pts).cpu().numpy()
    assert _rel(us, oracle.mie_scattered_field(k, 2.0, dirs[:10, 2])) < 2e-3
    P.close()


def test_reciprocity_from_gpu_solutions():
    from paper_1403_4747_gb300 import FDAProblem
    v, f = ellipsoid_from_icosphere(5)
    P = FDAProblem(v, f, 3.0, precision=1)
    d = np.array([0.0, 0.0, 1.0])
    a = np.array([0.6, 0.0, 0.8])
    u1, _ = P.solve(P.rhs_plane_wave(d), 1e-7)
    u2, _ = P.solve(P.rhs_plane_wave(-a), 1e-7)
    f1 = P.far_field(u1, [a]).cpu().numpy()[0]
    f2 = P.far_field(u2, [-d]).cpu().numpy()[0]
    assert abs(f1 - f2) < 7e-3 * abs(f1)  # oracle at level 4: 9.0e-3, first order in h
    P.close()


@pytest.mark.parametrize("mesh,k", [("sphere4", 20.0), ("ellipsoid4", 15.0), ("sphere5", 25.0)])
@pytest.mark.parametrize("with_q", [False, True])
def test_fast_pattern_matches_direct_and_oracle(mesh, k, with_q):
    """fda_far_field_fast (the upward pass of the fast algorithm: S2M, M2M,
    and each box's equivalent sources at the coarsest far-field level, the
    cone of the direction at a high-frequency level) agrees with the direct
    six-point sums and the oracle's pattern.  Bound 1e-3: a high-frequency
    cone's densities are fitted on check points out to the body's size plus
    two box widths, and the pattern (the field at infinity) extrapolates
    beyond them, which lets the eps = 1e-4 truncation grow a few times
    (2.0e-4 measured on the level-4 sphere at k = 20)."""
    from paper_1403_4747_gb300 import FDAProblem
    level = int(mesh[-1])
    v, f = icosphere(level) if mesh.startswith("sphere") else ellipsoid_from_icosphere(level)
    P = FDAProblem(v, f, k)
    st = P.stats()
    assert any(st.level_regime[l] == 1 for l in range(st.n_levels)) or level < 5
    u = complex_normal(len(f), seed=41)
    q = complex_normal(len(f), seed=42) if with_q else None
    dirs = fibonacci_directions(61)
    ud, qd = _dev(u), (_dev(q) if with_q else None)
    fast = P.far_field(ud, dirs, qd, fast=True).cpu().numpy()
    direct = P.far_field(ud, dirs, qd).cpu().numpy()
    ref = oracle.far_field(v, f, k, u, dirs, q=q)
    e_dir, e_ref = _rel(fast, direct), _rel(fast, ref)
    print("%s k %g q %s: fast pattern vs direct %.2e, vs oracle %.2e" % (mesh, k, with_q, e_dir, e_ref))
    assert e_dir < 1e-3 and e_ref < 1e-3


def test_fast_pattern_without_far_field_is_the_direct_sum():
    """A 20-triangle mesh is one leaf (no interaction lists): the fast pattern
    sums every element directly, equal to fda_far_field to round-off."""
    from paper_1403_4747_gb300 import FDAProblem
    v, f = icosphere(0)
    P = FDAProblem(v, f, 3.0)
    u = _dev(complex_normal(len(f), seed=43))
    dirs = fibonacci_directions(9)
    assert _rel(P.far_field(u, dirs, fast=True).cpu().numpy(), P.far_field(u, dirs).cpu().numpy()) < 1e-13


def _field_points(seed):
    """Points of every kind the fast field distinguishes: just off the
    surface (inside leaf boxes: L2T at the point's leaf), a shell in the
    empty part of the tree's cubes, inside the body, and outside the root
    cube at growing distance (the whole tree through equivalent sources)."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(96, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    radii = np.concatenate([np.full(24, 1.04), np.full(24, 1.3), np.full(16, 0.45), np.full(16, 2.5),
                            np.full(16, 9.0)])
    return d * radii[:, None], radii


@pytest.mark.parametrize("mesh,k", [("sphere4", 20.0), ("ellipsoid4", 15.0), ("sphere5", 25.0)])
@pytest.mark.parametrize("with_q", [False, True])
@pytest.mark.parametrize("precision", [0, 1])
def test_fast_field_matches_direct_and_oracle(mesh, k, with_q, precision):
    """fda_scattered_field_fast (L2T at the point's low-frequency box from
    the downward pass, equivalent sources of the boxes the point is not
    near, six-point sums of the near leaves) agrees with the direct
    six-point sums and the oracle's field, group by group of points, with
    the translations and the point arithmetic in FP64 (plain) and in the
    chosen precision (translations as in its apply: FP32 S2M, tensor-core
    M2M / M2L / L2L; point arithmetic in FP32).  Bound 1e-3 relative per
    group: the translations are truncated at eps = 1e-4 relative to each
    box's field."""
    from paper_1403_4747_gb300 import FDAProblem
    level = int(mesh[-1])
    v, f = icosphere(level) if mesh.startswith("sphere") else ellipsoid_from_icosphere(level)
    P = FDAProblem(v, f, k, precision=precision)
    st = P.stats()
    assert any(st.level_regime[l] == 1 for l in range(st.n_levels))
    u = complex_normal(len(f), seed=51)
    q = complex_normal(len(f), seed=52) if with_q else None
    pts, radii = _field_points(53)
    ud, qd = _dev(u), (_dev(q) if with_q else None)
    fast = P.scattered_field(ud, pts, qd, fast=True).cpu().numpy()
    direct = P.scattered_field(ud, pts, qd).cpu().numpy()
    ref = oracle.scattered_field(v, f, k, u, pts, q=q)
    for r in np.unique(radii):
        m = radii == r
        e_dir, e_ref = _rel(fast[m], direct[m]), _rel(fast[m], ref[m])
        print("%s k %g q %s precision %d r %.2f: fast field vs direct %.2e, vs oracle %.2e"
              % (mesh, k, with_q, precision, r, e_dir, e_ref))
        assert e_dir < 1e-3 and e_ref < 1e-3
    P.close()


def test_fast_field_of_gpu_solution_against_mie():
    from paper_1403_4747_gb300 import FDAProblem
    k = 5.0
    v, f = icosphere(5)
    P = FDAProblem(v, f, k, precision=1)
    u, info = P.solve(P.rhs_plane_wave([0.0, 0.0, 1.0]), 1e-6)
    dirs = fibonacci_directions(10)
    us = P.scattered_field(u, dirs * 2.0, fast=True).cpu().numpy()
    assert _rel(us, oracle.mie_scattered_field(k, 2.0, dirs[:, 2])) < 2e-3
    assert _rel(us, P.scattered_field(u, dirs * 2.0).cpu().numpy()) < 1e-4
    P.close()


def test_fast_field_without_far_field_is_the_direct_sum():
    """One leaf, no interaction lists: the fast field is the direct sum."""
    from paper_1403_4747_gb300 import FDAProblem
    v, f = icosphere(0)
    P = FDAProblem(v, f, 3.0)
    u = _dev(complex_normal(len(f), seed=54))
    pts, _ = _field_points(55)
    assert _rel(P.scattered_field(u, pts, fast=True).cpu().numpy(), P.scattered_field(u, pts).cpu().numpy()) < 1e-13
    P.close()
