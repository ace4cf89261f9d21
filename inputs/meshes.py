"""Synthetic surface meshes and right-hand-side data.

Conventions (shared by every consumer):
  * vertices: float64 array [V, 3];
  * triangles: int32 array [N, 3], oriented so that (v1 - v0) x (v2 - v0)
    points out of the body, into the acoustic domain;
  * complex vectors: complex128 arrays.
"""
from __future__ import annotations

import functools
import itertools

import numpy as np

_PHI = (1.0 + 5.0 ** 0.5) / 2.0


def _icosahedron():
    """Regular icosahedron: vertices (0, +-1, +-phi) and cyclic permutations,
    projected onto the unit sphere; faces found as mutually adjacent vertex
    triples and oriented outward."""
    base = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            base.append((0.0, s1, s2 * _PHI))
    verts = []
    for (a, b, c) in base:
        verts.append((a, b, c))
        verts.append((b, c, a))
        verts.append((c, a, b))
    v = np.array(verts, dtype=np.float64)
    # adjacent vertices are at distance 2 before normalisation
    d = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=-1)
    adj = np.abs(d - 2.0) < 1e-9
    faces = []
    for i, j, k in itertools.combinations(range(12), 3):
        if adj[i, j] and adj[j, k] and adj[i, k]:
            n = np.cross(v[j] - v[i], v[k] - v[i])
            if np.dot(n, v[i] + v[j] + v[k]) < 0:
                faces.append((i, k, j))
            else:
                faces.append((i, j, k))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array(sorted(faces), dtype=np.int64)
    assert f.shape == (20, 3)
    return v, f


def _subdivide(v, f, levels):
    """`levels` rounds of midpoint subdivision (each triangle into four) with
    the new vertices projected onto the unit sphere; orientation kept."""
    for _ in range(levels):
        nv = v.shape[0]
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
        e.sort(axis=1)
        key = e[:, 0] * (1 << 32) + e[:, 1]
        uniq, inv = np.unique(key, return_inverse=True)
        a = (uniq >> 32).astype(np.int64)
        b = (uniq & 0xFFFFFFFF).astype(np.int64)
        mid = v[a] + v[b]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        v = np.concatenate([v, mid], axis=0)
        nt = f.shape[0]
        m01 = nv + inv[:nt]
        m12 = nv + inv[nt:2 * nt]
        m20 = nv + inv[2 * nt:]
        f = np.concatenate([
            np.stack([f[:, 0], m01, m20], axis=1),
            np.stack([m01, f[:, 1], m12], axis=1),
            np.stack([m20, m12, f[:, 2]], axis=1),
            np.stack([m01, m12, m20], axis=1),
        ], axis=0)
    return v, f.astype(np.int32)


@functools.lru_cache(maxsize=8)
def _icosphere_cached(level: int):
    v, f = _icosahedron()
    return _subdivide(v, f, level)


def _octahedron():
    """Regular octahedron (+-e_x, +-e_y, +-e_z), faces oriented outward."""
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=np.float64)
    faces = []
    for i in (0, 1):
        for j in (2, 3):
            for k in (4, 5):
                n = np.cross(v[j] - v[i], v[k] - v[i])
                faces.append((i, j, k) if np.dot(n, v[i] + v[j] + v[k]) > 0 else (i, k, j))
    return v, np.array(faces, dtype=np.int64)


@functools.lru_cache(maxsize=8)
def _octasphere_cached(level: int):
    v, f = _octahedron()
    return _subdivide(v, f, level)


def octasphere(level: int):
    """Unit sphere from the octahedron after `level` rounds of midpoint
    subdivision with re-projection: 8 * 4**level flat triangles (level 3:
    512, the coarsest sphere of the paper's pulsating-sphere family
    N = 512 * 4**m)."""
    v, f = _octasphere_cached(int(level))
    return v.copy(), f.copy()


def icosphere(level: int):
    """Unit icosphere after `level` rounds of midpoint subdivision with
    re-projection: 20 * 4**level flat triangles, 10 * 4**level + 2 vertices."""
    v, f = _icosphere_cached(int(level))
    return v.copy(), f.copy()


def ellipsoid_from_icosphere(level: int, axes=(1.0, 0.6, 0.3)):
    """Icosphere mapped by (x, y, z) -> (a x, b y, c z); orientation kept."""
    v, f = icosphere(level)
    return v * np.asarray(axes, dtype=np.float64)[None, :], f


def fibonacci_directions(m: int):
    """m unit vectors of the Fibonacci lattice on S^2:
    z_j = 1 - (2j + 1)/m, azimuth j * pi * (3 - sqrt 5)."""
    j = np.arange(m, dtype=np.float64)
    z = 1.0 - (2.0 * j + 1.0) / m
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = j * np.pi * (3.0 - 5.0 ** 0.5)
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def complex_normal(n: int, seed: int, nrhs: int | None = None):
    """Seeded complex standard normal vector(s) (Philox bit generator);
    shape [n] or, with nrhs, column-major-friendly [nrhs, n]."""
    rng = np.random.Generator(np.random.Philox(seed))
    shape = (n,) if nrhs is None else (nrhs, n)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def icosahedral_rotations():
    """The 60 proper rotations mapping the icosahedron of `_icosahedron` onto
    itself, as 3x3 matrices (found by matching vertex triples)."""
    v, f = _icosahedron()
    mats = []
    src = v[list(f[0])]
    a = np.linalg.inv(src)
    for tri in f:
        for perm in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
            dst = v[[tri[p] for p in perm]]
            r = (a @ dst).T
            if abs(np.linalg.det(r) - 1.0) < 1e-9 and np.allclose(r @ r.T, np.eye(3), atol=1e-9):
                mats.append(r)
    out = []
    for r in mats:
        if not any(np.allclose(r, q, atol=1e-9) for q in out):
            out.append(r)
    assert len(out) == 60
    return out


def multi_mesh_set():
    """Eight meshes for the many-mesh batch: (verts, tris, k) for sphere and
    ellipsoid icospheres of levels 5-7 (20,480-327,680 triangles), kD 20-100,
    at least 10 elements per wavelength."""
    spec = [("s", 5, 10.0), ("e", 5, 15.0), ("s", 6, 25.0), ("e", 6, 30.0),
            ("s", 6, 33.0), ("e", 7, 45.0), ("s", 7, 50.0), ("e", 7, 50.0)]
    out = []
    for kind, level, k in spec:
        v, f = icosphere(level) if kind == "s" else ellipsoid_from_icosphere(level)
        out.append((v, f, k))
    return out


def mesh_for_config(name: str):
    """Named synthetic workloads: returns (verts, tris, k, direction).

    sphere_l4_k5   : icosphere level 4 (5,120 triangles), k = 5
    sphere_l7_k50  : icosphere level 7 (327,680 triangles), k = 50
    ellipsoid_l7_k50: level-7 icosphere mapped to semi-axes (1, 0.6, 0.3), k = 50
    sphere_l9_k200 : icosphere level 9 (5,242,880 triangles), k = 200
    """
    d = np.array([0.0, 0.0, 1.0])
    table = {
        "sphere_l4_k5": (lambda: icosphere(4), 5.0),
        "sphere_l5_k25": (lambda: icosphere(5), 25.0),
        "sphere_l6_k25": (lambda: icosphere(6), 25.0),
        "sphere_l7_k50": (lambda: icosphere(7), 50.0),
        "ellipsoid_l7_k50": (lambda: ellipsoid_from_icosphere(7), 50.0),
        "sphere_l9_k200": (lambda: icosphere(9), 200.0),
    }
    gen, k = table[name]
    v, f = gen()
    return v, f, k, d
