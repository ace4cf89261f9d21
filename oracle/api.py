"""ctypes wrappers around the C oracle (oracle/bem_oracle.c).  Test
infrastructure only."""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_lp = ctypes.POINTER(ctypes.c_int64)


def load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i64, dbl, cint = ctypes.c_int64, ctypes.c_double, ctypes.c_int
        lib.orc_geometry.argtypes = [_dp, _ip, i64, _dp, _dp, _dp, _dp]
        lib.orc_kernels.argtypes = [_dp, _dp, _dp, _dp, dbl, _dp]
        lib.orc_integrate_triangle.argtypes = [_dp, _dp, _dp, _dp, dbl, dbl, cint, _dp]
        lib.orc_self_hypersingular.argtypes = [_dp, _ip, i64, dbl, _dp]
        lib.orc_entry.argtypes = [_dp, _ip, i64, dbl, i64, i64, _dp]
        lib.orc_is_near_pair.argtypes = [_dp, _ip, i64, i64]
        lib.orc_is_near_pair.restype = cint
        lib.orc_matvec.argtypes = [_dp, _ip, i64, dbl, _dp, cint, _lp, i64, _dp, cint]
        lib.orc_assemble.argtypes = [_dp, _ip, i64, dbl, _dp, cint]
        lib.orc_rhs_plane_wave.argtypes = [_dp, _ip, i64, dbl, _dp, cint, _dp]
        lib.orc_gauss_legendre.argtypes = [cint, _dp, _dp]
        lib.orc_num_threads.restype = cint
        lib.orc_rule6.argtypes = [_dp, _dp]
        lib.orc_set_alpha_sign.argtypes = [dbl]
        lib.orc_layer_rowsum.argtypes = [_dp, _ip, i64, dbl, cint, _dp, cint]
        lib.orc_set_side.argtypes = [cint]
        lib.orc_rhs_point_source.argtypes = [_dp, _ip, i64, dbl, _dp, cint, _dp]
        lib.orc_scattered_field.argtypes = [_dp, _ip, i64, dbl, _dp, _dp, _dp, i64, _dp, cint]
        lib.orc_far_field.argtypes = [_dp, _ip, i64, dbl, _dp, _dp, _dp, i64, _dp, cint]
        lib.orc_self_single.argtypes = [_dp, _ip, i64, dbl, _dp]
        _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _mesh(verts, tris):
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    return v, t


def num_threads() -> int:
    return int(load().orc_num_threads())


def geometry(verts, tris):
    """centroids [N,3], normals n (into the body) [N,3], areas [N], h^2 [N]"""
    v, t = _mesh(verts, tris)
    n = t.shape[0]
    c = np.empty((n, 3)); nr = np.empty((n, 3)); a = np.empty(n); h2 = np.empty(n)
    load().orc_geometry(_d(v), t.ctypes.data_as(_ip), n, _d(c), _d(nr), _d(a), _d(h2))
    return c, nr, a, h2


def kernels(x, nx, y, ny, k):
    """(G, dG/dn_y, dG/dn_x, d2G/dn_x dn_y) at one point pair."""
    arrs = [np.ascontiguousarray(q, dtype=np.float64) for q in (x, nx, y, ny)]
    out = np.empty(8)
    load().orc_kernels(*[_d(q) for q in arrs], float(k), _d(out))
    return out[0::2] + 1j * out[1::2]


def integrate_triangle(x, nx, tri_pts, ny, area, k, levels):
    load().orc_set_alpha_sign(1.0)
    arrs = [np.ascontiguousarray(q, dtype=np.float64) for q in (x, nx, tri_pts, ny)]
    out = np.empty(2)
    load().orc_integrate_triangle(*[_d(q) for q in arrs], float(area), float(k), int(levels), _d(out))
    return complex(out[0], out[1])


def self_hypersingular(verts, tris, t, k):
    v, tt = _mesh(verts, tris)
    out = np.empty(2)
    load().orc_self_hypersingular(_d(v), tt.ctypes.data_as(_ip), int(t), float(k), _d(out))
    return complex(out[0], out[1])


def gauss_legendre(n):
    xs = np.empty(n); ws = np.empty(n)
    load().orc_gauss_legendre(int(n), _d(xs), _d(ws))
    return xs, ws


def entry(verts, tris, k, i, j, alpha_sign=-1.0):
    v, t = _mesh(verts, tris)
    load().orc_set_alpha_sign(float(alpha_sign))
    out = np.empty(2)
    load().orc_entry(_d(v), t.ctypes.data_as(_ip), t.shape[0], float(k), int(i), int(j), _d(out))
    return complex(out[0], out[1])


def is_near_pair(verts, tris, i, j) -> bool:
    v, t = _mesh(verts, tris)
    return bool(load().orc_is_near_pair(_d(v), t.ctypes.data_as(_ip), int(i), int(j)))


def matvec(verts, tris, k, x, rows=None, nthreads=0, alpha_sign=-1.0):
    """y = A x (all rows, or the listed rows).  x: complex [N] or [nrhs, N];
    returns complex [len(rows)] or [nrhs, len(rows)].  alpha = alpha_sign i/k."""
    v, t = _mesh(verts, tris)
    load().orc_set_alpha_sign(float(alpha_sign))
    n = t.shape[0]
    x = np.asarray(x, dtype=np.complex128)
    squeeze = x.ndim == 1
    xs = np.ascontiguousarray(x.reshape(-1, n))
    nrhs = xs.shape[0]
    if rows is None:
        nr, rp = n, None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        nr, rp = rows.shape[0], rows.ctypes.data_as(_lp)
    y = np.empty((nrhs, nr), dtype=np.complex128)
    load().orc_matvec(_d(v), t.ctypes.data_as(_ip), n, float(k), xs.ctypes.data_as(_dp), nrhs,
                      rp, nr, y.ctypes.data_as(_dp), int(nthreads))
    return y[0] if squeeze else y


def assemble(verts, tris, k, nthreads=0, alpha_sign=-1.0):
    v, t = _mesh(verts, tris)
    load().orc_set_alpha_sign(float(alpha_sign))
    n = t.shape[0]
    a = np.empty((n, n), dtype=np.complex128)
    load().orc_assemble(_d(v), t.ctypes.data_as(_ip), n, float(k), a.ctypes.data_as(_dp), int(nthreads))
    return a


def rhs_plane_wave(verts, tris, k, dirs, alpha_sign=-1.0):
    """b = u_inc + alpha du_inc/dn at centroids; dirs [nrhs, 3] -> [nrhs, N]"""
    v, t = _mesh(verts, tris)
    load().orc_set_alpha_sign(float(alpha_sign))
    d = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
    n = t.shape[0]
    b = np.empty((d.shape[0], n), dtype=np.complex128)
    load().orc_rhs_plane_wave(_d(v), t.ctypes.data_as(_ip), n, float(k), _d(d), d.shape[0],
                              b.ctypes.data_as(_dp))
    return b


def rule6():
    """The regular six-point rule on the reference triangle: (pts [6,2], w [6])."""
    pts = np.empty((6, 2)); w = np.empty(6)
    load().orc_rule6(_d(pts), _d(w))
    return pts, w


def layer_rowsum(verts, tris, k, part, nthreads=0):
    """part 1: 1/2 + sum_j D_ij (double layer); part 2: sum_j H_ij
    (hypersingular, no alpha).  Complex [N]."""
    v, t = _mesh(verts, tris)
    load().orc_set_alpha_sign(1.0)
    n = t.shape[0]
    out = np.empty(2 * n)
    load().orc_layer_rowsum(_d(v), t.ctypes.data_as(_ip), n, float(k), int(part), _d(out), int(nthreads))
    return out[0::2] + 1j * out[1::2]


# ---- right-hand side's layers of Eq. eq_bm acting on Neumann data q = du/dn
def _with_side(fn):
    load().orc_set_side(1)
    try:
        return fn()
    finally:
        load().orc_set_side(0)


def rhs_layers_matvec(verts, tris, k, q, rows=None, nthreads=0, alpha_sign=-1.0):
    """b = B q: b_i = -alpha q_i / 2 + sum_j int_{tri_j} [G + alpha dG/dn_x](x_i, y) dy q_j
    (all rows or the listed rows; q complex [N] or [nrhs, N])."""
    return _with_side(lambda: matvec(verts, tris, k, q, rows=rows, nthreads=nthreads, alpha_sign=alpha_sign))


def rhs_layers_assemble(verts, tris, k, nthreads=0, alpha_sign=-1.0):
    """Dense B (row-major [N, N], small meshes only)."""
    return _with_side(lambda: assemble(verts, tris, k, nthreads=nthreads, alpha_sign=alpha_sign))


def rhs_layers_entry(verts, tris, k, i, j, alpha_sign=-1.0):
    load().orc_set_alpha_sign(float(alpha_sign))
    return _with_side(lambda: entry(verts, tris, k, i, j, alpha_sign=alpha_sign))


def self_single_layer(verts, tris, t, k):
    """int over triangle t of G(x_t, y) dy, x_t its centroid."""
    v, tr = _mesh(verts, tris)
    out = np.empty(2)
    load().orc_self_single(_d(v), tr.ctypes.data_as(_ip), int(t), float(k), _d(out))
    return out[0] + 1j * out[1]


def rhs_point_source(verts, tris, k, sources, alpha_sign=-1.0):
    """b = u_inc + alpha du_inc/dn at centroids for u_inc = G(x, x_s);
    sources [nrhs, 3] -> [nrhs, N]"""
    v, t = _mesh(verts, tris)
    load().orc_set_alpha_sign(float(alpha_sign))
    src = np.ascontiguousarray(np.atleast_2d(sources), dtype=np.float64)
    n = t.shape[0]
    b = np.empty((src.shape[0], n), dtype=np.complex128)
    load().orc_rhs_point_source(_d(v), t.ctypes.data_as(_ip), n, float(k), _d(src), src.shape[0],
                                b.ctypes.data_as(_dp))
    return b


def _surface_data(u, q, n):
    uc = np.ascontiguousarray(u, dtype=np.complex128).reshape(n)
    qc = None if q is None else np.ascontiguousarray(q, dtype=np.complex128).reshape(n)
    return uc, qc


def scattered_field(verts, tris, k, u, points, q=None, nthreads=0):
    """u_sc(x) = int G q - int dG/dn_y u at points [M, 3] off the surface (q None = 0)."""
    v, t = _mesh(verts, tris)
    n = t.shape[0]
    uc, qc = _surface_data(u, q, n)
    p = np.ascontiguousarray(np.atleast_2d(points), dtype=np.float64)
    out = np.empty(p.shape[0], dtype=np.complex128)
    load().orc_scattered_field(_d(v), t.ctypes.data_as(_ip), n, float(k), uc.ctypes.data_as(_dp),
                               qc.ctypes.data_as(_dp) if qc is not None else None, _d(p), p.shape[0],
                               out.ctypes.data_as(_dp), int(nthreads))
    return out


def far_field(verts, tris, k, u, dirs, q=None, nthreads=0):
    """Far-field pattern F(xh) for unit directions [M, 3] (q None = 0)."""
    v, t = _mesh(verts, tris)
    n = t.shape[0]
    uc, qc = _surface_data(u, q, n)
    d = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
    out = np.empty(d.shape[0], dtype=np.complex128)
    load().orc_far_field(_d(v), t.ctypes.data_as(_ip), n, float(k), uc.ctypes.data_as(_dp),
                         qc.ctypes.data_as(_dp) if qc is not None else None, _d(d), d.shape[0],
                         out.ctypes.data_as(_dp), int(nthreads))
    return out
