"""Thin object wrapper over the C ABI: holds a handle and marshals torch
CUDA tensors (complex128) to device pointers.  No arithmetic here."""
from __future__ import annotations

from . import _lib


class FDAProblem:
    def __init__(self, verts, tris, k, stream=None, **cfg):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("FDAProblem needs a CUDA device; there is no CPU path")
        c = _lib.fda_default_config(**cfg)
        if stream is not None:
            c.cuda_stream = stream.cuda_stream
        self.h = _lib.fda_create(c)
        self.k = float(k)
        self.n = int(len(tris))
        _lib.fda_build_tree(self.h, verts, tris, k)
        _lib.fda_precompute_translations(self.h)

    def _c(self, t):
        import torch
        if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous():
            raise TypeError("expected a contiguous complex128 CUDA tensor")
        return t.data_ptr()

    def apply(self, x, y=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        _lib.fda_apply(self.h, self._c(x), self._c(y), nrhs, self.n)
        return y

    def rhs_plane_wave(self, dirs):
        import numpy as np
        import torch
        d = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
        b = torch.empty((d.shape[0], self.n), dtype=torch.complex128, device="cuda")
        _lib.fda_rhs_plane_wave(self.h, d, self._c(b))
        return b[0] if np.ndim(dirs) == 1 else b

    def rhs_point_source(self, sources):
        """Right-hand side for point sources u_inc = G(x, x_s) (host positions [nrhs, 3] or [3])."""
        import numpy as np
        import torch
        src = np.atleast_2d(np.asarray(sources, dtype=np.float64))
        b = torch.empty((src.shape[0], self.n), dtype=torch.complex128, device="cuda")
        _lib.fda_rhs_point_source(self.h, src, b.data_ptr())
        return b[0] if np.ndim(sources) == 1 else b

    def far_field(self, u, dirs, q=None, fast=False):
        """Far-field pattern of the scattered field at unit directions (host
        [M, 3]); fast=True through the fast algorithm's upward pass."""
        import numpy as np
        import torch
        d = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
        F = torch.empty(d.shape[0], dtype=torch.complex128, device="cuda")
        fn = _lib.fda_far_field_fast if fast else _lib.fda_far_field
        fn(self.h, self._c(u), self._c(q) if q is not None else None, d, F.data_ptr())
        return F

    def scattered_field(self, u, points, q=None, fast=False):
        """Scattered field at host points [M, 3] off the surface; fast=True
        through the fast algorithm (L2T at each point's box, equivalent
        sources and direct sums for the rest)."""
        import numpy as np
        import torch
        p = np.atleast_2d(np.asarray(points, dtype=np.float64))
        out = torch.empty(p.shape[0], dtype=torch.complex128, device="cuda")
        fn = _lib.fda_scattered_field_fast if fast else _lib.fda_scattered_field
        fn(self.h, self._c(u), self._c(q) if q is not None else None, p, out.data_ptr())
        return out

    def rhs_neumann(self, q, b=None):
        """Right-hand side of the Burton-Miller equation for Neumann data q = du/dn."""
        import torch
        if b is None:
            b = torch.empty_like(q)
        nrhs = 1 if q.dim() == 1 else q.shape[0]
        _lib.fda_rhs_neumann(self.h, self._c(q), self._c(b), nrhs, self.n)
        return b

    def solve(self, b, tol, x0=None, raise_on_not_converged=True):
        import torch
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        nrhs = 1 if b.dim() == 1 else b.shape[0]
        info, st = _lib.fda_solve(self.h, self._c(b), self._c(x), nrhs, tol, raise_on_not_converged)
        return x, info

    def stats(self):
        return _lib.fda_get_stats(self.h)

    def close(self):
        if self.h:
            _lib.fda_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FDABatch:
    """Several meshes behind one operator application (one CUDA graph per
    call, one branch per mesh).  meshes: list of (verts, tris); ks: one
    wavenumber per mesh."""

    def __init__(self, meshes, ks, stream=None, **cfg):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("FDABatch needs a CUDA device; there is no CPU path")
        c = _lib.fda_default_config(**cfg)
        if stream is not None:
            c.cuda_stream = stream.cuda_stream
        self.b = _lib.fda_create_batch(c, len(meshes))
        self.ns = [int(len(t)) for _, t in meshes]
        self.ks = [float(k) for k in ks]
        _lib.fda_build_batch(self.b, meshes, self.ks)
        _lib.fda_precompute_batch(self.b)

    def apply(self, xs, ys=None):
        """xs: per mesh a complex128 CUDA tensor [nrhs, n_i] (or [n_i]); same nrhs for all."""
        import torch
        if ys is None:
            ys = [torch.empty_like(x) for x in xs]
        for t in list(xs) + list(ys):
            if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous():
                raise TypeError("expected contiguous complex128 CUDA tensors")
        nrhs = 1 if xs[0].dim() == 1 else xs[0].shape[0]
        _lib.fda_apply_batch(self.b, [x.data_ptr() for x in xs], [y.data_ptr() for y in ys], nrhs, self.ns)
        return ys

    def mesh(self, i):
        """The handle of mesh i (owned by the batch)."""
        return _lib.fda_batch_mesh(self.b, i)

    def stats(self):
        return _lib.fda_get_batch_stats(self.b)

    def close(self):
        if self.b:
            _lib.fda_destroy_batch(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
