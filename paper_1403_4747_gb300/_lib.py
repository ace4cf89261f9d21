"""ctypes binding of include/fda_bem.h: same names, argument marshalling only.

Every computation happens inside libfdabem.so (CUDA kernels).  If the
library has not been built, or no CUDA device is present, these calls fail
with an exception: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfdabem.so")

FDA_OK, FDA_ERR_ARG, FDA_ERR_STATE, FDA_ERR_CUDA, FDA_ERR_OOM = 0, 1, 2, 3, 4
FDA_ERR_NOT_CONVERGED, FDA_ERR_TIMEOUT, FDA_ERR_NUMERIC = 5, 6, 7
STATUS_NAMES = {0: "FDA_OK", 1: "FDA_ERR_ARG", 2: "FDA_ERR_STATE", 3: "FDA_ERR_CUDA", 4: "FDA_ERR_OOM",
                5: "FDA_ERR_NOT_CONVERGED", 6: "FDA_ERR_TIMEOUT", 7: "FDA_ERR_NUMERIC"}
FDA_PLAIN_FP64, FDA_CHOSEN_FP32 = 0, 1
FDA_MODE_FDA, FDA_MODE_DENSE = 0, 1


class fda_config(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("p_lf", ctypes.c_int), ("p_hf", ctypes.c_int), ("hf_nr", ctypes.c_int),
                ("hf_na", ctypes.c_int), ("leaf_max", ctypes.c_int), ("hf_wavelengths", ctypes.c_double),
                ("rho_min", ctypes.c_double), ("precision", ctypes.c_int), ("mode", ctypes.c_int),
                ("restart", ctypes.c_int), ("maxit", ctypes.c_int), ("precond", ctypes.c_int),
                ("alpha_sign", ctypes.c_double), ("max_rhs", ctypes.c_int), ("tensor_cores", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p), ("graphs", ctypes.c_int),
                ("autotune", ctypes.c_int), ("autotune_cache", ctypes.c_char_p), ("lowrank", ctypes.c_int)]


class fda_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("refinements", ctypes.c_int), ("rel_resid_fp64", ctypes.c_double),
                ("setup_s", ctypes.c_double), ("solve_s", ctypes.c_double), ("matvec_s", ctypes.c_double)]


class fda_stats(ctypes.Structure):
    _fields_ = [("n_elements", ctypes.c_int64), ("n_boxes", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("n_levels", ctypes.c_int64), ("nnz_near", ctypes.c_int64), ("n_m2l", ctypes.c_int64),
                ("n_m2l_ops", ctypes.c_int64), ("bytes_near", ctypes.c_int64), ("bytes_far", ctypes.c_int64),
                ("flops_far", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("level_regime", ctypes.c_int32 * 32), ("level_rank", ctypes.c_int32 * 32),
                ("level_boxes", ctypes.c_int32 * 32), ("level_cones", ctypes.c_int32 * 32),
                ("precompute_s", ctypes.c_double), ("tree_s", ctypes.c_double), ("near_s", ctypes.c_double),
                ("level_m2l_pairs", ctypes.c_int64 * 32),
                ("level_m2l_ops", ctypes.c_int32 * 32), ("graph_replays", ctypes.c_int64),
                ("graph_fallback", ctypes.c_int32), ("autotune_cached", ctypes.c_int32),
                ("autotune_timed", ctypes.c_int32), ("level_lr_ops", ctypes.c_int32 * 32),
                ("level_lr_rank_max", ctypes.c_int32 * 32), ("level_lr_rank_mean", ctypes.c_float * 32),
                ("level_lr_pairs", ctypes.c_int64 * 32), ("level_m2l_flops", ctypes.c_double * 32),
                ("level_m2l_bytes", ctypes.c_double * 32), ("level_lr_tc", ctypes.c_int32 * 32),
                ("level_tc_shape", (ctypes.c_int32 * 3) * 32)]


class fda_sai_config(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int), ("lr", ctypes.c_double), ("seed", ctypes.c_ulonglong),
                ("pattern", ctypes.c_int), ("sample_leaves", ctypes.c_int)]


class fda_sai_report(ctypes.Structure):
    _fields_ = [("loss_init", ctypes.c_double), ("loss_final", ctypes.c_double), ("train_s", ctypes.c_double)]


class fda_batch_stats(ctypes.Structure):
    _fields_ = [("nmesh", ctypes.c_int), ("n_total", ctypes.c_int64), ("graph_replays", ctypes.c_int64),
                ("graph_fallback", ctypes.c_int), ("device_bytes", ctypes.c_size_t)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libfdabem.so (built by build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libfdabem.so not built (run paper_1403_4747_gb300.build.build()); "
                           "there is no CPU fallback")
    lib = ctypes.CDLL(path)
    vp, i64, dbl, cint = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    H = ctypes.c_void_p
    lib.fda_default_config.argtypes = [ctypes.POINTER(fda_config)]
    lib.fda_default_config.restype = None
    lib.fda_create.argtypes = [ctypes.POINTER(fda_config), ctypes.POINTER(H)]
    lib.fda_build_tree.argtypes = [H, vp, i64, vp, i64, dbl]
    lib.fda_precompute_translations.argtypes = [H]
    lib.fda_apply.argtypes = [H, vp, vp, cint, i64]
    lib.fda_apply_host.argtypes = [H, vp, vp, cint, i64]
    lib.fda_rhs_plane_wave.argtypes = [H, vp, cint, vp]
    lib.fda_rhs_plane_wave_noalloc.argtypes = [H, vp, cint, vp]
    lib.fda_rhs_neumann.argtypes = [H, vp, vp, cint, i64]
    lib.fda_rhs_point_source.argtypes = [H, vp, cint, vp]
    lib.fda_far_field.argtypes = [H, vp, vp, vp, cint, vp]
    lib.fda_scattered_field.argtypes = [H, vp, vp, vp, i64, vp]
    lib.fda_far_field_fast.argtypes = [H, vp, vp, vp, cint, vp]
    lib.fda_scattered_field_fast.argtypes = [H, vp, vp, vp, i64, vp]
    lib.fda_solve.argtypes = [H, vp, vp, cint, dbl, ctypes.POINTER(fda_info)]
    lib.fda_get_stats.argtypes = [H, ctypes.POINTER(fda_stats)]
    lib.fda_set_timing.argtypes = [H, cint]
    lib.fda_set_precision.argtypes = [H, cint]
    lib.fda_set_precond.argtypes = [H, cint]
    lib.fda_set_tensor_cores.argtypes = [H, cint]
    lib.fda_set_tc_tiles.argtypes = [H, cint, cint, cint]
    lib.fda_tree_sizes.argtypes = [H, vp]
    lib.fda_get_tree.argtypes = [H] + [vp] * 12
    lib.fda_get_pass_times.argtypes = [H, ctypes.POINTER(ctypes.c_float)]
    lib.fda_cone_symmetry_table.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.fda_cone_symmetry_table.restype = ctypes.c_int
    lib.fda_sai_num_params.argtypes = []
    lib.fda_sai_num_params.restype = cint
    lib.fda_sai_default_config.argtypes = [ctypes.POINTER(fda_sai_config)]
    lib.fda_sai_init_weights.argtypes = [ctypes.c_ulonglong, vp]
    lib.fda_sai_train.argtypes = [vp, cint, ctypes.POINTER(fda_sai_config), vp, ctypes.POINTER(fda_sai_report)]
    lib.fda_sai_set.argtypes = [H, vp, vp]
    lib.fda_sai_loss_grad.argtypes = [i64, vp, vp, vp, dbl, cint, vp, vp, vp, vp, cint, vp, vp]
    lib.fda_sai_set_pattern.argtypes = [H, vp, cint, vp]
    lib.fda_sai_loss_grad_near.argtypes = [H, vp, cint, vp, cint, vp, vp]
    for name in ("fda_sai_default_config", "fda_sai_init_weights", "fda_sai_train", "fda_sai_set",
                 "fda_sai_loss_grad", "fda_sai_set_pattern", "fda_sai_loss_grad_near"):
        getattr(lib, name).restype = cint
    B = ctypes.c_void_p
    lib.fda_create_batch.argtypes = [ctypes.POINTER(fda_config), cint, ctypes.POINTER(B)]
    lib.fda_build_batch.argtypes = [B, vp, vp, vp, vp, vp]
    lib.fda_precompute_batch.argtypes = [B]
    lib.fda_apply_batch.argtypes = [B, vp, vp, cint, vp]
    lib.fda_batch_mesh.argtypes = [B, cint]
    lib.fda_batch_mesh.restype = H
    lib.fda_get_batch_stats.argtypes = [B, ctypes.POINTER(fda_batch_stats)]
    lib.fda_batch_last_error.argtypes = [B]
    lib.fda_batch_last_error.restype = ctypes.c_char_p
    lib.fda_destroy_batch.argtypes = [B]
    lib.fda_destroy_batch.restype = None
    for name in ("fda_create_batch", "fda_build_batch", "fda_precompute_batch", "fda_apply_batch",
                 "fda_get_batch_stats"):
        getattr(lib, name).restype = cint
    lib.fda_launch_count.argtypes = []
    lib.fda_launch_count.restype = ctypes.c_longlong
    lib.fda_last_error.argtypes = [H]
    lib.fda_last_error.restype = ctypes.c_char_p
    lib.fda_struct_size.argtypes = [cint]
    lib.fda_struct_size.restype = ctypes.c_size_t
    for which, cls in enumerate((fda_config, fda_info, fda_stats, fda_sai_config, fda_sai_report, fda_batch_stats)):
        if lib.fda_struct_size(which) != ctypes.sizeof(cls):
            raise ImportError("%s: the library's struct has %d bytes, this binding's %d"
                              % (cls.__name__, lib.fda_struct_size(which), ctypes.sizeof(cls)))
    lib.fda_destroy.argtypes = [H]
    lib.fda_destroy.restype = None
    for name in ("fda_create", "fda_build_tree", "fda_precompute_translations", "fda_apply", "fda_apply_host",
                 "fda_rhs_plane_wave", "fda_rhs_plane_wave_noalloc", "fda_rhs_neumann", "fda_rhs_point_source", "fda_far_field", "fda_far_field_fast", "fda_scattered_field", "fda_scattered_field_fast", "fda_solve", "fda_get_stats", "fda_set_timing", "fda_get_pass_times",
                 "fda_set_precision", "fda_set_precond", "fda_set_tensor_cores", "fda_set_tc_tiles",
                 "fda_tree_sizes", "fda_get_tree"):
        getattr(lib, name).restype = cint
    _lib = lib
    return lib


class FDAError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def _check(h, st):
    if st != FDA_OK:
        raise FDAError(st, load().fda_last_error(h).decode() if h else "")


def fda_default_config(**overrides) -> fda_config:
    c = fda_config()
    load().fda_default_config(ctypes.byref(c))
    for k, v in overrides.items():
        setattr(c, k, v.encode() if isinstance(v, str) else v)
    return c


def fda_create(cfg: fda_config | None = None):
    h = ctypes.c_void_p()
    st = load().fda_create(ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(h))
    if st != FDA_OK:
        raise FDAError(st, "fda_create failed")
    return h


def fda_build_tree(h, verts, tris, k):
    """verts: float64 [V,3], tris: int32 [N,3] host arrays (numpy)."""
    import numpy as np
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    _check(h, load().fda_build_tree(h, v.ctypes.data, v.shape[0], t.ctypes.data, t.shape[0], float(k)))


def fda_precompute_translations(h):
    _check(h, load().fda_precompute_translations(h))


def fda_apply(h, x_ptr, y_ptr, nrhs, ld):
    """x_ptr, y_ptr: device addresses (e.g. torch complex128 tensor.data_ptr())."""
    _check(h, load().fda_apply(h, x_ptr, y_ptr, int(nrhs), int(ld)))


def fda_apply_host(h, x_ptr, y_ptr, nrhs, ld):
    _check(h, load().fda_apply_host(h, x_ptr, y_ptr, int(nrhs), int(ld)))


def fda_rhs_plane_wave(h, dirs, b_ptr):
    import numpy as np
    d = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
    _check(h, load().fda_rhs_plane_wave(h, d.ctypes.data, d.shape[0], b_ptr))


def fda_rhs_point_source(h, sources, b_ptr):
    """sources: host [nrhs, 3] positions; b_ptr: device address (ld = nt)."""
    import numpy as np
    s = np.ascontiguousarray(np.atleast_2d(sources), dtype=np.float64)
    _check(h, load().fda_rhs_point_source(h, s.ctypes.data, s.shape[0], b_ptr))


def fda_far_field(h, u_ptr, q_ptr, dirs, F_ptr):
    """Far-field pattern at host unit directions [M, 3] into device F (q_ptr 0 / None = sound-hard)."""
    import numpy as np
    d = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
    _check(h, load().fda_far_field(h, u_ptr, q_ptr or None, d.ctypes.data, d.shape[0], F_ptr))


def fda_far_field_fast(h, u_ptr, q_ptr, dirs, F_ptr):
    """Far-field pattern through the fast algorithm's upward pass (same arguments as fda_far_field)."""
    import numpy as np
    d = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
    _check(h, load().fda_far_field_fast(h, u_ptr, q_ptr or None, d.ctypes.data, d.shape[0], F_ptr))


def fda_scattered_field(h, u_ptr, q_ptr, points, out_ptr):
    """Scattered field at host points [M, 3] into device out (q_ptr 0 / None = sound-hard)."""
    import numpy as np
    p = np.ascontiguousarray(np.atleast_2d(points), dtype=np.float64)
    _check(h, load().fda_scattered_field(h, u_ptr, q_ptr or None, p.ctypes.data, p.shape[0], out_ptr))


def fda_scattered_field_fast(h, u_ptr, q_ptr, points, out_ptr):
    """Scattered field at host points [M, 3] through the fast algorithm (same arguments as fda_scattered_field)."""
    import numpy as np
    p = np.ascontiguousarray(np.atleast_2d(points), dtype=np.float64)
    _check(h, load().fda_scattered_field_fast(h, u_ptr, q_ptr or None, p.ctypes.data, p.shape[0], out_ptr))


def fda_rhs_neumann(h, q_ptr, b_ptr, nrhs, ld):
    """b = right-hand side of the Burton-Miller equation for Neumann data q (device addresses)."""
    _check(h, load().fda_rhs_neumann(h, q_ptr, b_ptr, int(nrhs), int(ld)))


def fda_rhs_plane_wave_noalloc(h, dirs, b_ptr):
    """Allocation-free right-hand side (at most 256 directions per call)."""
    import numpy as np
    d = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
    _check(h, load().fda_rhs_plane_wave_noalloc(h, d.ctypes.data, d.shape[0], b_ptr))


def fda_solve(h, b_ptr, x_ptr, nrhs, tol, raise_on_not_converged=True):
    info = fda_info()
    st = load().fda_solve(h, b_ptr, x_ptr, int(nrhs), float(tol), ctypes.byref(info))
    if st != FDA_OK and (raise_on_not_converged or st != FDA_ERR_NOT_CONVERGED):
        _check(h, st)
    return info, st


def fda_get_stats(h) -> fda_stats:
    s = fda_stats()
    _check(h, load().fda_get_stats(h, ctypes.byref(s)))
    return s


def fda_set_precision(h, precision):
    _check(h, load().fda_set_precision(h, int(precision)))


def fda_set_precond(h, precond):
    _check(h, load().fda_set_precond(h, int(precond)))


def fda_set_tensor_cores(h, on):
    _check(h, load().fda_set_tensor_cores(h, 1 if on else 0))


def fda_get_tree(h):
    """Host copies of the device octree and lists (dict of numpy arrays)."""
    import numpy as np
    sz = np.zeros(4, dtype=np.int64)
    _check(h, load().fda_tree_sizes(h, sz.ctypes.data))
    nb, nl, nil, ncol = (int(v) for v in sz)
    st = fda_get_stats(h)
    n = int(st.n_elements)
    out = {"box_level": np.zeros(nb, np.int32), "box_coord": np.zeros((nb, 3), np.int32),
           "box_leaf": np.zeros(nb, np.int32), "box_parent": np.zeros(nb, np.int32),
           "box_begin": np.zeros(nb, np.int32), "box_end": np.zeros(nb, np.int32), "perm": np.zeros(n, np.int32),
           "il_ptr": np.zeros(nb + 1, np.int64), "il_src": np.zeros(max(nil, 1), np.int32),
           "leaf_box": np.zeros(nl, np.int32), "nf_colptr": np.zeros(nl + 1, np.int64),
           "nf_cols": np.zeros(max(ncol, 1), np.int32)}
    order = ["box_level", "box_coord", "box_leaf", "box_parent", "box_begin", "box_end", "perm", "il_ptr", "il_src",
             "leaf_box", "nf_colptr", "nf_cols"]
    _check(h, load().fda_get_tree(h, *[out[k].ctypes.data for k in order]))
    out["il_src"] = out["il_src"][:nil]
    out["nf_cols"] = out["nf_cols"][:ncol]
    return out


def fda_set_tc_tiles(h, columns=0, row_tiles=0, stages=0):
    _check(h, load().fda_set_tc_tiles(h, int(columns), int(row_tiles), int(stages)))


def fda_set_timing(h, enable=True):
    _check(h, load().fda_set_timing(h, 1 if enable else 0))


def fda_get_pass_times(h):
    arr = (ctypes.c_float * 6)()
    _check(h, load().fda_get_pass_times(h, arr))
    return list(arr)


def fda_cone_symmetry_table(nc: int):
    """(rep, g) of the cone partition with nc x nc cells per face: rep[u] is
    cone u's representative and g[u] the 3x3 signed permutation mapping it to u."""
    import numpy as np
    n = 6 * nc * nc
    rep = np.zeros(n, dtype=np.int32)
    g = np.zeros((n, 3, 3), dtype=np.int32)
    _check(None, load().fda_cone_symmetry_table(nc, rep.ctypes.data, g.ctypes.data))
    return rep, g


def fda_sai_num_params() -> int:
    return int(load().fda_sai_num_params())


def fda_sai_default_config(**overrides) -> fda_sai_config:
    c = fda_sai_config()
    _check(None, load().fda_sai_default_config(ctypes.byref(c)))
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


def fda_sai_init_weights(seed: int):
    """Initial network weights (float32 numpy array)."""
    import numpy as np
    w = np.zeros(fda_sai_num_params(), dtype=np.float32)
    _check(None, load().fda_sai_init_weights(seed, w.ctypes.data))
    return w


def fda_sai_train(handles, cfg: fda_sai_config, weights):
    """Train in place on the leaf blocks of the given handles; returns the report."""
    import numpy as np
    assert weights.dtype == np.float32 and weights.flags.c_contiguous
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    rep = fda_sai_report()
    _check(handles[0], load().fda_sai_train(ctypes.cast(arr, ctypes.c_void_p), len(handles), ctypes.byref(cfg),
                                            weights.ctypes.data, ctypes.byref(rep)))
    return rep


def fda_sai_set(h, weights) -> float:
    """Evaluate the network on h's leaf blocks as its learned preconditioner; returns the loss."""
    import numpy as np
    assert weights.dtype == np.float32 and weights.flags.c_contiguous
    loss = ctypes.c_double()
    _check(h, load().fda_sai_set(h, weights.ctypes.data, ctypes.byref(loss)))
    return loss.value


def fda_sai_set_pattern(h, weights, pattern, want_loss=True):
    """Evaluate the network on h's leaf blocks (pattern 0) or its whole
    near-field pattern (pattern 1) as its learned preconditioner; returns the
    loss (None without want_loss)."""
    import numpy as np
    assert weights.dtype == np.float32 and weights.flags.c_contiguous
    loss = ctypes.c_double()
    _check(h, load().fda_sai_set_pattern(h, weights.ctypes.data, int(pattern),
                                         ctypes.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def fda_sai_loss_grad_near(h, weights, leaves, precision=FDA_PLAIN_FP64):
    """Loss and gradient of the near-field objective over the given leaves of h."""
    import numpy as np
    W = np.ascontiguousarray(weights, dtype=np.float64)
    lv = np.ascontiguousarray(leaves, dtype=np.int32)
    loss = ctypes.c_double()
    grad = np.zeros(fda_sai_num_params(), dtype=np.float64)
    _check(h, load().fda_sai_loss_grad_near(h, W.ctypes.data, len(lv), lv.ctypes.data, precision,
                                            ctypes.byref(loss), grad.ctypes.data))
    return loss.value, grad


def fda_sai_loss_grad(cent, nrm, area, k, block_ptr, block_elems, blocks, weights, precision=FDA_PLAIN_FP64):
    """Loss and gradient of the training kernels for caller-supplied blocks (host numpy arrays)."""
    import numpy as np
    cent = np.ascontiguousarray(cent, dtype=np.float64)
    nrm = np.ascontiguousarray(nrm, dtype=np.float64)
    area = np.ascontiguousarray(area, dtype=np.float64)
    bp = np.ascontiguousarray(block_ptr, dtype=np.int64)
    be = np.ascontiguousarray(block_elems, dtype=np.int32)
    A = np.ascontiguousarray(blocks, dtype=np.complex128)
    W = np.ascontiguousarray(weights, dtype=np.float64)
    loss = ctypes.c_double()
    grad = np.zeros(fda_sai_num_params(), dtype=np.float64)
    _check(None, load().fda_sai_loss_grad(len(area), cent.ctypes.data, nrm.ctypes.data, area.ctypes.data, float(k),
                                          len(bp) - 1, bp.ctypes.data, be.ctypes.data, A.ctypes.data, W.ctypes.data,
                                          precision, ctypes.byref(loss), grad.ctypes.data))
    return loss.value, grad


def _bcheck(b, st):
    if st != FDA_OK:
        raise FDAError(st, load().fda_batch_last_error(b).decode() if b else "")


def fda_create_batch(cfg: fda_config | None, nmesh: int):
    b = ctypes.c_void_p()
    st = load().fda_create_batch(ctypes.byref(cfg) if cfg is not None else None, int(nmesh), ctypes.byref(b))
    if st != FDA_OK:
        raise FDAError(st, "fda_create_batch failed")
    return b


def fda_build_batch(b, meshes, ks):
    """meshes: list of (verts float64 [V,3], tris int32 [N,3]) host arrays; ks: wavenumbers."""
    import numpy as np
    vs = [np.ascontiguousarray(v, dtype=np.float64) for v, _ in meshes]
    ts = [np.ascontiguousarray(t, dtype=np.int32) for _, t in meshes]
    n = len(meshes)
    vp = (ctypes.c_void_p * n)(*[v.ctypes.data for v in vs])
    tp = (ctypes.c_void_p * n)(*[t.ctypes.data for t in ts])
    nv = np.array([v.shape[0] for v in vs], dtype=np.int64)
    nt = np.array([t.shape[0] for t in ts], dtype=np.int64)
    k = np.ascontiguousarray(ks, dtype=np.float64)
    _bcheck(b, load().fda_build_batch(b, ctypes.cast(vp, ctypes.c_void_p), nv.ctypes.data,
                                      ctypes.cast(tp, ctypes.c_void_p), nt.ctypes.data, k.ctypes.data))


def fda_precompute_batch(b):
    _bcheck(b, load().fda_precompute_batch(b))


def fda_apply_batch(b, x_ptrs, y_ptrs, nrhs, lds):
    """x_ptrs, y_ptrs: per-mesh device addresses; lds: per-mesh leading dimensions."""
    import numpy as np
    n = len(x_ptrs)
    xp = (ctypes.c_void_p * n)(*x_ptrs)
    yp = (ctypes.c_void_p * n)(*y_ptrs)
    ld = np.ascontiguousarray(lds, dtype=np.int64)
    _bcheck(b, load().fda_apply_batch(b, ctypes.cast(xp, ctypes.c_void_p), ctypes.cast(yp, ctypes.c_void_p),
                                      int(nrhs), ld.ctypes.data))


def fda_batch_mesh(b, i: int):
    """The handle of mesh i (owned by the batch)."""
    h = load().fda_batch_mesh(b, int(i))
    if not h:
        raise FDAError(FDA_ERR_ARG, "no mesh %d in the batch" % i)
    return ctypes.c_void_p(h)


def fda_get_batch_stats(b) -> fda_batch_stats:
    s = fda_batch_stats()
    _bcheck(b, load().fda_get_batch_stats(b, ctypes.byref(s)))
    return s


def fda_batch_last_error(b) -> str:
    return load().fda_batch_last_error(b).decode()


def fda_destroy_batch(b):
    if b:
        load().fda_destroy_batch(b)


def fda_launch_count() -> int:
    """Kernels launched by the library since it was loaded (all handles)."""
    return int(load().fda_launch_count())


def fda_last_error(h) -> str:
    return load().fda_last_error(h).decode()


def fda_destroy(h):
    if h:
        load().fda_destroy(h)
