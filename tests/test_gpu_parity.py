"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: the dense mode evaluates exactly the oracle's operator in FP64
(only the summation order differs): relative L2 error <= 1e-12.  The FDA
matvec approximates it; the bar is a relative L2 error <= 1e-4 (plain FP64
and chosen FP32 forms alike).  Solutions: GMRES to tol against dense LU.
"""
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


def _problem(v, f, k, **cfg):
    from paper_1403_4747_gb300 import FDAProblem
    return FDAProblem(v, f, k, **cfg)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


def test_rhs_matches_oracle():
    v, f = icosphere(3)
    P = _problem(v, f, 5.0, mode=1)
    d = fibonacci_directions(3)
    b = P.rhs_plane_wave(d).cpu().numpy()
    ref = oracle.rhs_plane_wave(v, f, 5.0, d)
    assert _rel(b, ref) < 1e-13


@pytest.mark.parametrize("level,k", [(2, 3.0), (3, 5.0), (3, 40.0)])
def test_dense_mode_matches_oracle(level, k):
    v, f = icosphere(level)
    x = complex_normal(len(f), seed=11)
    P = _problem(v, f, k, mode=1)
    y = P.apply(_dev(x)).cpu().numpy()
    ref = oracle.matvec(v, f, k, x)
    assert _rel(y, ref) < 1e-12


@pytest.mark.parametrize("level,k,precision", [(4, 5.0, 0), (4, 20.0, 0), (4, 20.0, 1), (4, 5.0, 1)])
def test_fda_matvec_parity(level, k, precision):
    v, f = icosphere(level)
    x = complex_normal(len(f), seed=3)
    P = _problem(v, f, k, precision=precision)
    st = P.stats()
    assert st.n_m2l > 0  # the far field is exercised
    y = P.apply(_dev(x)).cpu().numpy()
    ref = oracle.matvec(v, f, k, x)
    assert _rel(y, ref) < 1e-4


def test_fda_high_frequency_levels_present():
    v, f = icosphere(4)
    P = _problem(v, f, 20.0)
    st = P.stats()
    regimes = [st.level_regime[l] for l in range(st.n_levels)]
    assert 1 in regimes and 0 in regimes


def test_fda_ellipsoid_ragged_leaves():
    v, f = ellipsoid_from_icosphere(4)
    x = complex_normal(len(f), seed=5)
    P = _problem(v, f, 15.0)
    y = P.apply(_dev(x)).cpu().numpy()
    ref = oracle.matvec(v, f, 15.0, x)
    assert _rel(y, ref) < 1e-4


def test_fda_sampled_rows_larger_mesh():
    v, f = icosphere(6)
    k = 25.0
    x = complex_normal(len(f), seed=9)
    P = _problem(v, f, k)
    y = P.apply(_dev(x)).cpu().numpy()
    rows = np.random.default_rng(7).choice(len(f), 192, replace=False)
    ref = oracle.matvec(v, f, k, x, rows=rows)
    assert _rel(y[rows], ref) < 1e-4


def test_multi_rhs_columns():
    v, f = icosphere(3)
    x = complex_normal(len(f), seed=1, nrhs=2)
    P = _problem(v, f, 8.0)
    y2 = P.apply(_dev(x)).cpu().numpy()
    y0 = P.apply(_dev(x[0])).cpu().numpy()
    y1 = P.apply(_dev(x[1])).cpu().numpy()
    # translations accumulate with atomics, so the summation order (and the
    # last bits) may differ between calls
    assert _rel(y2[0], y0) < 1e-13 and _rel(y2[1], y1) < 1e-13


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_matches_dense_lu(precision):
    v, f = icosphere(3)
    k = 5.0
    P = _problem(v, f, k, precision=precision)
    b = P.rhs_plane_wave(np.array([0.0, 0.0, 1.0]))
    x, info = P.solve(b, 1e-8)
    a = oracle.assemble(v, f, k)
    u = oracle.lu_solve(a, oracle.rhs_plane_wave(v, f, k, [[0, 0, 1.0]])[0])
    assert info.rel_resid_fp64 <= 1e-8
    # FDA operator differs from the dense one by <= ~1e-4 relative
    assert _rel(x.cpu().numpy(), u) < 1e-3


def test_tiny_mesh_and_small_k():
    v, f = icosphere(0)  # 20 triangles: a single leaf, near field only
    x = complex_normal(len(f), seed=2)
    for k in (0.05, 3.0):
        P = _problem(v, f, k)
        y = P.apply(_dev(x)).cpu().numpy()
        assert _rel(y, oracle.matvec(v, f, k, x)) < 1e-12


def test_errors_are_reported():
    from paper_1403_4747_gb300 import (fda_create, fda_default_config, fda_build_tree, fda_apply,
                                       fda_precompute_translations, FDAError, FDA_ERR_ARG, FDA_ERR_STATE,
                                       fda_destroy)
    v, f = icosphere(1)
    h = fda_create(fda_default_config())
    with pytest.raises(FDAError) as e:
        fda_precompute_translations(h)
    assert e.value.status == FDA_ERR_STATE
    with pytest.raises(FDAError) as e:
        fda_build_tree(h, v, f, -1.0)
    assert e.value.status == FDA_ERR_ARG
    bad = f.copy(); bad[0, 0] = len(v) + 5
    with pytest.raises(FDAError) as e:
        fda_build_tree(h, v, bad, 1.0)
    assert e.value.status == FDA_ERR_ARG
    deg = f.copy(); deg[0, 1] = deg[0, 0]
    with pytest.raises(FDAError) as e:
        fda_build_tree(h, v, deg, 1.0)
    assert e.value.status == FDA_ERR_ARG
    from paper_1403_4747_gb300 import fda_set_tc_tiles
    for shape in ((16, 1, 2), (32, 4, 2), (64, 1, 5)):
        with pytest.raises(FDAError) as e:
            fda_set_tc_tiles(h, *shape)
        assert e.value.status == FDA_ERR_ARG
    fda_set_tc_tiles(h, 32, 3, 3)
    fda_set_tc_tiles(h, 0, 0, 0)
    fda_destroy(h)


@pytest.mark.parametrize("precision", [0, 1])
def test_blockdiag_preconditioner_same_solution(precision):
    """Right preconditioning leaves the solution unchanged (the residual is
    the unpreconditioned one).  It does not lower the iteration count for
    this operator; that is measured in the benchmark, not asserted here."""
    from paper_1403_4747_gb300 import fda_set_precond
    v, f = icosphere(3)
    k = 6.0
    P = _problem(v, f, k, precision=precision, precond=1, maxit=4000, restart=200)
    b = P.rhs_plane_wave(np.array([0.0, 0.0, 1.0]))
    fda_set_precond(P.h, 0)
    x0, i0 = P.solve(b, 1e-6)
    fda_set_precond(P.h, 1)
    x1, i1 = P.solve(b, 1e-6)
    assert i0.rel_resid_fp64 <= 1e-6 and i1.rel_resid_fp64 <= 1e-6
    assert _rel(x1.cpu().numpy(), x0.cpu().numpy()) < 1e-5


def test_blockdiag_is_exact_inverse_on_a_single_leaf():
    """20 triangles form one leaf: the block-diagonal preconditioner is then
    the exact inverse, and GMRES converges in one iteration to the LU
    solution."""
    v, f = icosphere(0)
    k = 2.0
    P = _problem(v, f, k, precond=1)
    b = P.rhs_plane_wave(np.array([0.0, 0.0, 1.0]))
    x, info = P.solve(b, 1e-10)
    assert info.iters <= 2
    u = oracle.lu_solve(oracle.assemble(v, f, k), oracle.rhs_plane_wave(v, f, k, [[0, 0, 1.0]])[0])
    assert _rel(x.cpu().numpy(), u) < 1e-9


@pytest.mark.parametrize("alpha_sign", [1.0, -1.0])
def test_coupling_parity(alpha_sign):
    """alpha = +i/k (as printed) and -i/k (the default): the GPU matvec and
    right-hand side match the oracle with the same coupling."""
    v, f = icosphere(4)
    k = 20.0
    x = complex_normal(len(f), seed=4)
    P = _problem(v, f, k, alpha_sign=alpha_sign)
    y = P.apply(_dev(x)).cpu().numpy()
    assert _rel(y, oracle.matvec(v, f, k, x, alpha_sign=alpha_sign)) < 1e-4
    b = P.rhs_plane_wave(np.array([0.0, 0.0, 1.0])).cpu().numpy()
    assert _rel(b, oracle.rhs_plane_wave(v, f, k, [[0.0, 0.0, 1.0]], alpha_sign=alpha_sign)[0]) < 1e-13


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_right_hand_sides(precision):
    """max_rhs = 12: 11 columns in one pass (S2M/translations/L2T over all of
    them, the near field in groups of 8) equal the one-column applies, and
    column 4 matches the oracle."""
    v, f = icosphere(4)
    k = 20.0
    x = complex_normal(len(f), seed=21, nrhs=11)
    P1 = _problem(v, f, k, precision=precision)
    Pm = _problem(v, f, k, precision=precision, max_rhs=12)
    ym = Pm.apply(_dev(x)).cpu().numpy()
    for m in range(11):
        y1 = P1.apply(_dev(x[m])).cpu().numpy()
        assert _rel(ym[m], y1) < (1e-12 if precision == 0 else 1e-5)
    assert _rel(ym[4], oracle.matvec(v, f, k, x[4])) < 1e-4


@pytest.mark.parametrize("level,k,nrhs", [(4, 20.0, 1), (5, 25.0, 1), (4, 20.0, 5)])
def test_tensor_core_m2l_matches_simt_and_oracle(level, k, nrhs):
    """Chosen precision: the split-bf16 tcgen05 M2L agrees with the FP32
    SIMT M2L to ~1e-5 and with the oracle to the FDA tolerance."""
    from paper_1403_4747_gb300 import fda_set_tensor_cores
    v, f = icosphere(level)
    x = complex_normal(len(f), seed=31, nrhs=nrhs if nrhs > 1 else None)
    P = _problem(v, f, k, precision=1, tensor_cores=1, max_rhs=max(1, nrhs))
    xd = _dev(x)
    y_tc = P.apply(xd).cpu().numpy()
    fda_set_tensor_cores(P.h, 0)
    y_simt = P.apply(xd).cpu().numpy()
    assert _rel(y_tc, y_simt) < 2e-5
    if nrhs == 1:
        rows = np.random.default_rng(5).choice(len(f), 256, replace=False)
        assert _rel(y_tc[rows], oracle.matvec(v, f, k, x, rows=rows)) < 1e-4
    else:
        assert _rel(y_tc[2], oracle.matvec(v, f, k, x[2])) < 1e-4


def test_graph_replay_matches_eager_launches():
    """Applies replayed from the captured CUDA graph (third call on) agree with
    eager launches, for one and several right-hand sides and both precisions;
    a solve through the graph cache reaches the same solution."""
    v, f = icosphere(4)
    k = 20.0
    x1 = _dev(complex_normal(len(f), seed=41))
    x3 = _dev(complex_normal(len(f), seed=42, nrhs=3))
    G = _problem(v, f, k, precision=1, max_rhs=3, graphs=1)
    E = _problem(v, f, k, precision=1, max_rhs=3, graphs=0)
    from paper_1403_4747_gb300 import fda_set_precision
    for prec, tol in ((1, 1e-6), (0, 1e-12)):
        fda_set_precision(G.h, prec)
        fda_set_precision(E.h, prec)
        ref1 = E.apply(x1).cpu().numpy()
        ref3 = E.apply(x3).cpu().numpy()
        for _ in range(4):  # eager, capture, replay, replay
            assert _rel(G.apply(x1).cpu().numpy(), ref1) < tol
            assert _rel(G.apply(x3).cpu().numpy(), ref3) < tol
    st = G.stats()
    assert st.graph_fallback == 0 and st.graph_replays >= 8
    assert E.stats().graph_replays == 0
    fda_set_precision(G.h, 1)
    fda_set_precision(E.h, 1)
    b = G.rhs_plane_wave(np.array([0.0, 0.0, 1.0]))
    xg, ig = G.solve(b, 1e-6)
    xe, ie = E.solve(b, 1e-6)
    assert abs(ig.iters - ie.iters) <= 2
    assert _rel(xg.cpu().numpy(), xe.cpu().numpy()) < 1e-5


@pytest.mark.parametrize("nrhs", [2, 20, 40, 64])
def test_leaf_products_on_tensor_cores(nrhs):
    """Several right-hand sides in the chosen precision: the near field, S2M
    and L2T run as tcgen05 GEMMs with the right-hand sides as columns (16, 32
    or 64 per tile; 40 leaves a partial group).  They agree with the CUDA-core
    path (tensor cores off) to the split-bf16 accuracy, and a column agrees
    with the oracle to the FDA tolerance."""
    from paper_1403_4747_gb300 import fda_set_tensor_cores
    v, f = icosphere(4)
    k = 20.0
    x = complex_normal(len(f), seed=51, nrhs=nrhs)
    P = _problem(v, f, k, precision=1, max_rhs=nrhs)
    xd = _dev(x)
    y_tc = P.apply(xd).cpu().numpy()
    fda_set_tensor_cores(P.h, 0)
    y_simt = P.apply(xd).cpu().numpy()
    assert np.all(np.isfinite(y_tc))
    assert _rel(y_tc, y_simt) < 2e-5
    m = nrhs - 1
    assert _rel(y_tc[m], oracle.matvec(v, f, k, x[m])) < 1e-4


@pytest.mark.parametrize("precision", [0, 1])
def test_lowrank_m2l_matches_full_and_oracle(precision):
    """Sec. 4.2: with each reduced M2L operator factorised as U^ V^ at eps
    (Eq. epsk) and applied as two products, the matvec stays within the FDA
    tolerance of the oracle and close to the same matvec with every operator
    in full; the statistics show low-rank operators with r < T/2 at the levels
    where T is large enough for the two stages to be cheaper."""
    v, f = icosphere(5)
    k = 25.0
    x = complex_normal(len(f), seed=61)
    on = _problem(v, f, k, precision=precision)
    off = _problem(v, f, k, precision=precision, lowrank=0)
    st = on.stats()
    nl = st.n_levels
    assert sum(st.level_lr_ops[l] for l in range(nl)) > 0
    assert sum(off.stats().level_lr_ops[l] for l in range(nl)) == 0
    for l in range(nl):
        if st.level_lr_ops[l]:
            assert 0 < st.level_lr_rank_max[l] < st.level_rank[l] / 2
            assert st.level_lr_pairs[l] > 0
            # the method's flops of that level drop below the full form's
            # where the handle's precision applies the low-rank form (always
            # on the CUDA cores; on the tensor cores where the setup
            # autotuner found it faster)
            if precision == 0 or (st.level_lr_tc[l] & 1):
                assert st.level_m2l_flops[l] < 8.0 * st.level_rank[l] ** 2 * st.level_m2l_pairs[l]
    so = off.stats()
    for l in range(nl):
        T = so.level_rank[l]
        if T == 0 or so.level_m2l_pairs[l] == 0:
            continue
        # full form: 8 T^2 flops per pair; each distinct operator once, source
        # densities once, target densities read and written once (8 bytes each)
        assert so.level_m2l_flops[l] == 8.0 * T * T * so.level_m2l_pairs[l]
        assert so.level_m2l_bytes[l] == 8.0 * so.level_m2l_ops[l] * T * T + 24.0 * so.level_boxes[l] * so.level_cones[l] * T
    xd = _dev(x)
    y_on = on.apply(xd).cpu().numpy()
    y_off = off.apply(xd).cpu().numpy()
    ref = oracle.matvec(v, f, k, x)
    assert _rel(y_on, ref) < 1e-4 and _rel(y_off, ref) < 1e-4
    assert _rel(y_on, y_off) < 1e-4


def test_graphs_survive_changing_right_hand_side_counts():
    """One handle with graphs and the low-rank M2L applies one, then eight,
    then one right-hand side again (each count captured and replayed), then
    solves: every result equals an eager handle's, so no captured graph
    points at a buffer that a later count re-sized."""
    v, f = icosphere(5)
    k = 25.0
    x1 = _dev(complex_normal(len(f), seed=71))
    x8 = _dev(complex_normal(len(f), seed=72, nrhs=8))
    G = _problem(v, f, k, precision=1, max_rhs=8, graphs=1)
    E = _problem(v, f, k, precision=1, max_rhs=8, graphs=0)
    assert sum(G.stats().level_lr_ops[l] for l in range(G.stats().n_levels)) > 0
    r1, r8 = E.apply(x1).cpu().numpy(), E.apply(x8).cpu().numpy()
    for x, r in ((x1, r1), (x8, r8), (x1, r1)):
        for _ in range(3):
            assert _rel(G.apply(x).cpu().numpy(), r) < 1e-6
    b = G.rhs_plane_wave(np.array([0.0, 0.0, 1.0]))
    xg, ig = G.solve(b, 1e-6)
    xe, ie = E.solve(b, 1e-6)
    assert ig.rel_resid_fp64 <= 1e-6 and _rel(xg.cpu().numpy(), xe.cpu().numpy()) < 1e-5
