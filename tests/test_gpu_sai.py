"""Learned SAI preconditioner on the GPU: the training kernels' loss and
gradient against the FP64 CPU oracle (oracle/sai.py), and what the trained
network gains in GMRES iterations over the method without it."""
import numpy as np
import pytest

import oracle
from oracle import sai
from inputs.meshes import icosphere, ellipsoid_from_icosphere

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1403_4747_gb300 import build
    build.build()
    import paper_1403_4747_gb300 as F
    return F


def _oracle_blocks(level=2, k=5.0, nb=14):
    v, f = icosphere(level)
    cent, nrm, area, _ = oracle.geometry(v, f)
    A = oracle.assemble(v, f, k)
    order = np.argsort(cent[:, 2] + 1e-3 * cent[:, 0], kind="stable")
    groups = [g for g in np.array_split(order, nb)] + [order[:1]]  # plus a 1-element block
    bp = np.concatenate([[0], np.cumsum([len(g) for g in groups])]).astype(np.int64)
    be = np.concatenate(groups).astype(np.int32)
    blocks = [A[np.ix_(g, g)] for g in groups]
    flat = np.concatenate([b.ravel() for b in blocks])
    return cent, nrm, area, k, bp, be, blocks, flat


@pytest.mark.parametrize("precision,tol_l,tol_g", [(0, 1e-12, 1e-10), (1, 2e-5, 2e-3)])
def test_loss_and_gradient_match_oracle(F, precision, tol_l, tol_g):
    cent, nrm, area, k, bp, be, blocks, flat = _oracle_blocks()
    w = np.random.default_rng(11).normal(size=sai.NPARAMS) * 0.25
    if precision == 1:
        w = w.astype(np.float32).astype(np.float64)  # the FP32 kernels see the same weights
    L_ref, g_ref = sai.loss_grad(w, cent, nrm, area, k, bp, be, blocks)
    L, g = F.fda_sai_loss_grad(cent, nrm, area, k, bp, be, flat, w, precision)
    assert abs(L - L_ref) <= tol_l * abs(L_ref)
    assert np.linalg.norm(g - g_ref) <= tol_g * np.linalg.norm(g_ref)


def test_trained_network_gain(F):
    """Train on an ellipsoid's leaf blocks, apply to the sphere of the first
    workload (level 4, k = 5, alpha = -i/k): the loss falls, the
    preconditioned solves reach the unpreconditioned solution, and the
    measured relation of the iteration counts holds: the exact block inverse
    saves a few iterations (19 against 22 when measured), the learned network
    saves none (26: its per-pair prediction of the block inverse is close in
    Frobenius norm on the training geometry, loss 0.06, but not on the sphere,
    loss 0.23, and not in the directions GMRES needs).  Asserted: the target
    loss is below that of M = 0 (1.0), block-diagonal needs no more iterations
    than none, learned at most 6 more than none."""
    import torch
    k, tol = 5.0, 1e-5
    ve, fe = ellipsoid_from_icosphere(4)
    E = F.FDAProblem(ve, fe, k)
    vs, fs = icosphere(4)
    P = F.FDAProblem(vs, fs, k, precond=1, maxit=3000, restart=100)
    w = F.fda_sai_init_weights(1)
    rep = F.fda_sai_train([E.h], F.fda_sai_default_config(epochs=400), w)
    assert np.isfinite(rep.loss_final) and rep.loss_final < 0.5 * rep.loss_init
    set_loss = F.fda_sai_set(P.h, w)
    assert np.isfinite(set_loss)
    b = P.rhs_plane_wave(np.array([0.0, 0.0, 1.0]))
    res = {}
    for name, pc in (("none", 0), ("blockdiag", 1), ("learned", 2)):
        F.fda_set_precond(P.h, pc)
        x, info = P.solve(b, tol, raise_on_not_converged=False)
        res[name] = (x.clone(), info.iters, info.rel_resid_fp64)
    x0 = res["none"][0]
    for name in ("blockdiag", "learned"):
        x, it, rr = res[name]
        assert rr <= 1.5 * tol
        assert float((x - x0).norm() / x0.norm()) <= 50 * tol
    gain = res["none"][1] - res["learned"][1]
    assert set_loss < 1.0
    assert res["blockdiag"][1] <= res["none"][1]
    assert res["learned"][1] <= res["none"][1] + 6
    print("learned SAI: train loss %.4f -> %.4f (%.2f s), sphere loss %.4f; GMRES iterations none %d, "
          "block-diagonal %d, learned %d (gain %d)" % (rep.loss_init, rep.loss_final, rep.train_s, set_loss,
                                                      res["none"][1], res["blockdiag"][1], res["learned"][1], gain))
    E.close()
    P.close()


# ---- near-field pattern

def _near_reference(F, v, f, k):
    """The handle's leaves with their rows and near-field columns (caller
    indices) from the plain construction of the tree and lists (after
    checking that the device's near field equals it), the dense near-field
    matrix A_near of the oracle, and the oracle's geometry."""
    from tree_reference import reference_tree, reference_lists
    P = F.FDAProblem(v, f, k, precision=F.FDA_PLAIN_FP64)
    t = F.fda_get_tree(P.h)
    _, near = reference_lists(reference_tree(v, f, k))
    perm = t["perm"]
    rows, cols = [], []
    for li, b in enumerate(t["leaf_box"]):
        key = (int(t["box_level"][b]), tuple(int(x) for x in t["box_coord"][b]))
        dev_cols = perm[t["nf_cols"][t["nf_colptr"][li]:t["nf_colptr"][li + 1]]]
        assert set(dev_cols.tolist()) == near[key]
        rows.append(np.sort(perm[t["box_begin"][b]:t["box_end"][b]]))
        cols.append(np.array(sorted(near[key])))
    A = oracle.assemble(v, f, k)
    A_near = np.zeros_like(A)
    for r, c in zip(rows, cols):
        A_near[np.ix_(r, c)] = A[np.ix_(r, c)]
    cent, nrm, area, _ = oracle.geometry(v, f)
    return P, rows, cols, A_near, cent, nrm, area


@pytest.mark.parametrize("precision,tol_l,tol_g", [(0, 1e-9, 1e-8), (1, 3e-5, 3e-3)])
def test_near_loss_and_gradient_match_oracle(F, precision, tol_l, tol_g):
    """Loss and gradient of the near-field objective on 12 leaves (seed 21)
    of the level-3 sphere at k = 6 against the FP64 oracle on the same
    leaves, with A_near from the oracle's own matrix."""
    v, f = icosphere(3)
    k = 6.0
    P, rows, cols, A_near, cent, nrm, area = _near_reference(F, v, f, k)
    try:
        leaves = np.sort(np.random.default_rng(21).choice(len(rows), min(12, len(rows)), replace=False))
        assert max(len(c) for c in cols) > 2 * max(len(r) for r in rows)  # wider than the leaf blocks
        w = np.random.default_rng(22).normal(size=sai.NPARAMS) * 0.25
        if precision == 1:
            w = w.astype(np.float32).astype(np.float64)
        L_ref, g_ref = sai.loss_grad_near(w, cent, nrm, area, k, [rows[i] for i in leaves],
                                          [cols[i] for i in leaves], A_near)
        L, g = F.fda_sai_loss_grad_near(P.h, w, leaves.astype(np.int32), precision)
    finally:
        P.close()
    print("near pattern, precision %d: loss %.6e (oracle %.6e), gradient rel %.2e"
          % (precision, L, L_ref, np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)))
    assert abs(L - L_ref) <= tol_l * abs(L_ref)
    assert np.linalg.norm(g - g_ref) <= tol_g * np.linalg.norm(g_ref)


def test_near_pattern_training_and_solve(F):
    """Train on the near-field pattern of an ellipsoid (level 4, k = 5),
    apply to the level-4 sphere at k = 5 (alpha = -i/k): the loss on a fixed
    draw of leaves falls (1626 -> 0.21 when measured), M covers the whole
    near-field pattern (loss 0.38 there), and the preconditioned solve
    reaches the unpreconditioned solution.  The measured relation: the
    network loses, 130 GMRES iterations against 22 without a preconditioner
    and 19 with the block-diagonal inverse, although the exact minimiser of
    the same objective needs 10 on this sphere (7 against 16 at level 3:
    test_sai_near_objective.py) -- a per-pair prediction from local geometry
    does not reproduce the rows of A_near[C_B, C_B]^-1 in the directions
    GMRES needs.  Asserted: it converges and needs at most ten times the
    unpreconditioned count."""
    k, tol = 5.0, 1e-5
    ve, fe = ellipsoid_from_icosphere(4)
    E = F.FDAProblem(ve, fe, k)
    vs, fs = icosphere(4)
    P = F.FDAProblem(vs, fs, k, precond=1, maxit=3000, restart=100)
    try:
        w = F.fda_sai_init_weights(1)
        rep = F.fda_sai_train([E.h], F.fda_sai_default_config(epochs=300, pattern=1, sample_leaves=64), w)
        assert np.isfinite(rep.loss_final) and rep.loss_final < rep.loss_init
        set_loss = F.fda_sai_set_pattern(P.h, w, 1)
        assert np.isfinite(set_loss)
        b = P.rhs_plane_wave(np.array([0.0, 0.0, 1.0]))
        res = {}
        for name, pc in (("none", 0), ("blockdiag", 1), ("learned_near", 2)):
            F.fda_set_precond(P.h, pc)
            x, info = P.solve(b, tol, raise_on_not_converged=False)
            res[name] = (x.clone(), info.iters, info.rel_resid_fp64)
        x0 = res["none"][0]
        x, it, rr = res["learned_near"]
        assert rr <= 1.5 * tol
        assert float((x - x0).norm() / x0.norm()) <= 50 * tol
        assert set_loss < 1.0
        assert res["blockdiag"][1] <= res["none"][1]
        assert it <= 10 * res["none"][1]
        print("learned near-field SAI: train loss %.4f -> %.4f (%.2f s), sphere loss %.4f; GMRES iterations "
              "none %d, block-diagonal %d, learned near-field %d"
              % (rep.loss_init, rep.loss_final, rep.train_s, set_loss, res["none"][1], res["blockdiag"][1],
                 res["learned_near"][1]))
    finally:
        E.close()
        P.close()
