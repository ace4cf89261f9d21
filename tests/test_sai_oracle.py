"""Pins of the learned-preconditioner oracle (oracle/sai.py) that need no GPU:
the chain-rule gradient against central finite differences, a closed-form
special case of the loss, invariance of the features under rotations of the
geometry, and the library's host-side weight initialisation."""
import numpy as np
import pytest

from oracle import sai


def _problem(seed=0, nblocks=3):
    rng = np.random.default_rng(seed)
    sizes = [3, 5, 4][:nblocks]
    n = sum(sizes)
    cent = rng.normal(size=(n, 3)) * 0.05
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    area = rng.uniform(1e-4, 4e-4, size=n)
    bp = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    be = rng.permutation(n).astype(np.int32)
    blocks = [rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m)) + 2 * np.eye(m) for m in sizes]
    return cent, nrm, area, 7.5, bp, be, blocks


def test_gradient_matches_central_differences():
    cent, nrm, area, k, bp, be, blocks = _problem()
    w = np.random.default_rng(1).normal(size=sai.NPARAMS) * 0.3
    L, g = sai.loss_grad(w, cent, nrm, area, k, bp, be, blocks)
    assert np.isclose(L, sai.loss(w, cent, nrm, area, k, bp, be, blocks), rtol=1e-13)
    idx = np.random.default_rng(2).choice(sai.NPARAMS, 60, replace=False)
    idx = np.concatenate([idx, [sai.NPARAMS - 1, sai.NPARAMS - 2, 0]])  # biases of the output, first weight
    h = 1e-6
    for p in idx:
        wp, wm = w.copy(), w.copy()
        wp[p] += h
        wm[p] -= h
        fd = (sai.loss(wp, cent, nrm, area, k, bp, be, blocks) - sai.loss(wm, cent, nrm, area, k, bp, be, blocks)) / (2 * h)
        assert abs(fd - g[p]) <= 1e-6 * max(1.0, abs(g[p])), (p, fd, g[p])


def test_constant_network_gives_closed_form_loss():
    # W3 = 0: every entry of M equals b3 = c, so M_B = c J (J all ones)
    cent, nrm, area, k, bp, be, blocks = _problem(3)
    w = np.random.default_rng(4).normal(size=sai.NPARAMS)
    c = 0.3 - 0.7j
    P = sai.unpack(w)
    o = sai.NPARAMS
    w[o - 2 - 2 * sai.NH:o - 2] = 0.0
    w[o - 2], w[o - 1] = c.real, c.imag
    expect = sum(np.sum(np.abs(c * np.ones((len(A), len(A))) @ A - np.eye(len(A))) ** 2) for A in blocks) / bp[-1]
    assert np.isclose(sai.loss(w, cent, nrm, area, k, bp, be, blocks), expect, rtol=1e-12)
    assert P["W1"].shape == (sai.NH, sai.NF)


def test_features_are_rotation_invariant():
    cent, nrm, area, k, bp, be, blocks = _problem(5)
    q, _ = np.linalg.qr(np.random.default_rng(6).normal(size=(3, 3)))
    w = np.random.default_rng(7).normal(size=sai.NPARAMS) * 0.2
    a = sai.loss(w, cent, nrm, area, k, bp, be, blocks)
    b = sai.loss(w, cent @ q.T, nrm @ q.T, area, k, bp, be, blocks)
    assert np.isclose(a, b, rtol=1e-12)


def test_library_initial_weights():
    F = pytest.importorskip("paper_1403_4747_gb300")
    from paper_1403_4747_gb300 import build
    build.build()
    assert F.fda_sai_num_params() == sai.NPARAMS
    w = F.fda_sai_init_weights(3).astype(np.float64)
    P = sai.unpack(w)
    for name, fan in (("W1", sai.NF + sai.NH), ("W2", 2 * sai.NH), ("W3", sai.NH + 2)):
        bound = np.sqrt(6.0 / fan)
        assert np.abs(P[name]).max() <= bound and np.abs(P[name]).max() > 0.5 * bound
    for name in ("b1", "b2", "b3"):
        assert not P[name].any()
    assert np.array_equal(w, F.fda_sai_init_weights(3).astype(np.float64))
    assert not np.array_equal(w, F.fda_sai_init_weights(4).astype(np.float64))


# ---- near-field pattern (rows of a leaf x the leaf's near-field columns)

def _near_problem(seed=10):
    """Four blocks of 3-5 elements; block b's columns are its own elements
    and those of one or two other blocks; A_near random on the union of the
    block x column patterns, 0 elsewhere."""
    rng = np.random.default_rng(seed)
    sizes = [4, 3, 5, 4]
    n = sum(sizes)
    cent = rng.normal(size=(n, 3)) * 0.05
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    area = rng.uniform(1e-4, 4e-4, size=n)
    perm = rng.permutation(n)
    bounds = np.concatenate([[0], np.cumsum(sizes)])
    rows = [perm[bounds[b]:bounds[b + 1]] for b in range(4)]
    nbrs = [[0, 1], [1, 0, 2], [2, 1, 3], [3, 2]]
    cols = [np.sort(np.concatenate([rows[c] for c in nb])) for nb in nbrs]
    A = np.zeros((n, n), dtype=complex)
    for r, c in zip(rows, cols):
        A[np.ix_(r, c)] = rng.normal(size=(len(r), len(c))) + 1j * rng.normal(size=(len(r), len(c)))
    A += 2.0 * np.eye(n)
    return cent, nrm, area, 6.0, rows, cols, A


def test_near_gradient_matches_central_differences():
    cent, nrm, area, k, rows, cols, A = _near_problem()
    w = np.random.default_rng(11).normal(size=sai.NPARAMS) * 0.3
    L, g = sai.loss_grad_near(w, cent, nrm, area, k, rows, cols, A)
    idx = np.random.default_rng(12).choice(sai.NPARAMS, 50, replace=False)
    idx = np.concatenate([idx, [sai.NPARAMS - 1, sai.NPARAMS - 2, 0]])
    h = 1e-6
    for p in idx:
        wp, wm = w.copy(), w.copy()
        wp[p] += h
        wm[p] -= h
        fd = (sai.loss_grad_near(wp, cent, nrm, area, k, rows, cols, A)[0]
              - sai.loss_grad_near(wm, cent, nrm, area, k, rows, cols, A)[0]) / (2 * h)
        assert abs(fd - g[p]) <= 1e-6 * max(1.0, abs(g[p])), (p, fd, g[p])


def test_near_objective_on_self_blocks_is_the_block_objective():
    """Columns = the block's own rows and A_near block-diagonal: the
    near-pattern objective and its gradient reduce to the leaf-block ones."""
    cent, nrm, area, k, bp, be, blocks = _problem(13)
    n = len(cent)
    rows = [be[bp[b]:bp[b + 1]] for b in range(len(blocks))]
    A = np.zeros((n, n), dtype=complex)
    for r, B in zip(rows, blocks):
        A[np.ix_(r, r)] = B
    w = np.random.default_rng(14).normal(size=sai.NPARAMS) * 0.3
    L0, g0 = sai.loss_grad(w, cent, nrm, area, k, bp, be, blocks)
    L1, g1 = sai.loss_grad_near(w, cent, nrm, area, k, rows, rows, A)
    assert np.isclose(L0, L1, rtol=1e-13)
    assert np.allclose(g0, g1, rtol=1e-12, atol=1e-14 * np.abs(g0).max())


def test_near_constant_network_on_identity_closed_form():
    """W3 = 0 (M_ij = c on the pattern) and A_near = I: each row of a block
    with nc columns has residual c - 1 once and c nc - 1 times, so
    L = sum_B n_B (nc_B |c|^2 - 2 Re c + 1) / sum_B n_B and
    dL/db3 = 2 sum_B n_B (nc_B c - 1) / sum_B n_B (Re and Im parts)."""
    cent, nrm, area, k, rows, cols, _ = _near_problem(15)
    n = len(cent)
    w = np.random.default_rng(16).normal(size=sai.NPARAMS)
    c = 0.4 - 0.25j
    o = sai.NPARAMS
    w[o - 2 - 2 * sai.NH:o - 2] = 0.0
    w[o - 2], w[o - 1] = c.real, c.imag
    L, g = sai.loss_grad_near(w, cent, nrm, area, k, rows, cols, np.eye(n, dtype=complex))
    nb = np.array([len(r) for r in rows], dtype=float)
    nc = np.array([len(q) for q in cols], dtype=float)
    expect = np.sum(nb * (nc * abs(c) ** 2 - 2 * c.real + 1)) / nb.sum()
    assert np.isclose(L, expect, rtol=1e-13)
    assert np.isclose(g[o - 2], 2 * np.sum(nb * (nc * c.real - 1)) / nb.sum(), rtol=1e-12)
    assert np.isclose(g[o - 1], 2 * np.sum(nb * nc * c.imag) / nb.sum(), rtol=1e-12)
    # the weights of the last layer see only h2, which the closed form does not fix; the
    # hidden layers get no gradient through W3 = 0
    assert np.all(g[:o - 2 - 2 * sai.NH] == 0.0)


def test_near_objective_ignores_entries_outside_the_pattern():
    """Entries of A_near in rows or columns outside a block's near field do
    not enter that block's term."""
    cent, nrm, area, k, rows, cols, A = _near_problem(17)
    w = np.random.default_rng(18).normal(size=sai.NPARAMS) * 0.3
    one = ([rows[0]], [cols[0]])
    L0, g0 = sai.loss_grad_near(w, cent, nrm, area, k, *one, A)
    B = A.copy()
    outside = np.setdiff1d(np.arange(len(cent)), cols[0])
    B[np.ix_(cols[0], outside)] = 5.0 + 3.0j
    B[np.ix_(outside, cols[0])] = -2.0j
    L1, g1 = sai.loss_grad_near(w, cent, nrm, area, k, *one, B)
    assert L0 == L1 and np.array_equal(g0, g1)
