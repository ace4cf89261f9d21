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
