"""Learned sparse-approximate-inverse preconditioner: plain FP64 reference of
the network, its training loss and the loss gradient (TEST INFRASTRUCTURE).

This is the library's learned preconditioner, not a method of the paper (the
paper solves without a preconditioner, Sec. 5.3).  Definitions:

  pair features (i, j), r = x_j - x_i, d = |r|, h_e = sqrt(area_e):
      f = [k d, (r . n_i)/d, (r . n_j)/d, n_i . n_j, k h_i, k h_j,
           [i == j], h_j / max(d, h_j)]         (the two projections are 0 for i == j)
  network:  h1 = tanh(W1 f + b1), h2 = tanh(W2 h1 + b2), (Re, Im) M_ij = W3 h2 + b3
            W1 32x8, W2 32x32, W3 2x32; flat weights W1, b1, W2, b2, W3, b3
  loss over blocks B (element index lists) with matrices A_B = A[B, B]:
      L = (1 / sum_B n_B) sum_B || M_B A_B - I ||_F^2

The gradient is written out by the chain rule (dL/dRe M_ij + i dL/dIm M_ij =
2 (R A^H)_ij / sum n_B with R = M A - I, then back through the two layers);
tests pin it by central finite differences of `loss`.

Near-field pattern (`loss_grad_near`): the same network predicts M_ij for
every row i of a leaf B and every column j of B's near field C_B (the leaf's
own elements and those of its near leaves), and the objective compares
M A_near with the identity on that pattern:
      L = (1 / sum_B n_B) sum_B || M[B, C_B] A_near[C_B, C_B] - I[B, C_B] ||_F^2,
A_near the near-field part of the matrix (entries of pairs outside the near
field are 0), I[B, C_B] the identity's rows B restricted to the columns C_B.
With C_B = B and a block-diagonal A_near it is `loss` above.
"""
from __future__ import annotations

import numpy as np

NF, NH = 8, 32
SIZES = [("W1", (NH, NF)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (2, NH)), ("b3", (2,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(w):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(w[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def features(cent, nrm, area, k, I, J):
    """Feature rows for the pairs (I[q], J[q])."""
    r = cent[J] - cent[I]
    d = np.linalg.norm(r, axis=1)
    self_ = I == J
    dsafe = np.where(self_, 1.0, d)
    hi, hj = np.sqrt(area[I]), np.sqrt(area[J])
    f = np.empty((len(I), NF))
    f[:, 0] = k * d
    f[:, 1] = np.where(self_, 0.0, np.einsum("qc,qc->q", r, nrm[I]) / dsafe)
    f[:, 2] = np.where(self_, 0.0, np.einsum("qc,qc->q", r, nrm[J]) / dsafe)
    f[:, 3] = np.einsum("qc,qc->q", nrm[I], nrm[J])
    f[:, 4] = k * hi
    f[:, 5] = k * hj
    f[:, 6] = self_.astype(np.float64)
    f[:, 7] = hj / np.maximum(d, hj)
    return f


def _pairs(block_ptr, block_elems, b):
    e = np.asarray(block_elems[block_ptr[b]:block_ptr[b + 1]])
    n = len(e)
    return np.repeat(e, n), np.tile(e, n), n


def predict(w, cent, nrm, area, k, block_ptr, block_elems):
    """M_B (complex, row-major n_B x n_B) for every block."""
    P = unpack(w)
    out = []
    for b in range(len(block_ptr) - 1):
        I, J, n = _pairs(block_ptr, block_elems, b)
        f = features(cent, nrm, area, k, I, J)
        h1 = np.tanh(f @ P["W1"].T + P["b1"])
        h2 = np.tanh(h1 @ P["W2"].T + P["b2"])
        o = h2 @ P["W3"].T + P["b3"]
        out.append((o[:, 0] + 1j * o[:, 1]).reshape(n, n))
    return out


def loss(w, cent, nrm, area, k, block_ptr, block_elems, blocks):
    """L for blocks given as a list of n_B x n_B complex matrices."""
    Ms = predict(w, cent, nrm, area, k, block_ptr, block_elems)
    total = sum(np.sum(np.abs(M @ A - np.eye(len(A))) ** 2) for M, A in zip(Ms, blocks))
    return total / float(block_ptr[-1])


def loss_grad(w, cent, nrm, area, k, block_ptr, block_elems, blocks):
    """(L, dL/dw) with the chain rule written out."""
    P = unpack(w)
    g = {name: np.zeros(shape) for name, shape in SIZES}
    scale = 1.0 / float(block_ptr[-1])
    total = 0.0
    for b, A in enumerate(blocks):
        I, J, n = _pairs(block_ptr, block_elems, b)
        f = features(cent, nrm, area, k, I, J)
        h1 = np.tanh(f @ P["W1"].T + P["b1"])
        h2 = np.tanh(h1 @ P["W2"].T + P["b2"])
        o = h2 @ P["W3"].T + P["b3"]
        M = (o[:, 0] + 1j * o[:, 1]).reshape(n, n)
        R = M @ A - np.eye(n)
        total += np.sum(np.abs(R) ** 2)
        G = (2.0 * scale) * (R @ A.conj().T)          # dL/dRe M + i dL/dIm M
        d3 = np.stack([G.real.ravel(), G.imag.ravel()], axis=1)
        g["W3"] += d3.T @ h2
        g["b3"] += d3.sum(axis=0)
        d2 = (d3 @ P["W3"]) * (1.0 - h2 ** 2)
        g["W2"] += d2.T @ h1
        g["b2"] += d2.sum(axis=0)
        d1 = (d2 @ P["W2"]) * (1.0 - h1 ** 2)
        g["W1"] += d1.T @ f
        g["b1"] += d1.sum(axis=0)
    flat = np.concatenate([g[name].ravel() for name, _ in SIZES])
    return total * scale, flat


def _forward(P, f):
    h1 = np.tanh(f @ P["W1"].T + P["b1"])
    h2 = np.tanh(h1 @ P["W2"].T + P["b2"])
    o = h2 @ P["W3"].T + P["b3"]
    return h1, h2, o


def predict_near(w, cent, nrm, area, k, row_sets, col_sets):
    """M[B, C_B] (complex, len(B) x len(C_B)) for every block."""
    P = unpack(w)
    out = []
    for rows, cols in zip(row_sets, col_sets):
        rows, cols = np.asarray(rows), np.asarray(cols)
        I, J = np.repeat(rows, len(cols)), np.tile(cols, len(rows))
        _, _, o = _forward(P, features(cent, nrm, area, k, I, J))
        out.append((o[:, 0] + 1j * o[:, 1]).reshape(len(rows), len(cols)))
    return out


def loss_grad_near(w, cent, nrm, area, k, row_sets, col_sets, A_near):
    """(L, dL/dw) of the near-field-pattern objective for blocks with rows
    row_sets[b] and near-field columns col_sets[b] (element indices; each
    block's rows among its columns), A_near a dense complex matrix holding
    the near-field entries and 0 elsewhere.  The gradient is the chain rule
    of `loss_grad` with R = M[B, C] A_near[C, C] - I[B, C] and
    dL/dRe M + i dL/dIm M = 2 R A_near[C, C]^H / sum n_B."""
    P = unpack(w)
    g = {name: np.zeros(shape) for name, shape in SIZES}
    nrows = sum(len(r) for r in row_sets)
    scale = 1.0 / float(nrows)
    total = 0.0
    for rows, cols in zip(row_sets, col_sets):
        rows, cols = np.asarray(rows), np.asarray(cols)
        n, nc = len(rows), len(cols)
        I, J = np.repeat(rows, nc), np.tile(cols, n)
        f = features(cent, nrm, area, k, I, J)
        h1, h2, o = _forward(P, f)
        M = (o[:, 0] + 1j * o[:, 1]).reshape(n, nc)
        Asub = A_near[np.ix_(cols, cols)]
        E = (rows[:, None] == cols[None, :]).astype(np.float64)
        R = M @ Asub - E
        total += np.sum(np.abs(R) ** 2)
        G = (2.0 * scale) * (R @ Asub.conj().T)
        d3 = np.stack([G.real.ravel(), G.imag.ravel()], axis=1)
        g["W3"] += d3.T @ h2
        g["b3"] += d3.sum(axis=0)
        d2 = (d3 @ P["W3"]) * (1.0 - h2 ** 2)
        g["W2"] += d2.T @ h1
        g["b2"] += d2.sum(axis=0)
        d1 = (d2 @ P["W2"]) * (1.0 - h1 ** 2)
        g["W1"] += d1.T @ f
        g["b1"] += d1.sum(axis=0)
    flat = np.concatenate([g[name].ravel() for name, _ in SIZES])
    return total * scale, flat
