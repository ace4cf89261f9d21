"""Oracle solvers (test infrastructure): dense LU and a plain restarted GMRES.

GMRES follows the paper's solver setting (Sec. 5): no preconditioner,
convergence when the relative 2-norm of the residual of the unpreconditioned
system falls to the tolerance.  Restart length, zero initial guess and
modified Gram-Schmidt with one re-orthogonalisation are readings of what the
paper leaves open.
"""
from __future__ import annotations

import numpy as np


def lu_solve(a, b):
    """Dense direct solve (LAPACK getrf/getrs through numpy)."""
    return np.linalg.solve(a, b)


def gmres(apply, b, tol=1e-5, restart=200, maxit=2000, x0=None):
    """Restarted GMRES(m).  apply(x) -> A x.  Returns (x, iters, history)."""
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, [0.0]
    hist = []
    iters = 0
    while iters < maxit:
        r = b - apply(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta / bnorm <= tol:
            break
        m = min(restart, maxit - iters)
        V = np.zeros((m + 1, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        V[0] = r / beta
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        j_done = 0
        for j in range(m):
            w = apply(V[j])
            for _ in range(2):  # MGS plus one re-orthogonalisation pass
                for i in range(j + 1):
                    h = np.vdot(V[i], w)
                    H[i, j] += h
                    w = w - h * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            # apply previous Givens rotations to column j
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
                H[i, j] = t
            a_, b_ = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a_) ** 2 + abs(b_) ** 2)
            if den == 0.0:
                cs[j], sn[j] = 1.0, 0.0
            else:
                cs[j] = a_ / den
                sn[j] = b_ / den
                cs[j], sn[j] = np.conj(cs[j]), np.conj(sn[j])
            H[j, j] = cs[j] * a_ + sn[j] * b_
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= tol or iters >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + V[:j_done].T @ y
        if hist[-1] <= tol:
            r = b - apply(x)
            hist.append(np.linalg.norm(r) / bnorm)
            if hist[-1] <= tol * 1.0000001:
                break
    return x, iters, hist
