"""What the near-field-pattern objective of the learned preconditioner can
reach (CPU, no GPU): its exact minimiser, M[B, C_B] = rows B of
A_near[C_B, C_B]^-1 for every leaf B (zero objective), used as a right
preconditioner of the oracle's dense operator in the oracle's GMRES.

Unit sphere, icosphere levels 3 and 4 (N = 1,280 and 5,120), k = 5,
alpha = -i/k, plane wave +z, tolerance 1e-5, restart 100; leaves and
near-field columns from the plain construction of the tree and lists
(tests/tree_reference.py).  Measured: none 16 / 22 iterations, leaf
block-diagonal inverse 14 / 19, exact minimiser of the near-field objective
7 / 10.  The learned network on the same
objective does not come close to this (test_gpu_sai.py); this test pins the
bound it is measured against."""
import numpy as np
import pytest

import oracle
from inputs import icosphere
from tree_reference import reference_tree, reference_lists


def _leaves(v, f, k):
    levels = reference_tree(v, f, k)
    _, near = reference_lists(levels)
    out = []
    for l, L in enumerate(levels):
        for cc, isleaf in L["leaf"].items():
            if isleaf:
                out.append((np.array(sorted(L["boxes"][cc])), np.array(sorted(near[(l, cc)]))))
    return out


@pytest.mark.parametrize("level", [3, 4])
def test_exact_minimiser_of_the_near_objective_halves_gmres(level):
    v, f = icosphere(level)
    k = 5.0
    n = len(f)
    A = oracle.assemble(v, f, k)
    b = np.asarray(oracle.rhs_plane_wave(v, f, k, np.array([[0.0, 0.0, 1.0]]))).reshape(-1)
    leaves = _leaves(v, f, k)
    A_near = np.zeros_like(A)
    for r, c in leaves:
        A_near[np.ix_(r, c)] = A[np.ix_(r, c)]
    M = np.zeros_like(A)
    D = np.zeros_like(A)
    for r, c in leaves:
        sub = A_near[np.ix_(c, c)]
        inv = np.linalg.inv(sub)
        M[np.ix_(r, c)] = inv[np.searchsorted(c, r), :]
        # zero objective: M[B, C] A_near[C, C] = I[B, C]
        R = M[np.ix_(r, c)] @ sub - (r[:, None] == c[None, :])
        assert np.abs(R).max() < 1e-8 * np.abs(sub).max()
        D[np.ix_(r, r)] = np.linalg.inv(A[np.ix_(r, r)])
    its = {}
    x_ref = None
    for name, P in (("none", None), ("blockdiag", D), ("near_exact", M)):
        apply = (lambda y: A @ y) if P is None else (lambda y, P=P: A @ (P @ y))
        y, it, _ = oracle.gmres(apply, b, tol=1e-5, restart=100, maxit=500)
        x = y if P is None else P @ y
        if x_ref is None:
            x_ref = x
        assert np.linalg.norm(A @ x - b) <= 1.5e-5 * np.linalg.norm(b)
        assert np.linalg.norm(x - x_ref) <= 1e-3 * np.linalg.norm(x_ref)
        its[name] = it
    print("GMRES iterations:", its)
    assert its["blockdiag"] <= its["none"]
    assert 2 * its["near_exact"] <= its["none"] + 1
    assert n == 20 * 4 ** level
