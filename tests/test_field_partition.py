"""The source partition behind the fast off-surface field
(fda_scattered_field_fast), on the plain tree construction of
tests/tree_reference.py (no GPU).  A point is placed in the deepest box of
the tree whose cube contains it.  If that box A is a low-frequency box at
or below the coarsest level with interaction lists, A's local density
covers the sources in the interaction lists of A and its ancestors, and the
rest is A's near field by the leaf rule of Sec. 3.3 Step 1 with every near
box that has children opened; otherwise the whole tree is opened from the
root.  Opening box B at level l: a child whose cube is not near the point's
cube of level l + 1 (at a level with interaction lists) counts through its
equivalent sources, the other children are opened in turn, and a leaf is
summed element by element.  Every element must be counted exactly once, for
points of every kind (inside leaf cubes, in empty cubes around and inside
the body, outside the root cube).  The count does not depend on which boxes
the admissibility test accepts (any test partitions an opened box); that
the accepted boxes' equivalent sources are accurate is checked on the GPU
against the oracle (test_gpu_field.py)."""
from collections import Counter

import numpy as np

from inputs import icosphere, ellipsoid_from_icosphere
from tree_reference import reference_tree, reference_lists, is_near

OFFS = [np.array([dx, dy, dz]) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _cell(L, x):
    return tuple(int(c) for c in np.floor((x - L["root"]) / L["w"]))


def _partition(levels, il, lev_lo, x):
    nlev = len(levels)
    counts = Counter()
    chain = []
    for l in range(nlev):
        c = _cell(levels[l], x)
        if c not in levels[l]["boxes"]:
            break
        chain.append(c)
        if levels[l]["leaf"][c]:
            break
    lA = len(chain) - 1
    S, l0 = [], 0
    l2t = lA >= 0 and not levels[lA]["hf"] and lA >= lev_lo
    if l2t:
        for l in range(lev_lo, lA + 1):  # the local density of A
            for c in il.get((l, chain[l]), ()):
                counts.update(levels[l]["boxes"][c])
        for l in range(lA + 1):  # A's near field as if A were a leaf
            if levels[l]["hf"] and l != lA:
                continue
            for d in OFFS:
                X = tuple(np.array(chain[l]) + d)
                if X not in levels[l]["boxes"]:
                    continue
                if levels[l]["leaf"][X]:
                    counts.update(levels[l]["boxes"][X])
                elif l == lA:
                    S.append(X)
        l0 = lA
    elif 0 < nlev:
        S = [next(iter(levels[0]["boxes"]))]
    l = l0
    while S and l < nlev:
        nxt = []
        for B in S:
            if levels[l]["leaf"][B]:
                counts.update(levels[l]["boxes"][B])
                continue
            cx = np.array(_cell(levels[l + 1], x))
            for C in levels[l + 1]["boxes"]:
                if tuple(np.array(C) >> 1) != B:
                    continue
                if l + 1 >= lev_lo and not is_near(levels[l + 1], cx - np.array(C)):
                    counts.update(levels[l + 1]["boxes"][C])  # equivalent sources
                else:
                    nxt.append(C)
        S, l = nxt, l + 1
    return counts, l2t


def _points(seed):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(40, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = np.concatenate([np.full(12, 1.03), np.full(8, 1.3), np.full(8, 0.45), np.full(6, 2.5), np.full(6, 9.0)])
    return d * r[:, None]


def _check(v, f, k):
    levels = reference_tree(v, f, k)
    il, _ = reference_lists(levels)
    lev_lo = min(l for (l, _), s in il.items() if s)
    assert any(levels[l]["hf"] and l >= lev_lo for l in range(len(levels)))  # directional M2T exercised
    modes = Counter()
    for x in _points(7):
        counts, l2t = _partition(levels, il, lev_lo, x)
        modes[l2t] += 1
        assert set(counts) == set(range(len(f))), "element missed"
        assert max(counts.values()) == 1, "element counted twice"
    assert modes[True] > 0 and modes[False] > 0  # both placements occur


def test_partition_sphere():
    v, f = icosphere(3)
    _check(v, f, 20.0)


def test_partition_ellipsoid():
    v, f = ellipsoid_from_icosphere(3)
    _check(v, f, 16.0)


def test_partition_two_high_frequency_levels():
    """Level-4 sphere at k = 40: levels 2 and 3 are high-frequency (rho 3.2
    and 2.2 widths), level 4 low-frequency, so the walk opens boxes through
    two directional levels before it reaches the leaves."""
    v, f = icosphere(4)
    _check(v, f, 40.0)
