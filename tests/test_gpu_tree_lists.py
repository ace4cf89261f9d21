"""Exact integer check of the device octree and lists (Sec. 3.3 Step 1)
against a plain construction written here from the same rules:

  * root cube: the bounding cube of the centroids, widened by 1e-6, centred;
    elements are placed by the integer cell of their centroid on a 2^20 grid;
  * a cube is high-frequency iff its width w >= lambda; high-frequency cubes
    are always split; a low-frequency cube with at most 64 elements is a leaf;
  * "near" at level l for an integer offset D between cubes: max|D_i| <= 1,
    or, at a high-frequency level, |D| < rho_l = max(2.2, w_l / lambda);
  * interaction list of a cube: the cubes of its level that are not near it
    and whose parents are near its parent;
  * near field of a leaf B: every leaf of a level l <= level(B) near B's
    ancestor at level l, and every non-leaf cube near B at B's level.

Beyond equality with that construction, two invariants that do not depend
on it: the far field (every interaction-list block) and the near field
together cover every ordered element pair exactly once, and every pair the
oracle integrates with the subdivided near-singular rule lies in the near
field (so the far field never needs that rule).
"""
import numpy as np
import pytest

import oracle
from inputs import icosphere, ellipsoid_from_icosphere
from tree_reference import reference_tree, reference_lists

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_4747_gb300 import build
    build.build()


@pytest.mark.parametrize("mesh,k", [("sphere3", 12.0), ("sphere4", 20.0), ("ellipsoid4", 15.0)])
def test_tree_and_lists_equal_reference_construction(mesh, k):
    from paper_1403_4747_gb300 import FDAProblem, fda_get_tree
    level = int(mesh[-1])
    v, f = icosphere(level) if mesh.startswith("sphere") else ellipsoid_from_icosphere(level)
    n = len(f)
    P = FDAProblem(v, f, k)
    try:
        t = fda_get_tree(P.h)
    finally:
        P.close()
    perm = t["perm"]
    assert sorted(perm.tolist()) == list(range(n))
    ref = reference_tree(v, f, k)
    # boxes, element sets and leaf flags, level by level
    dev = {}
    for b in range(len(t["box_level"])):
        key = (int(t["box_level"][b]), tuple(int(x) for x in t["box_coord"][b]))
        dev[key] = b
    assert len(dev) == len(t["box_level"])
    assert len(dev) == sum(len(L["boxes"]) for L in ref)
    for l, L in enumerate(ref):
        for cc, el in L["boxes"].items():
            b = dev[(l, cc)]
            got = sorted(perm[t["box_begin"][b]:t["box_end"][b]].tolist())
            assert got == el, (l, cc)
            assert bool(t["box_leaf"][b]) == L["leaf"][cc], (l, cc)
            if l > 0:
                p = t["box_parent"][b]
                assert (int(t["box_level"][p]), tuple(t["box_coord"][p])) == (l - 1, tuple(np.array(cc) >> 1))
    # interaction lists
    il, near = reference_lists(ref)
    for b in range(len(t["box_level"])):
        l = int(t["box_level"][b])
        cc = tuple(int(x) for x in t["box_coord"][b])
        srcs = t["il_src"][t["il_ptr"][b]:t["il_ptr"][b + 1]]
        got = [tuple(int(x) for x in t["box_coord"][a]) for a in srcs]
        assert all(int(t["box_level"][a]) == l for a in srcs)
        assert len(got) == len(set(got))
        assert set(got) == il.get((l, cc), set()), (l, cc)
    # near-field columns of every leaf
    for li, b in enumerate(t["leaf_box"]):
        l = int(t["box_level"][b])
        cc = tuple(int(x) for x in t["box_coord"][b])
        cols = t["nf_cols"][t["nf_colptr"][li]:t["nf_colptr"][li + 1]]
        got = perm[cols].tolist()
        assert len(got) == len(set(got))
        assert set(got) == near[(l, cc)], (l, cc)


@pytest.mark.parametrize("mesh,k", [("sphere4", 20.0), ("ellipsoid4", 15.0), ("sphere4", 3.0)])
def test_far_and_near_fields_partition_all_pairs(mesh, k):
    from paper_1403_4747_gb300 import FDAProblem, fda_get_tree
    v, f = icosphere(4) if mesh.startswith("sphere") else ellipsoid_from_icosphere(4)
    n = len(f)
    P = FDAProblem(v, f, k)
    try:
        t = fda_get_tree(P.h)
    finally:
        P.close()
    cover = np.zeros((n, n), dtype=np.int16)  # Morton order
    beg, end = t["box_begin"], t["box_end"]
    for b in range(len(beg)):
        for a in t["il_src"][t["il_ptr"][b]:t["il_ptr"][b + 1]]:
            cover[beg[b]:end[b], beg[a]:end[a]] += 1
    for li, b in enumerate(t["leaf_box"]):
        cols = t["nf_cols"][t["nf_colptr"][li]:t["nf_colptr"][li + 1]]
        cover[beg[b]:end[b], cols] += 1
    assert cover.min() == 1 and cover.max() == 1
    # pairs that need the subdivided rule lie in the near field
    c, _, _, h2 = oracle.geometry(v, f)
    perm = t["perm"]
    pos = np.empty(n, dtype=np.int64)
    pos[perm] = np.arange(n)
    near = np.zeros((n, n), dtype=bool)
    for li, b in enumerate(t["leaf_box"]):
        cols = t["nf_cols"][t["nf_colptr"][li]:t["nf_colptr"][li + 1]]
        near[np.ix_(perm[beg[b]:end[b]], perm[cols])] = True
    d2 = np.sum((c[:, None, :] - c[None, :, :]) ** 2, axis=2)
    special = d2 < 4.0 * h2[None, :]
    np.fill_diagonal(special, True)
    assert np.all(near[special])
    # spot-check the threshold against the oracle's own near-pair test
    rng = np.random.default_rng(3)
    for i, j in zip(rng.integers(0, n, 40), rng.integers(0, n, 40)):
        if i != j:
            assert oracle.is_near_pair(v, f, int(i), int(j)) == bool(special[i, j])
