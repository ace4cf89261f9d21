"""Plain construction of the octree, interaction lists and near-field sets
from the rules of Sec. 3.3 Step 1 (TEST INFRASTRUCTURE; numpy, no GPU):

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
"""
import numpy as np

MAXD = 20


def reference_tree(v, f, k, leaf_max=64, rho_min=2.2):
    """Boxes per level as {cell: sorted caller indices}, leaf flags, and the
    level parameters (width, high-frequency flag, rho)."""
    c = np.mean(v[f], axis=1)
    lo, hi = c.min(axis=0), c.max(axis=0)
    ext = float(np.max(hi - lo))
    W = ext * (1.0 + 1e-6) if ext > 0 else 1.0
    root = 0.5 * (lo + hi) - 0.5 * W
    q = np.floor((c - root) * ((1 << MAXD) / W)).astype(np.int64)
    q = np.clip(q, 0, (1 << MAXD) - 1)
    lam = 2.0 * np.pi / k
    active = np.ones(len(f), dtype=bool)
    levels = []
    for l in range(MAXD + 1):
        idx = np.nonzero(active)[0]
        if len(idx) == 0:
            break
        w = W / (1 << l)
        hf = w >= lam
        cells = q[idx] >> (MAXD - l)
        boxes = {}
        for i, cc in zip(idx, map(tuple, cells)):
            boxes.setdefault(cc, []).append(int(i))
        leaf = {}
        for cc, el in boxes.items():
            leaf[cc] = (l == MAXD) or ((not hf) and len(el) <= leaf_max)
            if leaf[cc]:
                active[el] = False
        rho = max(rho_min, w / lam) if hf else 0.0
        levels.append({"boxes": {cc: sorted(el) for cc, el in boxes.items()}, "leaf": leaf, "hf": hf, "rho": rho,
                       "w": w, "root": root})
    return levels


def is_near(L, d):
    d = np.asarray(d)
    if np.max(np.abs(d)) <= 1:
        return True
    return bool(L["hf"] and np.sqrt(np.sum(d * d)) < L["rho"])


def reference_lists(levels):
    """Interaction lists {(level, cell): set of cells} and near-field element
    sets {(level, cell) of a leaf: set of caller indices}."""
    il = {}
    for l in range(1, len(levels)):
        L, Lp = levels[l], levels[l - 1]
        cells = list(L["boxes"])
        for b in cells:
            pb = tuple(np.array(b) >> 1)
            s = set()
            for a in cells:
                pa = tuple(np.array(a) >> 1)
                if not is_near(Lp, np.array(pa) - np.array(pb)):
                    continue
                if is_near(L, np.array(a) - np.array(b)):
                    continue
                s.add(a)
            il[(l, b)] = s
    near = {}
    for lb, L in enumerate(levels):
        for b, isleaf in L["leaf"].items():
            if not isleaf:
                continue
            s = set()
            for l in range(lb + 1):
                anc = np.array(b) >> (lb - l)
                for x, xleaf in levels[l]["leaf"].items():
                    if xleaf and is_near(levels[l], np.array(x) - anc):
                        s.update(levels[l]["boxes"][x])
            for x, xleaf in L["leaf"].items():
                if not xleaf and is_near(L, np.array(x) - np.array(b)):
                    s.update(L["boxes"][x])
            near[(lb, b)] = s
    return il, near
