"""Host logic of the cone symmetry (the rotation invariance of Sec. 4.1.1):
the library's table maps every cone of a high-frequency level to a
representative on the +z face by a signed axis permutation, and offsets
related by those maps give identical M2L kernel matrices, which is what lets
them share one operator.  No GPU needed."""
import itertools

import numpy as np
import pytest


@pytest.fixture(scope="module")
def F():
    from paper_1403_4747_gb300 import build
    build.build()
    import paper_1403_4747_gb300 as F
    return F


def _centre(u, nc):
    face, rem = divmod(u, nc * nc)
    a, b = divmod(rem, nc)
    ax, s = divmod(face, 2)
    o0, o1 = (1, 2) if ax == 0 else ((0, 2) if ax == 1 else (0, 1))
    c = np.zeros(3, dtype=int)
    c[ax] = nc if s else -nc
    c[o0] = 2 * a + 1 - nc
    c[o1] = 2 * b + 1 - nc
    return c


def _cone(d, nc):
    """Cone of direction d: the face of the largest |component| (first axis
    on ties), then the cell of the two other coordinates over that one."""
    ad = np.abs(d)
    ax = 0
    if ad[1] > ad[ax]:
        ax = 1
    if ad[2] > ad[ax]:
        ax = 2
    s = 1 if d[ax] > 0 else 0
    o0, o1 = (1, 2) if ax == 0 else ((0, 2) if ax == 1 else (0, 1))
    a = int(np.floor((d[o0] / ad[ax] + 1.0) * 0.5 * nc))
    b = int(np.floor((d[o1] / ad[ax] + 1.0) * 0.5 * nc))
    a, b = min(max(a, 0), nc - 1), min(max(b, 0), nc - 1)
    return (2 * ax + s) * nc * nc + a * nc + b


def _opposite(u, nc):
    face, rem = divmod(u, nc * nc)
    a, b = divmod(rem, nc)
    return (face ^ 1) * nc * nc + (nc - 1 - a) * nc + (nc - 1 - b)


@pytest.mark.parametrize("nc", [1, 2, 3, 4])
def test_table_maps_representatives_onto_every_cone(F, nc):
    rep, g = F.fda_cone_symmetry_table(nc)
    n = 6 * nc * nc
    assert rep.shape == (n,) and g.shape == (n, 3, 3)
    for u in range(n):
        m = g[u]
        assert np.all(np.abs(m).sum(axis=0) == 1) and np.all(np.abs(m).sum(axis=1) == 1)
        assert np.array_equal(m.T @ m, np.eye(3, dtype=int))
        cr = _centre(rep[u], nc)
        assert cr[2] == nc and 0 <= cr[0] <= cr[1]
        assert np.array_equal(m @ cr, _centre(u, nc))
        v = _opposite(u, nc)
        assert rep[v] == rep[u] and np.array_equal(g[v], -m)
        assert _cone(_centre(u, nc).astype(float), nc) == u


@pytest.mark.parametrize("nc", [1, 2, 4])
def test_related_offsets_have_identical_kernel_matrices(F, nc):
    rep, g = F.fda_cone_symmetry_table(nc)
    rng = np.random.default_rng(3)
    eq = rng.uniform(-0.9, 0.9, size=(24, 3))
    # any fixed orthogonal frame per representative: the identity holds for all
    frames = {}
    for r in set(rep.tolist()):
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        frames[r] = q
    R = np.array([g[u] @ frames[rep[u]] for u in range(len(rep))], dtype=float)
    classes = {}
    noff = 0
    for d in itertools.product(range(-5, 6), repeat=3):
        d = np.array(d)
        if np.abs(d).max() < 2:
            continue
        noff += 1
        u, ub = _cone(d.astype(float), nc), _cone(-d.astype(float), nc)
        key = (rep[u], tuple(g[u].T @ d), tuple((g[u].T @ g[ub]).ravel()), rep[ub])
        x = eq @ R[u].T                       # target equivalent points
        y = d * 2.0 + eq @ R[ub].T            # source equivalent points, box width 2
        dist = np.linalg.norm(x[:, None, :] - y[None, :, :], axis=2)
        if key in classes:
            assert np.abs(dist - classes[key]).max() < 1e-12
        else:
            classes[key] = dist
    # the symmetry shares operators across most offsets
    assert len(classes) < 0.3 * noff
