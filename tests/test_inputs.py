"""The synthetic meshes: sizes, closedness and outward orientation of the
icosphere, octahedral sphere and ellipsoid families, and the eight-mesh set
of the batch."""
import numpy as np
import pytest

from inputs import icosphere, octasphere, ellipsoid_from_icosphere, multi_mesh_set


def _check_closed_outward(v, f):
    n = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    c = v[f].mean(axis=1)
    assert (np.einsum("ij,ij->i", n, c) > 0).all()  # star-shaped about the origin: outward
    # every edge is shared by exactly two triangles, with opposite directions
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
    fwd = {tuple(x) for x in e}
    assert len(fwd) == len(e)
    assert all((b, a) in fwd for a, b in fwd)
    # divergence theorem: enclosed volume from the outward normals
    vol = np.einsum("ij,ij->i", v[f[:, 0]], np.cross(v[f[:, 1]], v[f[:, 2]])).sum() / 6.0
    assert vol > 0


@pytest.mark.parametrize("level", [0, 1, 3])
def test_octasphere(level):
    v, f = octasphere(level)
    assert len(f) == 8 * 4 ** level and len(v) == 4 * 4 ** level + 2
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0)
    _check_closed_outward(v, f)


@pytest.mark.parametrize("level", [0, 2])
def test_icosphere_and_ellipsoid(level):
    v, f = icosphere(level)
    assert len(f) == 20 * 4 ** level and len(v) == 10 * 4 ** level + 2
    _check_closed_outward(v, f)
    ve, fe = ellipsoid_from_icosphere(level)
    _check_closed_outward(ve, fe)


def test_octasphere_level_3_is_the_papers_coarsest_sphere():
    assert len(octasphere(3)[1]) == 512


def test_multi_mesh_set():
    mm = multi_mesh_set()
    assert [len(f) for _, f, _ in mm] == [20480, 20480, 81920, 81920, 81920, 327680, 327680, 327680]
    for v, f, k in mm:
        d = (v.max(axis=0) - v.min(axis=0)).max()
        assert 20 <= k * d <= 101
        # at least 10 elements per wavelength (mean edge length)
        h = np.linalg.norm(v[f[:, 1]] - v[f[:, 0]], axis=1).mean()
        assert 2 * np.pi / k / h >= 10
