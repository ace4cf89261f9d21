"""Parity at the large size of the preconditioner study: unit icosphere
level 9 (5,242,880 triangles), k = 200 (kD = 400, about 13 elements per
wavelength), eps = 1e-4.  The tree has high-frequency levels 2-5 (up to 384
cones) and leaves at level 8; the FDA matvec of both forms agrees with 128
rows (seed 7) of the FP64 oracle's dense matvec to the FDA's eps as a
relative L2 error.  About 150 GB on the device while it runs.
"""
import numpy as np
import pytest

import oracle
from inputs import icosphere, complex_normal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if torch.cuda.get_device_properties(0).total_memory < 200e9:
        pytest.skip("needs about 150 GB of device memory")
    from paper_1403_4747_gb300 import build
    build.build()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_level9_both_precisions_against_oracle_rows():
    from paper_1403_4747_gb300 import FDAProblem, fda_set_precision
    v, f = icosphere(9)
    k = 200.0
    n = len(f)
    x = complex_normal(n, seed=1234)
    rows = np.random.default_rng(7).choice(n, 128, replace=False)
    ref = oracle.matvec(v, f, k, x, rows=rows)
    P = FDAProblem(v, f, k, precision=1)
    try:
        st = P.stats()
        assert max(st.level_cones[l] for l in range(st.n_levels)) >= 96
        xd = torch.from_numpy(x).cuda()
        e32 = _rel(P.apply(xd).cpu().numpy()[rows], ref)
        fda_set_precision(P.h, 0)
        e64 = _rel(P.apply(xd).cpu().numpy()[rows], ref)
    finally:
        P.close()
    print("level 9, k = 200: chosen %.3e, plain %.3e against %d oracle rows" % (e32, e64, len(rows)))
    assert e32 < 1e-4 and e64 < 1e-4
