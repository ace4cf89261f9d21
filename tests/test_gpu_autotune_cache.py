"""The autotune cache of the tensor-core translation batches: the first
setup times every batch and appends one line per batch; a second setup of
the same problem takes every shape from the file without timing and gives
the same operator; a path that cannot be written only disables the cache."""
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
    from paper_1403_4747_gb300 import build
    build.build()


def test_autotune_cache_round_trip(tmp_path):
    from paper_1403_4747_gb300 import FDAProblem
    v, f = icosphere(4)
    k = 20.0
    path = str(tmp_path / "tune.txt")
    x = torch.from_numpy(complex_normal(len(f), seed=4)).cuda()
    P1 = FDAProblem(v, f, k, precision=1, autotune_cache=path)
    s1 = P1.stats()
    assert s1.autotune_timed > 0 and s1.autotune_cached == 0
    lines = open(path).read().splitlines()
    assert len(lines) == s1.autotune_timed
    y1 = P1.apply(x).cpu().numpy()
    P1.close()
    P2 = FDAProblem(v, f, k, precision=1, autotune_cache=path)
    s2 = P2.stats()
    assert s2.autotune_cached == s1.autotune_timed and s2.autotune_timed == 0
    y2 = P2.apply(x).cpu().numpy()
    P2.close()
    assert open(path).read().splitlines() == lines  # nothing new appended
    assert np.linalg.norm(y2 - y1) <= 1e-6 * np.linalg.norm(y1)
    ref = oracle.matvec(v, f, k, x.cpu().numpy())
    assert np.linalg.norm(y2 - ref) <= 1e-4 * np.linalg.norm(ref)


def test_unwritable_autotune_cache_is_ignored(tmp_path):
    from paper_1403_4747_gb300 import FDAProblem
    v, f = icosphere(4)
    P = FDAProblem(v, f, 20.0, precision=1, autotune_cache=str(tmp_path / "missing_dir" / "tune.txt"))
    s = P.stats()
    assert s.autotune_timed > 0 and s.autotune_cached == 0
    P.close()
