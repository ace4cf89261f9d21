"""Several meshes behind one operator application (fda_apply_batch): each
mesh's result against the FP64 oracle (relative L2 <= 1e-4, the FDA bar) and
against the same mesh's own handle (<= 1e-5: only the order of the float
atomics differs); the per-call CUDA graph is captured and replayed."""
import numpy as np
import pytest

import oracle
from inputs import icosphere, ellipsoid_from_icosphere, complex_normal, fibonacci_directions

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_4747_gb300 import build
    build.build()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


MESHES = [(icosphere(3), 5.0), (ellipsoid_from_icosphere(3), 6.0), (icosphere(4), 10.0),
          (ellipsoid_from_icosphere(4), 20.0)]


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_apply_matches_oracle_and_own_handles(precision):
    from paper_1403_4747_gb300 import FDABatch, FDAProblem
    meshes = [m for m, _ in MESHES]
    ks = [k for _, k in MESHES]
    B = FDABatch(meshes, ks, precision=precision, max_rhs=4)
    xs = [complex_normal(len(f), seed=20 + i, nrhs=5) for i, (v, f) in enumerate(meshes)]
    dx = [_dev(x) for x in xs]
    # 5 columns = chunks of 4 and 1; call 1 runs directly, call 2 captures, call 3 replays
    outs = [[y.cpu().numpy() for y in B.apply(dx)] for _ in range(3)]
    st = B.stats()
    assert st.nmesh == 4 and st.n_total == sum(len(f) for _, f in meshes)
    assert st.graph_fallback == 0 and st.graph_replays == 4
    for i, ((v, f), k) in enumerate(MESHES):
        for c in (1, 2):
            assert _rel(outs[c][i], outs[0][i]) < 1e-6
        ref = oracle.matvec(v, f, k, xs[i])
        assert _rel(outs[2][i], ref) < 1e-4
        P = FDAProblem(v, f, k, precision=precision, max_rhs=4)
        own = P.apply(dx[i]).cpu().numpy()
        P.close()
        assert _rel(outs[2][i], own) < 1e-5
    B.close()


def test_batch_mesh_handles_solve_and_graph_switch():
    from paper_1403_4747_gb300 import FDABatch, _lib
    meshes = [m for m, _ in MESHES[:2]]
    ks = [k for _, k in MESHES[:2]]
    B = FDABatch(meshes, ks, precision=1, max_rhs=2)
    # a mesh's handle serves the other entry points: right-hand side and solve
    h = B.mesh(0)
    n0 = len(meshes[0][1])
    b = torch.empty((1, n0), dtype=torch.complex128, device="cuda")
    _lib.fda_rhs_plane_wave(h, fibonacci_directions(1), b.data_ptr())
    x = torch.zeros_like(b)
    info, st = _lib.fda_solve(h, b.data_ptr(), x.data_ptr(), 1, 1e-5)
    assert st == 0 and info.rel_resid_fp64 <= 1e-5
    # switching one mesh to FP64 changes the graph key: a new graph, same results as FP64 alone
    xs = [complex_normal(len(f), seed=40 + i, nrhs=2) for i, (v, f) in enumerate(meshes)]
    dx = [_dev(x) for x in xs]
    for _ in range(2):
        y32 = [y.cpu().numpy() for y in B.apply(dx)]
    _lib.fda_set_precision(h, 0)
    for _ in range(3):
        y64 = [y.cpu().numpy() for y in B.apply(dx)]
    assert B.stats().graph_replays >= 3 and B.stats().graph_fallback == 0
    v, f = meshes[0]
    ref = oracle.matvec(v, f, ks[0], xs[0])
    assert _rel(y64[0], ref) < 1e-4 and _rel(y32[0], ref) < 1e-4
    assert _rel(y64[0], y32[0]) > 0  # mesh 0 really switched operator
    B.close()


def test_batch_rejects_bad_leading_dimension():
    from paper_1403_4747_gb300 import FDABatch, FDAError, FDA_ERR_ARG, _lib
    meshes = [m for m, _ in MESHES[:2]]
    B = FDABatch(meshes, [5.0, 6.0], precision=0)
    dx = [_dev(complex_normal(len(f), seed=1)) for v, f in meshes]
    with pytest.raises(FDAError) as e:
        _lib.fda_apply_batch(B.b, [x.data_ptr() for x in dx], [x.data_ptr() for x in dx], 1,
                             [len(meshes[0][1]), len(meshes[1][1]) - 1])
    assert e.value.status == FDA_ERR_ARG and "mesh 1" in str(e.value)
    B.close()
