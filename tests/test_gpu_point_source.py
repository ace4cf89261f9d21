"""Point-source scattering by the rigid unit sphere (the comparison of
Sec. 5.2, source at (-2, 0, 0)): the GPU right-hand side against the
oracle's (FP64, same formula: <= 1e-13), the GPU solution against the
oracle's dense-LU solution (<= 1e-3 at GMRES tol 1e-5) and against the
closed form under refinement."""
import numpy as np
import pytest

import oracle
from inputs import icosphere

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
SRC = np.array([-2.0, 0.0, 0.0])


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_4747_gb300 import build
    build.build()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("alpha_sign", [1.0, -1.0])
def test_point_source_rhs_matches_oracle(alpha_sign):
    from paper_1403_4747_gb300 import FDAProblem
    v, f = icosphere(3)
    src = np.array([SRC, [0.3, 1.7, -0.9]])
    P = FDAProblem(v, f, 5.0, mode=1, alpha_sign=alpha_sign)
    b = P.rhs_point_source(src).cpu().numpy()
    assert _rel(b, oracle.rhs_point_source(v, f, 5.0, src, alpha_sign=alpha_sign)) < 1e-13
    P.close()


@pytest.mark.parametrize("precision,alpha_sign", [(0, 1.0), (1, 1.0), (1, -1.0)])
def test_point_source_solution_matches_oracle(precision, alpha_sign):
    from paper_1403_4747_gb300 import FDAProblem
    k = 5.0
    v, f = icosphere(4)
    P = FDAProblem(v, f, k, precision=precision, alpha_sign=alpha_sign)
    b = P.rhs_point_source(SRC)
    u, info = P.solve(b, 1e-5)
    a = oracle.assemble(v, f, k, alpha_sign=alpha_sign)
    uo = oracle.lu_solve(a, oracle.rhs_point_source(v, f, k, [SRC], alpha_sign=alpha_sign)[0])
    assert _rel(u.cpu().numpy(), uo) < 1e-3
    P.close()


def test_point_source_converges_to_closed_form():
    from paper_1403_4747_gb300 import FDAProblem
    k = 5.0
    errs = []
    for L in (4, 5, 6):
        v, f = icosphere(L)
        P = FDAProblem(v, f, k, precision=1, alpha_sign=-1.0)
        u, info = P.solve(P.rhs_point_source(SRC), 1e-5)
        c = oracle.geometry(v, f)[0]
        cg = (c / np.linalg.norm(c, axis=1, keepdims=True)) @ (SRC / np.linalg.norm(SRC))
        ue = oracle.point_source_surface_field(k, 2.0, cg)
        errs.append(_rel(u.cpu().numpy(), ue))
        P.close()
    # first order in h: about halving per level
    assert errs[2] < errs[1] / 1.6 and errs[1] < errs[0] / 1.6
    assert errs[2] < 3e-3
