"""fda_rhs_plane_wave_noalloc: the allocation-free right-hand side.

Some callers cannot let the library allocate device memory during a call
(real-time loops that forbid allocator calls, applications whose device
memory belongs to their own pool).  This entry point stages the incidence
directions in a fixed device array instead.  The test calls it through the
C ABI and compares it with the allocating fda_rhs_plane_wave on two calls in
a row (the second with other directions, so stale staging contents would
show), and checks that an oversized request is rejected.
"""
import numpy as np
import pytest

from inputs import icosphere, fibonacci_directions

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_rhs_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_4747_gb300 import build
    build.build()
    import paper_1403_4747_gb300 as F

    v, f = icosphere(3)
    n = len(f)
    h = F.fda_create(F.fda_default_config())
    try:
        F.fda_build_tree(h, v, f, 7.0)
        for dirs in (fibonacci_directions(5), fibonacci_directions(9)[3:]):
            m = dirs.shape[0]
            ref = torch.zeros((m, n), dtype=torch.complex128, device="cuda")
            got = torch.full((m, n), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
            F.fda_rhs_plane_wave(h, dirs, ref.data_ptr())
            F.fda_rhs_plane_wave_noalloc(h, dirs, got.data_ptr())
            torch.cuda.synchronize()
            r, g = ref.cpu().numpy(), got.cpu().numpy()
            assert np.all(np.isfinite(g))
            assert np.linalg.norm(g - r) <= 1e-12 * np.linalg.norm(r)
        too_many = np.tile(np.array([[0.0, 0.0, 1.0]]), (257, 1))
        out = torch.zeros((257, n), dtype=torch.complex128, device="cuda")
        with pytest.raises(F.FDAError) as e:
            F.fda_rhs_plane_wave_noalloc(h, too_many, out.data_ptr())
        assert e.value.status == F.FDA_ERR_ARG
    finally:
        F.fda_destroy(h)
