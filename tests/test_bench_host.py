"""Host-side arithmetic of bench.py: the roofline's algorithmic bytes and
flops from the library's statistics, the committed traffic record (keyed to
the kernel source), and the clock sampler's parsing of nvidia-smi lines."""
import datetime
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _FakeProblem:
    def __init__(self, st):
        self._st = st

    def stats(self):
        return self._st


def _stats():
    st = types.SimpleNamespace()
    st.n_levels = 3
    st.level_rank = [0, 10, 4]
    st.level_m2l_pairs = [0, 7, 100]
    st.level_m2l_ops = [0, 2, 5]
    st.level_boxes = [1, 8, 64]
    st.level_cones = [1, 6, 1]
    return st


def test_m2l_bytes_and_flops():
    """The bench sums the library's per-level algorithmic M2L work over the
    levels in use (the per-level counts are checked against the closed form
    in the GPU tests)."""
    st = _stats()
    st.level_m2l_bytes = [0.0] * 32
    st.level_m2l_flops = [0.0] * 32
    st.level_m2l_bytes[1], st.level_m2l_bytes[2] = 1.5e6, 2.5e6
    st.level_m2l_flops[1], st.level_m2l_flops[2] = 3.0e9, 4.0e9
    P = _FakeProblem(st)
    assert bench._m2l_bytes(P) == 4000000
    assert bench._m2l_flops(P) == 7000000000


def test_traffic_record_is_keyed_to_the_kernel_source():
    args = types.SimpleNamespace(level=7, k=50.0, eps=1e-4)
    t = bench._m2l_traffic(args)
    assert t is None or t > 0  # None only if the kernel changed since the capture
    assert bench._m2l_traffic(types.SimpleNamespace(level=6, k=50.0, eps=1e-4)) is None


def test_clock_sampler_parses_the_timed_window(tmp_path):
    cs = bench.ClockSampler(0)
    cs.path = str(tmp_path / "clocks.csv")
    t0 = datetime.datetime(2026, 1, 1, 12, 0, 0)
    fmt = "%Y/%m/%d %H:%M:%S.%f"
    lines = []
    for i, (mhz, pc) in enumerate([(1000, "Not Active"), (2070, "Not Active"), (2055, "Active"),
                                   (2070, "Not Active"), (900, "Not Active")]):
        ts = (t0 + datetime.timedelta(seconds=i)).strftime(fmt)[:-3]
        lines.append("%s, 0, %d, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, %s" % (ts, mhz, pc))
    open(cs.path, "w").write("\n".join(lines) + "\n")
    cs.t_begin = t0 + datetime.timedelta(seconds=0.5)
    cs.t_end = t0 + datetime.timedelta(seconds=3.5)

    class _Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs.p = _Proc()
    cs.f = open(os.devnull, "w")
    out = cs.stop()
    assert out["samples"] == 3 and out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
