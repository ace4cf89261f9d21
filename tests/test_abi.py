"""The C-ABI library builds, loads and exports every entry point that
include/fda_bem.h declares; argument validation that needs no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fda_bem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fda_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1403_4747_gb300 import build
    build.build()
    from paper_1403_4747_gb300 import _lib
    return _lib.load()


def test_header_declares_the_four_calls():
    names = _declared()
    for n in ("fda_build_tree", "fda_precompute_translations", "fda_apply", "fda_solve"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_config(lib):
    from paper_1403_4747_gb300 import fda_default_config
    c = fda_default_config()
    assert c.eps == 1e-4 and c.leaf_max == 64 and c.p_lf == 8 and c.restart == 100
    assert c.precision == 0 and c.mode == 0 and c.graphs == 1 and c.autotune == 1
    assert c.alpha_sign == -1.0


def test_tile_shape_override_null_handle(lib):
    assert lib.fda_set_tc_tiles(None, 0, 0, 0) == 1


@pytest.mark.parametrize("field,value", [("eps", 0.0), ("eps", 0.5), ("eps", 1e-9), ("leaf_max", 0), ("leaf_max", 65),
                                         ("p_lf", 2), ("precision", 3), ("mode", 7), ("restart", 0), ("restart", 256),
                                         ("rho_min", 1.0), ("graphs", 2), ("autotune", 3), ("precond", 2)])
def test_invalid_config_rejected_without_gpu(lib, field, value):
    from paper_1403_4747_gb300 import fda_default_config, fda_create, FDAError, FDA_ERR_ARG
    c = fda_default_config(**{field: value})
    with pytest.raises(FDAError) as e:
        fda_create(c)
    assert e.value.status == FDA_ERR_ARG


def test_null_handle_calls(lib):
    assert lib.fda_apply(None, None, None, 1, 1) == 1
    assert lib.fda_last_error(None) == b"null handle"
    lib.fda_destroy(None)


def test_batch_arguments_rejected_without_gpu(lib):
    import ctypes
    from paper_1403_4747_gb300 import fda_default_config, fda_create_batch, FDAError, FDA_ERR_ARG
    out = ctypes.c_void_p()
    assert lib.fda_create_batch(None, 0, ctypes.byref(out)) == FDA_ERR_ARG and not out.value
    assert lib.fda_create_batch(None, 65, ctypes.byref(out)) == FDA_ERR_ARG and not out.value
    with pytest.raises(FDAError) as e:
        fda_create_batch(fda_default_config(eps=0.0), 2)
    assert e.value.status == FDA_ERR_ARG
    assert lib.fda_apply_batch(None, None, None, 1, None) == FDA_ERR_ARG
    assert lib.fda_batch_mesh(None, 0) is None
    assert lib.fda_batch_last_error(None) == b"null batch"
    lib.fda_destroy_batch(None)


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of fda_config, fda_stats, fda_info and
    fda_batch_stats have the C structs' sizes and field offsets (gcc)."""
    import shutil
    import subprocess
    from paper_1403_4747_gb300 import _lib
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    structs = {"fda_config": _lib.fda_config, "fda_stats": _lib.fda_stats, "fda_info": _lib.fda_info,
               "fda_batch_stats": _lib.fda_batch_stats, "fda_sai_config": _lib.fda_sai_config,
               "fda_sai_report": _lib.fda_sai_report}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fda_bem.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for fname, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, fname, name, fname))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(out[name + "." + fname]) == getattr(cls, fname).offset, (name, fname)


def test_struct_sizes_reported_by_the_library(lib):
    from paper_1403_4747_gb300 import _lib
    classes = (_lib.fda_config, _lib.fda_info, _lib.fda_stats, _lib.fda_sai_config, _lib.fda_sai_report,
               _lib.fda_batch_stats)
    for which, cls in enumerate(classes):
        assert lib.fda_struct_size(which) == ctypes.sizeof(cls), cls.__name__
    assert lib.fda_struct_size(-1) == 0 and lib.fda_struct_size(6) == 0


def test_null_handle_calls_of_the_right_hand_sides_and_fields(lib):
    from paper_1403_4747_gb300 import FDA_ERR_ARG
    assert lib.fda_rhs_neumann(None, None, None, 1, 1) == FDA_ERR_ARG
    assert lib.fda_rhs_point_source(None, None, 1, None) == FDA_ERR_ARG
    assert lib.fda_far_field(None, None, None, None, 1, None) == FDA_ERR_ARG
    assert lib.fda_scattered_field(None, None, None, None, 1, None) == FDA_ERR_ARG
    assert lib.fda_scattered_field_fast(None, None, None, None, 1, None) == FDA_ERR_ARG
