"""The C interface (no GPU needed): the library builds for sm_103a, loads, and
exports every entry point include/sbmt.h declares; argument errors come back
as codes before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2602_19474_gb300 as sb

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "sbmt.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    sb.build_library()
    return sb.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"mesh_create", "mesh_bitmap", "mesh_batch", "mesh_query", "mesh_release", "mesh_destroy"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layouts_match_header(tmp_path):
    # every field's offset and every struct's size, as the C compiler lays
    # out include/sbmt.h, against the ctypes declarations of the binding
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = (sb.sbmt_image, sb.sbmt_params, sb.sbmt_mesh_view, sb.sbmt_quality, sb.sbmt_pre_info, sb.sbmt_heat_params,
               sb.sbmt_server_config, sb.sbmt_request_info, sb.sbmt_server_stats)
    lines = []
    for st in structs:
        n = st.__name__
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (n, n))
        for f, _ in st._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (n, f, n, f))
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include "sbmt.h"\nint main(void) {\n%s\nreturn 0;\n}\n' % "\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True)
               .stdout.splitlines())
    for st in structs:
        n = st.__name__
        assert int(got[n]) == ctypes.sizeof(st), n
        for f, _ in st._fields_:
            assert int(got[n + "." + f]) == getattr(st, f).offset, (n, f)


def test_null_arguments_are_rejected(lib):
    assert lib.mesh_create(None, 0, 0, None) == sb.SBMT_EINVAL
    assert lib.mesh_bitmap(None, None, None, None) == sb.SBMT_EINVAL
    assert lib.mesh_query(None, 1, 0, None) == sb.SBMT_EINVAL
    assert lib.mesh_release(None, 1) == sb.SBMT_EINVAL
    assert lib.mesh_destroy(None) == sb.SBMT_EINVAL
    assert lib.mesh_preprocess(None, None, None, None) == sb.SBMT_EINVAL
    assert lib.mesh_preprocess_info(None, 1, None) == sb.SBMT_EINVAL
    assert lib.mesh_retriangulate(None, None, 1, None) == sb.SBMT_EINVAL
    assert lib.mesh_heat(None, 1, None, None, None, None) == sb.SBMT_EINVAL
    assert lib.mesh_autotune(None, None, 0, None, 1, 1) == sb.SBMT_EINVAL
    assert lib.mesh_tuning(None, None, 0, None, 1, None) == sb.SBMT_EINVAL
    assert lib.mesh_set_tuning(None, None, 0, None, 1, None) == sb.SBMT_EINVAL
    assert lib.mesh_footprint(None, 1, None) == sb.SBMT_EINVAL
    assert lib.server_create(None, 0, None) == sb.SBMT_EINVAL
    assert lib.server_submit(None, None, None, None) == sb.SBMT_EINVAL
    assert lib.server_wait(None, 1, 0, None, None) == sb.SBMT_EINVAL
    assert lib.server_destroy(None) == sb.SBMT_EINVAL
    assert isinstance(lib.sbmt_last_error(), bytes)


def test_requests_are_checked_without_a_device(lib):
    # mesh_check (which server_submit runs first) needs no GPU
    img = np.zeros((4, 5), np.uint8)
    assert sb.mesh_check(img, 2) == sb.SBMT_OK
    assert sb.mesh_check(img, 3) == sb.SBMT_EINVAL  # odd h_num: outside the degeneracy-free class
    assert sb.mesh_check(img, 2, 2) == sb.SBMT_EINVAL  # even h_den
    assert sb.mesh_check(np.zeros((4, 32769), np.uint8), 2) == sb.SBMT_EINVAL
    im, _ = sb._image(img)
    pr = sb._params(2, mode=sb.SBMT_PREPROCESS)
    assert lib.mesh_check(ctypes.byref(im), ctypes.byref(pr)) == sb.SBMT_EPROTO
    # the pre-count reservation grows with the image and shrinks with h
    assert sb.mesh_bound(np.zeros((100, 100), np.uint8), 2) < sb.mesh_bound(np.zeros((200, 200), np.uint8), 2)
    assert sb.mesh_bound(np.zeros((100, 100), np.uint8), 8) < sb.mesh_bound(np.zeros((100, 100), np.uint8), 2)


def test_mesh_import_checks_the_arrays_before_the_context(lib):
    """mesh_import's array checks are host logic: each bad mesh is refused
    with its own reason before the (null) context is looked at."""
    def call(xy, tri, nv=None, nt=None):
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        rc = lib.mesh_import(None, xy.ctypes.data, len(xy) if nv is None else nv, tri.ctypes.data,
                             len(tri) if nt is None else nt, None)
        return rc, lib.sbmt_last_error().decode()

    xy = [[0.0, 0.0], [2.0, 0.0], [0.0, 2.0]]
    assert call(xy, [[0, 1, 2]]) == (sb.SBMT_EINVAL, "null ctx or out")
    assert "vertex id out of range" in call(xy, [[0, 1, 3]])[1]
    assert "vertex id out of range" in call(xy, [[0, -1, 2]])[1]
    assert "repeated vertex id" in call(xy, [[0, 1, 1]])[1]
    assert "coordinate" in call([[0.0, 0.0], [np.nan, 0.0], [0.0, 2.0]], [[0, 1, 2]])[1]
    assert "coordinate" in call([[0.0, 0.0], [2.0, np.inf], [0.0, 2.0]], [[0, 1, 2]])[1]
    assert "coordinate" in call([[0.0, 0.0], [2.0 ** 25, 0.0], [0.0, 2.0]], [[0, 1, 2]])[1]
    assert "mesh of" in call(xy[:2], [[0, 1, 2]], nv=2)[1]
    assert "mesh of" in call(xy, [[0, 1, 2]], nt=0)[1]
    assert lib.mesh_import(None, None, 3, None, 1, None) == sb.SBMT_EINVAL
