"""The C interface (no GPU needed): the library builds for sm_103a, loads, and
exports every entry point include/sbmt.h declares; argument errors come back
as codes before any device work."""
import ctypes
import os
import re

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


def test_struct_layouts_match_header():
    # sizes of the C structs on LP64 (int32/int64/double/pointer alignment)
    assert ctypes.sizeof(sb.sbmt_image) == 40
    assert ctypes.sizeof(sb.sbmt_params) == 56
    assert ctypes.sizeof(sb.sbmt_mesh_view) == 120


def test_null_arguments_are_rejected(lib):
    assert lib.mesh_create(None, 0, 0, None) == sb.SBMT_EINVAL
    assert lib.mesh_bitmap(None, None, None, None) == sb.SBMT_EINVAL
    assert lib.mesh_query(None, 1, 0, None) == sb.SBMT_EINVAL
    assert lib.mesh_release(None, 1) == sb.SBMT_EINVAL
    assert lib.mesh_destroy(None) == sb.SBMT_EINVAL
    assert isinstance(lib.sbmt_last_error(), bytes)
