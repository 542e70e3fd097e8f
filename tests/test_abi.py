"""CPU-side checks of the boundary: the shared library loads, exports every
symbol include/hfs.h declares, the ctypes structure matches the C layout,
and host-side validation errors come back as status codes (no device work)."""
import ctypes
import os
import re

import pytest

from paper_1007_3470_gb300 import hfs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_1007_3470_gb300 import build as B
    B.build()
    return hfs.lib()


def _declared():
    import glob
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        names |= set(re.findall(r"\b(hfs_[a-z_0-9]+)\s*\(", open(h).read()))
    return sorted(names)


def test_header_declarations_match_binding():
    from paper_1007_3470_gb300 import fno
    assert sorted(set(hfs.EXPORTS) | set(fno.EXPORTS)) == _declared()


def test_library_exports_every_symbol(built):
    for name in _declared():
        assert hasattr(built, name), name


def test_error_strings(built):
    for code in range(10):
        assert hfs.hfs_error_string(code)
    assert hfs.hfs_error_string(0) == "ok"


def test_instance_struct_layout():
    # int32 n[3] (12) + pad (4) + 3+3 doubles + mu + (int32 + pad) + w0 + 3 + 3 + eps + (int32+pad) + vi_k + sigma
    assert ctypes.sizeof(hfs.hfs_instance) == 12 + 4 + 48 + 8 + 8 + 8 + 24 + 24 + 8 + 8 + 8 + 8
    assert hfs.hfs_instance.lo.offset == 16


def test_invalid_arguments_rejected_on_host(built):
    L = built
    h = ctypes.c_void_p()
    arr = hfs.make_instances([{"n": [100], "a": [-1.0], "b": [1.0]}])
    # non power of two -> unsupported, before any device call
    assert L.hfs_create(ctypes.byref(h), 1, hfs.HFS_C64, arr, 1) == 2
    arr = hfs.make_instances([{"n": [256], "a": [1.0], "b": [-1.0]}])
    assert L.hfs_create(ctypes.byref(h), 1, hfs.HFS_C64, arr, 1) == 1
    arr = hfs.make_instances([{"n": [256], "a": [-1.0], "b": [1.0], "mu": 0.0}])
    assert L.hfs_create(ctypes.byref(h), 1, hfs.HFS_C64, arr, 1) == 1
    assert L.hfs_create(ctypes.byref(h), 2, hfs.HFS_C64, arr, 1) == 2
    assert L.hfs_create(None, 1, hfs.HFS_C64, arr, 1) == 1
    # 1D grids are powers of two from 128 to 4096
    for n in (64, 8192):
        arr = hfs.make_instances([{"n": [n], "a": [-1.0], "b": [1.0]}])
        assert L.hfs_create(ctypes.byref(h), 1, hfs.HFS_C64, arr, 1) == 2
    ok = {"n": [256], "a": [-1.0], "b": [1.0]}
    arr = hfs.make_instances([ok])
    assert L.hfs_create(ctypes.byref(h), 1, 7, arr, 1) == 1                # precision
    assert L.hfs_create(ctypes.byref(h), 1, hfs.HFS_C64, arr, 0) == 1      # empty batch
    for bad in ({"omega_law": 4}, {"vi_kind": 3}):
        arr = hfs.make_instances([dict(ok, **bad)])
        assert L.hfs_create(ctypes.byref(h), 1, hfs.HFS_C64, arr, 1) == 1
    # 3D: one instance per context, centred boxes
    d3 = {"n": [32, 32, 32], "a": [-6.0] * 3, "b": [6.0] * 3}
    arr = hfs.make_instances([d3, d3])
    assert L.hfs_create(ctypes.byref(h), 3, hfs.HFS_C64, arr, 2) == 2
    arr = hfs.make_instances([dict(d3, a=[-5.0, -6.0, -6.0], b=[7.0, 6.0, 6.0])])
    assert L.hfs_create(ctypes.byref(h), 3, hfs.HFS_C64, arr, 1) == 2
