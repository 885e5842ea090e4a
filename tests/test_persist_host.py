"""rtree_load rejects what is not a tree file before any device work, so
these run without a GPU (the library is built for sm_103a and loaded)."""
import ctypes as C
import os
import shutil
import struct

import pytest

from persist_util import HEADER_BYTES, O_HEADER_HASH, file_hash

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


@pytest.fixture(scope="module")
def rt():
    from paper_2309_16913_gb300 import build
    from paper_2309_16913_gb300 import rtree as rt
    build.build()
    rt.load_library()
    return rt


def load_status(rt, path):
    lib = rt.load_library()
    out = C.c_void_p()
    st = lib.rtree_load(os.fsencode(str(path)), -1, None, C.byref(out))
    assert not out.value
    return st, lib.rtree_last_error().decode()


def test_missing_file(rt, tmp_path):
    st, msg = load_status(rt, tmp_path / "none.rtree")
    assert st == rt.RTREE_EIO and "cannot open" in msg


def test_short_and_foreign_files(rt, tmp_path):
    p = tmp_path / "empty.rtree"
    p.write_bytes(b"")
    assert load_status(rt, p) == (rt.RTREE_EINVAL, "rtree_load: file too short for a tree header (0 bytes)")
    p.write_bytes(os.urandom(4096))
    st, msg = load_status(rt, p)
    assert st == rt.RTREE_EINVAL and "magic" in msg


def test_header_checks(rt, tmp_path):
    p = tmp_path / "h.rtree"
    hdr = bytearray(HEADER_BYTES)
    hdr[0:8] = b"RTREEGB3"
    struct.pack_into("<II", hdr, 8, 1, 0x01020304)
    p.write_bytes(bytes(hdr))
    st, msg = load_status(rt, p)  # header checksum not set
    assert st == rt.RTREE_EINVAL and "header checksum" in msg
    struct.pack_into("<Q", hdr, O_HEADER_HASH, file_hash(bytes(hdr)))
    p.write_bytes(bytes(hdr))
    st, msg = load_status(rt, p)  # sealed, but fanout 0 is not a tree
    assert st == rt.RTREE_EINVAL and "fanout" in msg
    struct.pack_into("<I", hdr, 8, 2)
    p.write_bytes(bytes(hdr))
    st, msg = load_status(rt, p)
    assert st == rt.RTREE_EINVAL and "version 2" in msg
    struct.pack_into("<II", hdr, 8, 1, 0x04030201)
    p.write_bytes(bytes(hdr))
    st, msg = load_status(rt, p)
    assert st == rt.RTREE_EINVAL and "byte order" in msg


def test_save_argument_errors(rt):
    lib = rt.load_library()
    assert lib.rtree_save(None, b"/nonexistent", None) == rt.RTREE_EINVAL
    assert lib.rtree_load(None, -1, None, None) == rt.RTREE_EINVAL
