"""C ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every function include/rtree.h declares with the struct layouts the
binding assumes.  No compute call is made here."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rtree.h")

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


@pytest.fixture(scope="module")
def lib():
    from paper_2309_16913_gb300 import build
    from paper_2309_16913_gb300 import rtree as rt
    build.build()
    return rt.load_library()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"RTREE_API[^;(]*?\b(rtree_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rtree_build", "rtree_range_select", "rtree_join", "rtree_free",
                     "rtree_result_free", "rtree_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    so = os.path.join(ROOT, "paper_2309_16913_gb300", "_build", "librtree.so")
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    extra = sorted(n for n in exported if n.startswith("rtree_") and n not in declared_functions())
    assert not extra, f"exported but not declared: {extra}"
    for n in declared_functions():
        assert hasattr(lib, n)


def test_struct_layouts_match_header(tmp_path):
    from paper_2309_16913_gb300 import rtree as rt
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "rtree.h"\n'
                   "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(rtree_config_t),"
                   " sizeof(rtree_select_opts_t), sizeof(rtree_info_t), offsetof(rtree_info_t, device_bytes),"
                   " offsetof(rtree_info_t, root_mbr), sizeof(rtree_server_config_t),"
                   " offsetof(rtree_server_config_t, max_batch_ids), sizeof(rtree_reply_t),"
                   " offsetof(rtree_reply_t, latency_us), sizeof(rtree_server_stats_t)); "
                   "printf(\"%zu %zu %zu %zu\\n\", offsetof(rtree_config_t, sort_children), sizeof(rtree_join_opts_t),"
                   " offsetof(rtree_info_t, sort_children), (size_t)RTREE_PRUNE_ON); "
                   "printf(\"%zu %zu\\n\", offsetof(rtree_select_opts_t, order), (size_t)RTREE_ORDER_HILBERT); "
                   "printf(\"%zu %zu %zu\\n\", sizeof(rtree_tune_result_t), offsetof(rtree_tune_result_t, ms_all),"
                   " offsetof(rtree_tune_result_t, order_all)); "
                   "printf(\"%zu %zu\\n\", sizeof(rtree_allocator_t), offsetof(rtree_allocator_t, ctx)); return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [C.sizeof(rt.rtree_config_t), C.sizeof(rt.rtree_select_opts_t), C.sizeof(rt.rtree_info_t),
            rt.rtree_info_t.device_bytes.offset, rt.rtree_info_t.root_mbr.offset,
            C.sizeof(rt.rtree_server_config_t), rt.rtree_server_config_t.max_batch_ids.offset,
            C.sizeof(rt.rtree_reply_t), rt.rtree_reply_t.latency_us.offset,
            C.sizeof(rt.rtree_server_stats_t), rt.rtree_config_t.sort_children.offset,
            C.sizeof(rt.rtree_join_opts_t), rt.rtree_info_t.sort_children.offset, rt.PRUNES["on"],
            rt.rtree_select_opts_t.order.offset, rt.ORDERS["hilbert"],
            C.sizeof(rt.rtree_tune_result_t), rt.rtree_tune_result_t.ms_all.offset,
            rt.rtree_tune_result_t.order_all.offset,
            C.sizeof(rt.rtree_allocator_t), rt.rtree_allocator_t.ctx.offset]
    assert got == want


def test_argument_errors_need_no_gpu(lib):
    from paper_2309_16913_gb300 import rtree as rt
    # NULL out-pointer and bad sizes are rejected before any CUDA call.
    assert lib.rtree_build(None, None, 0, None, None, None, None) == rt.RTREE_EINVAL
    assert b"out is NULL" in lib.rtree_last_error()
    out = C.c_void_p()
    assert lib.rtree_build(None, None, -1, None, None, None, C.byref(out)) == rt.RTREE_EINVAL
    cfg = rt.rtree_config_t()
    cfg.fanout = 3
    assert lib.rtree_build(None, None, 0, C.byref(cfg), None, None, C.byref(out)) == rt.RTREE_EINVAL
    assert b"fanout" in lib.rtree_last_error()
    assert lib.rtree_range_select(None, None, 0, None, None, C.byref(out)) == rt.RTREE_EINVAL
    assert lib.rtree_join(None, None, None, C.byref(out)) == rt.RTREE_EINVAL
    assert lib.rtree_join_ex(None, None, None, None, C.byref(out)) == rt.RTREE_EINVAL
    cfg = rt.rtree_config_t()
    cfg.sort_children = 2
    assert lib.rtree_build(None, None, 0, C.byref(cfg), None, None, C.byref(out)) == rt.RTREE_EINVAL
    assert b"sort_children" in lib.rtree_last_error()
    half = rt.rtree_allocator_t()  # an allocator needs both functions
    half.alloc = rt.ALLOC_FN(lambda n, s, c: 0)
    assert lib.rtree_build(None, None, 0, None, C.byref(half), None, C.byref(out)) == rt.RTREE_EINVAL
    assert b"allocator" in lib.rtree_last_error()
    assert lib.rtree_result_wait(None) == rt.RTREE_EINVAL
    assert lib.rtree_result_total(None) == 0
    lib.rtree_free(None)
    lib.rtree_result_free(None)
    assert rt.rtree_version().startswith("rtree-gb300")


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2309_16913_gb300 import rtree as rt
    with pytest.raises(RuntimeError, match="not built"):
        rt.load_library(str(tmp_path / "missing.so"))
