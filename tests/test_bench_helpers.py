"""Host-side helpers of bench.py that decide which committed ncu figures a run
may use: the source stamp (kernel sources hashed without their comments) and
the configuration match (fanout and node layout) of a summary line."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_strip_comments_keeps_code_and_literals():
    src = ('int a = 1; // trailing\n'
           '/* block\n   over lines */ int b = 2;\n'
           'const char *s = "not // a comment /* nor this */";\n'
           "char c = '/'; char d = '\\''; char e = '\"';\n"
           '\n'
           'float f = x / y * z; /**/ int g;\n')
    got = bench.strip_comments(src)
    assert got.splitlines() == [
        "int a = 1;",
        " int b = 2;",
        'const char *s = "not // a comment /* nor this */";',
        "char c = '/'; char d = '\\''; char e = '\"';",
        "float f = x / y * z;  int g;",
    ]


def test_stamp_ignores_comments_but_not_code():
    files = {"k.cu": "__global__ void k() { int x = 1; }  // first\n"}
    base = bench.source_sha(["k.cu"], read=files.get)
    files["k.cu"] = "// a new note\n__global__ void k() { int x = 1; }  /* reworded */\n\n"
    assert bench.source_sha(["k.cu"], read=files.get) == base
    files["k.cu"] = "__global__ void k() { int x = 2; }\n"
    assert bench.source_sha(["k.cu"], read=files.get) != base


def test_config_match():
    line = {"kernel": "select_desc", "fanout": "64", "layout": "aos"}
    assert bench.config_matches(line, 64, "aos")
    assert not bench.config_matches(line, 128, "aos")
    assert not bench.config_matches(line, 64, "lohi")
    assert bench.config_matches(line, None, None)
    assert bench.config_matches({"kernel": "join_count", "fanout": "32"}, 32, "soa")  # no layout key
    assert bench.config_matches({"kernel": "k"}, 16, "soa")  # neither key: serves any run
