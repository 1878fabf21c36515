"""Host logic of the benchmark that needs no GPU: the code-only hash that
decides whether the committed DRAM traffic belongs to the current traversal
sources, and the lookup of that traffic."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_only_drops_comments_and_blank_lines():
    src = 'int a = 1; // note\n\n/* block\n comment */ float b = 2.0f;  \nconst char* s = "a // b /* c */";\n'
    assert bench._code_only(src) == 'int a = 1;\n float b = 2.0f;\nconst char* s = "a // b /* c */";'


def test_code_only_keeps_character_literals_and_escapes():
    src = "char q = '\\'';  // quote\nchar r = '/'; char t = '\"';\n"
    out = bench._code_only(src)
    assert "quote" not in out and "'\\''" in out and "'/'" in out and "'\"'" in out


def test_comment_edits_keep_the_hash_code_edits_change_it():
    a = "int f(int x) { return x + 1; }  // one\n"
    b = "// a new comment\nint f(int x) { return x + 1; }  // two\n\n"
    c = "int f(int x) { return x + 2; }\n"
    assert bench._code_only(a) == bench._code_only(b) != bench._code_only(c)


def test_committed_traffic_matches_the_current_sources():
    # the committed profile was taken on the current traversal sources, so
    # the benchmark reports its DRAM bytes (a source edit would make it stale)
    traffic, src = bench.committed_traffic("prismatic")
    assert src in ("ncu", "stale")
    if src == "ncu":
        assert traffic > 0
