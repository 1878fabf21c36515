"""Host logic of the benchmark that needs no GPU: the code-only hash that
decides whether a committed ncu summary belongs to the current traversal
sources, and the lookup of its per-ray figures."""
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


def test_committed_profile_lookup():
    # a committed summary is used only when it was taken on the current
    # traversal sources; otherwise the benchmark says why it has no figures
    for w in ("impeller", "prismatic"):
        prof = bench.committed_profile(w)
        assert "source" in prof
        if prof["source"].startswith("ncu, profiles/"):
            assert prof["dram_bytes_per_ray"] is not None and prof["dram_bytes_per_ray"] > 0
            assert 0 < prof["lanes_per_inst"] <= 32
