"""STL import (host only, no GPU): binary and ASCII files written here from
known meshes read back to the same vertices and faces, merged in order of
first appearance; malformed files are refused with a message."""
import numpy as np
import pytest

import synth

from common import stl_facets as _facets, write_stl_ascii as _write_ascii, write_stl_binary as _write_binary


@pytest.fixture(scope="module")
def rc():
    import paper_2609_05467_gb300 as rc
    rc.load()
    return rc


def _expected(V, F):
    """Vertices in order of first appearance over the facets (brute force)."""
    seen, out_v, out_f = {}, [], []
    for t in _facets(V, F):
        row = []
        for v in t:
            key = tuple((v + np.float32(0.0)).tobytes()[i:i + 4] for i in (0, 4, 8))
            if key not in seen:
                seen[key] = len(out_v)
                out_v.append(v + np.float32(0.0))
            row.append(seen[key])
        out_f.append(row)
    return np.array(out_v, np.float32).reshape(-1, 3), np.array(out_f, np.int32).reshape(-1, 3)


@pytest.mark.parametrize("kind", ["binary", "ascii"])
@pytest.mark.parametrize("part", ["pocket", "prismatic", "icosphere"])
def test_round_trip(rc, tmp_path, kind, part):
    V, F = {"pocket": lambda: synth.pocket_block(2), "prismatic": lambda: synth.prismatic(h=6.0),
            "icosphere": lambda: synth.icosphere(10.0, 2)}[part]()
    path = str(tmp_path / ("p." + kind))
    (_write_binary if kind == "binary" else _write_ascii)(path, V, F)
    RV, RF = rc.rc_stl_read(path)
    EV, EF = _expected(V, F)
    assert np.array_equal(RV.view(np.uint32), EV.view(np.uint32)) and np.array_equal(RF, EF)
    # the same geometry as the original mesh (the generators share vertices)
    assert np.array_equal(RV[RF], np.asarray(V, np.float32)[F])
    if part != "prismatic":
        assert len(RV) == len(np.unique(np.asarray(V)[np.unique(F)], axis=0))


def test_binary_header_may_start_with_solid(rc, tmp_path):
    V, F = synth.cube(10.0, 0)
    path = str(tmp_path / "c.stl")
    _write_binary(path, V, F, header=b"solid but binary")
    RV, RF = rc.rc_stl_read(path)
    assert len(RF) == len(F) and np.array_equal(RV[RF], V[F])


def test_negative_zero_merges_with_zero(rc, tmp_path):
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [-0.0, 0, 0]], np.float32)
    F = np.array([[0, 1, 2], [3, 2, 1]], np.int32)
    path = str(tmp_path / "z.stl")
    _write_binary(path, V, F)
    RV, RF = rc.rc_stl_read(path)
    assert len(RV) == 3 and RF.tolist() == [[0, 1, 2], [0, 2, 1]]
    assert not np.signbit(RV).any()


def test_empty_and_malformed_files(rc, tmp_path):
    p = tmp_path / "empty.stl"
    _write_binary(str(p), np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32))
    V, F = rc.rc_stl_read(str(p))
    assert V.shape == (0, 3) and F.shape == (0, 3)
    V0, F0 = synth.cube(10.0, 0)
    good = tmp_path / "good.stl"
    _write_binary(str(good), V0, F0)
    data = good.read_bytes()
    cases = {
        "missing": None,
        "truncated_binary": data[:-7],
        "garbage": b"\x01\x02 hello",
        "ascii_truncated": b"solid x\n facet normal 0 0 1\n outer loop\n vertex 0 0 0\n vertex 1 0 0\n",
        "ascii_bad_number": b"solid x\n facet normal 0 0 1\n outer loop\n vertex 0 0 zz\n",
        "ascii_four_vertices": b"solid x\nfacet normal 0 0 1\nouter loop\nvertex 0 0 0\nvertex 1 0 0\n"
                               b"vertex 0 1 0\nvertex 1 1 0\nendloop\nendfacet\nendsolid x\n",
        "ascii_nan": b"solid x\nfacet normal 0 0 1\nouter loop\nvertex nan 0 0\nvertex 1 0 0\n"
                     b"vertex 0 1 0\nendloop\nendfacet\nendsolid x\n",
    }
    for name, blob in cases.items():
        path = tmp_path / (name + ".stl")
        if blob is not None:
            path.write_bytes(blob)
        with pytest.raises(rc.RcError) as ei:
            rc.rc_stl_read(str(path))
        assert ei.value.status == 1, name


def test_small_output_arrays_are_refused(rc, tmp_path):
    import ctypes
    V0, F0 = synth.cube(10.0, 1)
    path = str(tmp_path / "c.stl")
    _write_binary(path, V0, F0)
    L = rc.load()
    nV, T = ctypes.c_int64(), ctypes.c_int64()
    V = np.zeros((3, 3), np.float32)
    F = np.zeros((3, 3), np.int32)
    st = L.rc_stl_read(path.encode(), V.ctypes.data_as(ctypes.c_void_p), 3, F.ctypes.data_as(ctypes.c_void_p), 3,
                       ctypes.byref(nV), ctypes.byref(T))
    assert st == 1 and nV.value > 3 and T.value == len(F0)
