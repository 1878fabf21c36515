"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every entry point that ``include/*.h`` declares, and its host-only logic
(parameters, direction table, classification, setup cover, argument
validation) agrees with the oracle.  No kernel is launched here."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rc():
    import paper_2609_05467_gb300 as rc
    rc.load()
    return rc


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(rc_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("rc_build_bvh", "rc_sample_points", "rc_hemisphere_cast", "rc_direction_variability",
                 "rc_orthogonal_cast", "rc_classify", "rc_min_setups"):
        assert must in names


def test_library_exports_every_declared_symbol(rc):
    L = ctypes.CDLL(rc.lib_path())
    missing = [n for n in sorted(declared_symbols()) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_declares_every_argument_type(rc):
    """Each entry point's ctypes prototype is set, with as many arguments
    as the header declares (so 64-bit sizes are never passed as C int)."""
    L = rc.load()
    txt = open(os.path.join(ROOT, "include", "rc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    for m in re.finditer(r"\b(rc_\w+)\s*\(([^)]*)\);", txt):
        name, args = m.group(1), m.group(2).strip()
        if name not in declared_symbols():
            continue
        n_args = 0 if args in ("", "void") else args.count(",") + 1
        fn = getattr(L, name)
        assert fn.argtypes is not None and len(fn.argtypes) == n_args, name


def test_header_compiles_as_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "rc.h"\nint main(void){rc_params p; return rc_params_default(&p);}\n')
    import subprocess
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only",
                           "-I", os.path.join(ROOT, "include"), str(src)])


def test_struct_layouts_match_header(rc, tmp_path):
    src = tmp_path / "s.c"
    src.write_text('#include <stdio.h>\n#include "rc.h"\nint main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu", '
                   'sizeof(rc_params), sizeof(rc_summary), sizeof(rc_setups), sizeof(rc_bvh_info), '
                   'sizeof(rc_part_result), sizeof(rc_server_config), sizeof(rc_request_result), '
                   'sizeof(rc_server_stats), sizeof(rc_frames));}\n')
    import subprocess
    exe = tmp_path / "s"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    assert [int(x) for x in out] == [ctypes.sizeof(rc.Params), ctypes.sizeof(rc.Summary),
                                     ctypes.sizeof(rc.Setups), ctypes.sizeof(rc.BvhInfo),
                                     ctypes.sizeof(rc.PartResult), ctypes.sizeof(rc.ServerConfig),
                                     ctypes.sizeof(rc.RequestResult), ctypes.sizeof(rc.ServerStats),
                                     ctypes.sizeof(rc.Frames)]


def test_params_default(rc):
    p = rc.rc_params_default()
    assert p.n_dirs == 256 and p.origin_offset == 1e-4 and list(p.frame) == [1, 0, 0, 0, 1, 0, 0, 0, 1]
    assert (p.t_acc, p.t_share, p.t_conc) == (0.60, 0.45, 0.41)
    assert p.parallel_tol == oracle.PARALLEL_TOL


def test_direction_table_bit_equal_to_oracle(rc):
    for N in (1, 32, 150, 256, 1024, 2048, 65536):
        _, h32 = oracle.direction_table(N)
        assert np.array_equal(rc.rc_direction_table(N).view(np.uint32), h32.view(np.uint32))
    with pytest.raises(rc.RcError):
        rc.rc_direction_table(0)


def test_classify_matches_oracle(rc):
    rng = np.random.default_rng(0)
    p = rc.rc_params_default()
    for _ in range(2000):
        s = rc.Summary()
        s.overall_access = float(rng.choice([rng.uniform(0, 1), 0.60]))
        sh = rng.dirichlet([1, 1, 1])
        for k in range(3):
            s.axis_share[k] = float(sh[k])
        s.mean_conc = float(rng.choice([rng.uniform(0.2, 0.7), 0.41]))
        d = {"overall_access": s.overall_access, "axis_share": list(s.axis_share), "mean_conc": s.mean_conc}
        assert rc.rc_classify(s, p) == oracle.classify(d)


def test_setup_cover_matches_oracle_brute_force(rc):
    rng = np.random.default_rng(1)
    for it in range(400):
        k = rng.integers(1, 12)
        masks = rng.integers(1, 64, size=k)
        if it % 3 == 0:
            masks = np.array([1 << rng.integers(0, 6) for _ in range(k)]) | (masks & rng.integers(0, 64))
            masks[masks == 0] = 1
        hist = np.zeros(64, np.int64)
        for m in masks:
            hist[m] += rng.integers(1, 5)
        pts = [m for m in range(64) for _ in range(hist[m])]
        out = rc.rc_setup_cover(hist)
        assert (out.setups_exact, out.chosen_exact) == oracle.setups_exact(pts)
        g, S = oracle.setups_greedy(pts)
        assert (out.setups_greedy, out.chosen_greedy) == (g, S)
    out = rc.rc_setup_cover(np.zeros(64, np.int64))
    assert out.setups_exact == 0 and out.setups_greedy == 0
    # the classic instance where greedy is not optimal
    hist = np.zeros(64, np.int64)
    for m in (0b011, 0b011, 0b101, 0b101, 0b010, 0b100):
        hist[m] += 1
    out = rc.rc_setup_cover(hist)
    assert out.setups_exact == 2 and out.setups_greedy == 3


def test_argument_validation_needs_no_gpu(rc):
    L = rc.load()
    h = ctypes.c_void_p()
    assert L.rc_build_bvh(None, 10, None, 10, None, ctypes.byref(h)) == 1
    assert b"NULL" in L.rc_last_error()
    assert L.rc_build_bvh(ctypes.c_void_p(16), 2, ctypes.c_void_p(16), 1, None, ctypes.byref(h)) == 1
    assert L.rc_build_bvh(ctypes.c_void_p(16), 3, ctypes.c_void_p(16), 0, None, ctypes.byref(h)) == 1
    p = rc.rc_params_default(n_dirs=0)
    assert L.rc_hemisphere_cast(ctypes.c_void_p(16), None, None, 1, ctypes.byref(p), None, None, None,
                                None) == 1
    assert L.rc_classify(None, None, None) == 1
    q = rc.rc_params_default(parallel_tol=-1e-3)
    assert L.rc_hemisphere_cast(ctypes.c_void_p(16), None, None, 1, ctypes.byref(q), None, None, None,
                                None) == 1 and b"parallel_tol" in L.rc_last_error()
    fr = rc.Frames()
    ok = rc.rc_params_default()
    assert L.rc_frame_candidates(None, ctypes.byref(ok), ctypes.byref(fr), None) == 1
    for k in (0, rc.RC_MAX_FRAMES + 1):
        fr.k = k
        assert L.rc_frame_select(ctypes.c_void_p(16), None, None, None, 0, ctypes.byref(ok), ctypes.byref(fr),
                                 None, None) == 1 and b"frames.k" in L.rc_last_error()
    z = rc.rc_params_default(frame=[1, 0, 0, 0, 0, 0, 0, 0, 1])          # Y' column is zero
    assert L.rc_hemisphere_cast(ctypes.c_void_p(16), None, None, 1, ctypes.byref(z), None, None, None,
                                None) == 1 and b"non-zero" in L.rc_last_error()
    fr.k = 1
    fr.frame[0][:] = [1, 0, 0, 0, 0, 0, 0, 0, 1]
    assert L.rc_frame_select(ctypes.c_void_p(16), None, None, None, 0, ctypes.byref(ok), ctypes.byref(fr),
                             None, None) == 1 and b"non-zero" in L.rc_last_error()
    fr.frame[0][:] = [1, 0, 0, 0, 1, 0, 0, 0, 1]
    fr.frame[0][4] = float("nan")
    assert L.rc_frame_select(ctypes.c_void_p(16), None, None, None, 0, ctypes.byref(ok), ctypes.byref(fr),
                             None, None) == 1 and b"finite" in L.rc_last_error()
    assert rc.rc_launch_count() == 0


def test_analysis_parameters_are_validated(rc):
    """tool_length (Section 3.3's reach threshold) takes any value >= 0 and
    +inf; the three classification thresholds take anything but NaN, which
    no comparison would decide; always_setups is 0 or 1.  A cast and the
    classification refuse anything else before touching the device."""
    L = rc.load()

    def cast_status(**kw):
        q = rc.rc_params_default(**kw)
        return L.rc_hemisphere_cast(ctypes.c_void_p(16), None, None, 1, ctypes.byref(q), None, None, None, None)

    nan, inf = float("nan"), float("inf")
    for kw, word in (({"tool_length": -1.0}, b"tool_length"), ({"tool_length": nan}, b"tool_length"),
                     ({"t_acc": nan}, b"NaN"), ({"t_share": nan}, b"NaN"), ({"t_conc": nan}, b"NaN"),
                     ({"always_setups": 2}, b"always_setups"), ({"always_setups": -1}, b"always_setups")):
        assert cast_status(**kw) == 1 and word in L.rc_last_error(), kw
    s = rc.Summary()
    label = ctypes.c_int32()
    for kw in ({"t_acc": nan}, {"t_share": nan}, {"t_conc": nan}):
        q = rc.rc_params_default(**kw)
        assert L.rc_classify(ctypes.byref(s), ctypes.byref(q), ctypes.byref(label)) == 1
        assert b"NaN" in L.rc_last_error()
    # accepted limits: classification runs on the host and gives the label the
    # oracle's rule gives
    s.overall_access, s.mean_conc = 0.5, 0.3
    for k in range(3):
        s.axis_share[k] = 1.0 / 3.0
    for kw in ({"tool_length": 0.0}, {"tool_length": inf}, {"t_acc": -inf, "t_share": -inf, "t_conc": inf},
               {"t_acc": inf}, {"always_setups": 1}):
        q = rc.rc_params_default(**kw)
        assert L.rc_classify(ctypes.byref(s), ctypes.byref(q), ctypes.byref(label)) == 0
        d = {"overall_access": s.overall_access, "axis_share": list(s.axis_share), "mean_conc": s.mean_conc}
        assert label.value == oracle.classify(d, t_acc=q.t_acc, t_share=q.t_share, t_conc=q.t_conc), kw
    assert rc.rc_launch_count() == 0


def test_product_path_does_not_touch_the_oracle():
    """The library package imports nothing from oracle/ and its sources name
    no oracle file."""
    pkg = os.path.join(ROOT, "paper_2609_05467_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            txt = open(f).read()
            assert "import oracle" not in txt and "from oracle" not in txt and "oracle.c" not in txt, f
