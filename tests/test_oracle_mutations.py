"""Planted mistakes: the pins of ``test_oracle_pins.py`` must catch a wrong
oracle, not only pass on the right one.  Each case below changes one step
of the oracle -- a sign, an index, an operand, a dropped term, a reversed
comparison or tie rule -- in a private copy (``oracle.c`` compiled into a
temporary directory with the oracle's own flags, or ``oracle/__init__.py``
executed as a separate module), runs the pins on that copy, and requires at
least one of them to fail.  The unchanged copy must pass them all, so a
failure is the planted mistake's and not the harness's.  The oracle's own
files are never written.  CPU only."""
import os
import subprocess
import types

import pytest

import test_oracle_frames as frame_pins
import test_oracle_pins as pins
import test_oracle_tool as tool_pins

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_C = os.path.join(ROOT, "oracle", "oracle.c")
ORACLE_PY = os.path.join(ROOT, "oracle", "__init__.py")

# (what is wrong, text in oracle.c, its replacement)
C_MUTATIONS = [
    ("splitmix64 shift", "z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;",
     "z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ULL;"),
    ("uniform counter drops the stream index", "uint64_t ctr = (uint64_t)(3 * i + k) * 0x9E3779B97F4A7C15ULL;",
     "uint64_t ctr = (uint64_t)(3 * i) * 0x9E3779B97F4A7C15ULL;"),
    ("normal from the transposed cross product", "cross3(e1, e2, c);", "cross3(e2, e1, c);"),
    ("area without the half", "if (area) area[f] = 0.5 * len;", "if (area) area[f] = len;"),
    ("centroid of two vertices", "centroid[3 * f + k] = (float)((A[k] + B[k] + C[k]) / 3.0);",
     "centroid[3 * f + k] = (float)((A[k] + B[k]) / 2.0);"),
    ("area CDF ignores the areas", "run += (int64_t)llround(area[f] / amax * 4294967296.0);",
     "run += 4294967296LL;"),
    ("square root of the area sampler dropped",
     "/* Osada et al. 2002: p = (1-s)A + s(1-u2)B + s*u2*C, s = sqrt(u1) */\n        double s = sqrt(u1);",
     "/* Osada et al. 2002: p = (1-s)A + s(1-u2)B + s*u2*C, s = sqrt(u1) */\n        double s = u1;"),
    ("direction index shifted", "double z = 1.0 - ((double)j + 0.5) / (double)N;",
     "double z = 1.0 - ((double)j + 1.0) / (double)N;"),
    ("wrong spiral angle", "const double ga = M_PI * (3.0 - sqrt(5.0));", "const double ga = M_PI * (3.0 - sqrt(3.0));"),
    ("tangent vectors swapped", "float x = t1[k] * h[0];\n        float y = t2[k] * h[1];",
     "float x = t2[k] * h[0];\n        float y = t1[k] * h[1];"),
    ("normal term takes the wrong component", "float z = n[k] * h[2];", "float z = n[k] * h[1];"),
    ("origin offset dropped", "double off = eps * (double)n[k];", "double off = 0.0 * eps * (double)n[k];"),
    ("origin offset against the normal", "o[k] = (float)((double)p[k] + off);", "o[k] = (float)((double)p[k] - off);"),
    ("edge function sign flipped", "cross3(b, ebc, w); E[0] = dot3(w, d);", "cross3(b, ebc, w); E[0] = -dot3(w, d);"),
    ("edge with a wrong vertex", "eca[k] = A[k] - C[k];", "eca[k] = A[k] - B[k];"),
    ("ambiguity band dropped", "const double band = OR_TAU * R;", "const double band = 0.0 * R;"),
    ("crossing behind the origin counted", "int ahead = (na > 0.0) == (nd > 0.0);",
     "int ahead = (na > 0.0) != (nd > 0.0);"),
    ("slab bounds not ordered", "if (a > b) { double t = a; a = b; b = t; }", "(void)0;"),
    ("last triangle of a leaf skipped", "for (int64_t i = nd->first; i < nd->first + nd->count; ++i) {",
     "for (int64_t i = nd->first; i + 1 < nd->first + nd->count; ++i) {"),
    ("visibility bits in reverse order", "if (r == OR_MISS) { brow[j >> 5] |= 1u << (j & 31); ++cnt; }",
     "if (r == OR_MISS) { brow[j >> 5] |= 1u << (31 - (j & 31)); ++cnt; }"),
    ("orthogonal eligibility reversed", "if (!(nd >= -J->par_tol)) continue;", "if (!(nd <= J->par_tol)) continue;"),
    ("fixed-point scale", "M[k] += (int64_t)llrint((double)d[k] * 1099511627776.0);",
     "M[k] += (int64_t)llrint((double)d[k] * 1048576.0);"),
    ("largest component compared with x only", "if (fabsf(d[2]) > fabsf(d[best])) best = 2;",
     "if (fabsf(d[2]) > fabsf(d[0])) best = 2;"),
    ("dominant axis by the smallest sum", "if (mk > md) dm = (int8_t)k;", "if (mk < md) dm = (int8_t)k;"),
]

# (what is wrong, text in oracle/__init__.py, its replacement)
PY_MUTATIONS = [
    ("machining axes without their negatives", "ax[2 * k + 1] = -R[:, k]", "ax[2 * k + 1] = R[:, k]"),
    ("mode-0 concentration from the z count",
     "conc[idx] = ac[idx, dom[idx]].astype(np.float64) / cnt[idx].astype(np.float64)",
     "conc[idx] = ac[idx, 2].astype(np.float64) / cnt[idx].astype(np.float64)"),
    ("accessibility ignores the weights", "num = float(np.sum(w * cnt.astype(np.float64)))",
     "num = float(np.sum(cnt.astype(np.float64)))"),
    ("accessibility over n N", "den = float(np.sum(w)) * N", "den = float(len(w)) * N"),
    ("shares over all points", "/ nc if nc else 0.0 for k in range(3)]", "/ n if nc else 0.0 for k in range(3)]"),
    ("mean concentration over all points", "mean_conc = float(csum) / (Q40 * nc) if nc else 0.0",
     "mean_conc = float(csum) / (Q40 * n) if nc else 0.0"),
    ("classification needs every indicator",
     'multi = (s["overall_access"] < t_acc) or (max(s["axis_share"]) < t_share) or \\',
     'multi = (s["overall_access"] < t_acc) and (max(s["axis_share"]) < t_share) and \\'),
    ("share threshold reversed", '(max(s["axis_share"]) < t_share)', '(max(s["axis_share"]) > t_share)'),
    ("concentration threshold reversed", '(s["mean_conc"] > t_conc)', '(s["mean_conc"] < t_conc)'),
    ("frame coordinates from the rows", "s = X[:, 0] * R[0, k] + X[:, 1] * R[1, k]\n        out[:, k] = s + X[:, 2] * R[2, k]",
     "s = X[:, 0] * R[k, 0] + X[:, 1] * R[k, 1]\n        out[:, k] = s + X[:, 2] * R[k, 2]"),
    ("travel directions swapped",
     "t[:, 2 * k] = (hi[k] - Pq[:, k]).astype(np.float32)\n        t[:, 2 * k + 1] = (Pq[:, k] - lo[k]).astype(np.float32)",
     "t[:, 2 * k] = (Pq[:, k] - lo[k]).astype(np.float32)\n        t[:, 2 * k + 1] = (hi[k] - Pq[:, k]).astype(np.float32)"),
    ("fixture plane tested against the wrong side", "on_hi = (np.abs(c - hi[k]) <= tol).all(1)",
     "on_hi = (np.abs(c - lo[k]) <= tol).all(1)"),
    ("tool length itself discarded", "(np.asarray(trav)[:, a] <= np.float32(tool_length))",
     "(np.asarray(trav)[:, a] < np.float32(tool_length))"),
    ("over-threshold and inaccessible swapped", "np.where(mask != 0, 1, 2)", "np.where(mask != 0, 2, 1)"),
    ("fixture faces not excluded", "cls[np.asarray(fixture)[np.asarray(face)]] = 3", "pass"),
    ("exact cover ties to the largest bitmask", "for S in range(1, 64):", "for S in range(63, 0, -1):"),
    ("greedy cover ties to the higher axis", "if c > bc:", "if c >= bc:"),
]

# (file under oracle/, what is wrong, text, its replacement): the automatic
# frame and the tool model, pinned by test_oracle_frames.py and
# test_oracle_tool.py
SUB_MUTATIONS = [
    ("frames.py", "second moment over 6", "S2 = ((A / 12.0)", "S2 = ((A / 6.0)"),
    ("frames.py", "vertex sum drops a vertex", "s = a + b + c\n    S0 = A.sum()", "s = a + b\n    S0 = A.sum()"),
    ("frames.py", "central moment adds the centroid term", "return S2 - S0 * np.outer(cen, cen), cen + r",
     "return S2 + S0 * np.outer(cen, cen), cen + r"),
    ("frames.py", "eigenvalues in ascending order", "order = np.argsort(-w, kind=\"stable\")",
     "order = np.argsort(w, kind=\"stable\")"),
    ("frames.py", "two equal largest eigenvalues accepted", "if not w[0] > 0.0 or (w[0] - w[1]) <= GAP * w[0] or",
     "if not w[0] > 0.0 or"),
    ("frames.py", "snapped sign rule reversed", "if w[k] < 0.0:", "if w[k] > 0.0:"),
    ("frames.py", "left-handed frame", "ec = _cross(ea, eb) if (col_a + 1) % 3 == col_b else _cross(eb, ea)",
     "ec = _cross(eb, ea) if (col_a + 1) % 3 == col_b else _cross(ea, eb)"),
    ("frames.py", "second column not made orthogonal",
     "eb = _unit([w[0] - d * ea[0], w[1] - d * ea[1], w[2] - d * ea[2]])", "eb = _unit(w)"),
    ("frames.py", "halves of the area quantisation rounded down", "(fl + (x - fl >= 0.5))", "(fl + (x - fl > 0.5))"),
    ("frames.py", "normal cell of a line depends on its sign", "sgn = np.where(nk < 0.0, -1.0, 1.0)",
     "sgn = np.where(nk < 0.0, 1.0, 1.0)"),
    ("frames.py", "cell components swapped", "u = (n[rows, (k + 1) % 3] * sgn) / m",
     "u = (n[rows, (k + 2) % 3] * sgn) / m"),
    ("frames.py", "normals frame with Z' and X' exchanged", "return frame_from(2, u1, 0, u2)",
     "return frame_from(0, u1, 2, u2)"),
    ("frames.py", "box volume of two extents", "return (ext[0] * ext[1]) * ext[2]", "return ext[0] * ext[1]"),
    ("frames.py", "box rotation not a rotation", "G[:, c] = cs * B[:, c] - sn * B[:, b]",
     "G[:, c] = cs * B[:, c] + sn * B[:, b]"),
    ("frames.py", "rotation angle halved", "sn = (2.0 * t) / den", "sn = t / den"),
    ("frames.py", "box search ties to the last", "if best is None or vol < best[3]:",
     "if best is None or vol <= best[3]:"),
    ("frames.py", "volume before flagged points", "keys = [(e[\"setups_exact\"], e[\"class_counts\"][1] + e[\"class_counts\"][2], c[\"volume\"], i)",
     "keys = [(e[\"setups_exact\"], c[\"volume\"], e[\"class_counts\"][1] + e[\"class_counts\"][2], i)"),
    ("tool.py", "ring angle's sine replaced", "math.sin(2.0 * math.pi * k / K)) for k in range(K)]",
     "math.cos(2.0 * math.pi * k / K)) for k in range(K)]"),
    ("tool.py", "basis vector sign", "v = (bb, sg + (ay * ay) * q, -ay)", "v = (bb, sg + (ay * ay) * q, ay)"),
    ("tool.py", "ring radius dropped", "rc, rs = radius * cs, radius * sn", "rc, rs = 0.0 * cs, 0.0 * sn"),
    ("tool.py", "eligibility without the tolerance", "elig = nd >= -parallel_tol", "elig = nd > parallel_tol"),
]

# the three pins that take a second or more run last
_SLOW = ("test_pair_matches_exact_rational_predicate", "test_pocket_block_matches_exact_visibility",
         "test_bvh_matches_brute_force")


def _pin_calls(module=pins):
    calls = []
    for name in sorted(vars(module), key=lambda nm: (nm in _SLOW, _SLOW.index(nm) if nm in _SLOW else 0, nm)):
        fn = getattr(module, name)
        if not name.startswith("test_") or not callable(fn):
            continue
        cases = [{}]
        for mark in getattr(fn, "pytestmark", []):
            if mark.name == "parametrize":
                argnames = [a.strip() for a in mark.args[0].split(",")]
                cases = [dict(zip(argnames, v if len(argnames) > 1 else (v,))) for v in mark.args[1]]
        calls += [(name, fn, kw) for kw in cases]
    return calls


def _oracle_copy(py=None, so=None):
    """The oracle package's module, executed afresh with one replacement in
    its Python source and/or bound to another compiled library."""
    src = open(ORACLE_PY).read()
    if py is not None:
        old, new = py
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    mod = types.ModuleType("oracle_copy")
    mod.__file__ = ORACLE_PY
    exec(compile(src, ORACLE_PY, "exec"), mod.__dict__)
    if so is not None:
        mod._SO = so
        mod.build = lambda force=False: so
    return mod


def _compiled_copy(tmp_path, old=None, new=None):
    src = open(ORACLE_C).read()
    if old is not None:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    c = tmp_path / "oracle_copy.c"
    c.write_text(src)
    so = str(tmp_path / "liboracle_copy.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-pthread", str(c), "-o", so, "-lm"])
    return so


def _submodule_copy(fname, old=None, new=None):
    """oracle/<fname> executed afresh, inside the real oracle package (its
    relative imports resolve there), with one replacement in its source."""
    path = os.path.join(ROOT, "oracle", fname)
    src = open(path).read()
    if old is not None:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    mod = types.ModuleType("oracle." + fname[:-3] + "_copy")
    mod.__file__ = path
    mod.__package__ = "oracle"
    exec(compile(src, path, "exec"), mod.__dict__)
    return mod


_SUB_PINS = {"frames.py": (frame_pins, "fr"), "tool.py": (tool_pins, "tool")}


def _first_failing_sub_pin(fname, mod):
    """Runs the pins of one oracle submodule with its module global bound to
    ``mod``; restores it afterwards."""
    pin_module, attr = _SUB_PINS[fname]
    saved = getattr(pin_module, attr)
    setattr(pin_module, attr, mod)
    try:
        for name, fn, kw in _pin_calls(pin_module):
            try:
                fn(**kw)
            except (AssertionError, pytest.fail.Exception) as e:   # a pin's own check failed
                return name, type(e).__name__
    finally:
        setattr(pin_module, attr, saved)
    return None


def _first_failing_pin(mod):
    for name, fn, kw in _pin_calls():
        try:
            fn(mod, **kw)
        except (AssertionError, pytest.fail.Exception) as e:   # a pin's own check failed
            return name, type(e).__name__
    return None


def test_unchanged_copy_passes_every_pin(tmp_path):
    assert _first_failing_pin(_oracle_copy(so=_compiled_copy(tmp_path))) is None
    assert _first_failing_pin(_oracle_copy(py=("Q40 = float(2 ** 40)", "Q40 = float(2 ** 40)"))) is None
    for fname in _SUB_PINS:
        assert _first_failing_sub_pin(fname, _submodule_copy(fname)) is None


@pytest.mark.parametrize("what,old,new", C_MUTATIONS, ids=[m[0] for m in C_MUTATIONS])
def test_planted_mistake_in_the_compiled_oracle_fails_a_pin(tmp_path, what, old, new):
    hit = _first_failing_pin(_oracle_copy(so=_compiled_copy(tmp_path, old, new)))
    assert hit is not None, "no pin catches: " + what


@pytest.mark.parametrize("what,old,new", PY_MUTATIONS, ids=[m[0] for m in PY_MUTATIONS])
def test_planted_mistake_in_the_python_oracle_fails_a_pin(what, old, new):
    hit = _first_failing_pin(_oracle_copy(py=(old, new)))
    assert hit is not None, "no pin catches: " + what


@pytest.mark.parametrize("fname,what,old,new", SUB_MUTATIONS, ids=[m[0][:-3] + ": " + m[1] for m in SUB_MUTATIONS])
def test_planted_mistake_in_the_frame_and_tool_oracle_fails_a_pin(fname, what, old, new):
    hit = _first_failing_sub_pin(fname, _submodule_copy(fname, old, new))
    assert hit is not None, "no pin catches: " + what
