"""FP64 CPU oracle for hemispherical ray-casting -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library
(``paper_2609_05467_gb300``) never does, and the two share no code: the C
part (``oracle.c``) is compiled on its own by :func:`build` with
``-ffp-contract=off``, and the Python part here uses numpy only.

Per-ray work (the occlusion predicate, brute force or a plain CPU BVH, the
hemisphere and orthogonal casts, the per-point direction sums) is in C for
speed; the part-level logic of Section 3.3 (indicators, classification,
fixture faces, face classes, setup covers) is plain numpy / Python below.

Every function cites the passage of the paper it follows; the readings taken
where the paper is silent are listed at the top of ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

MISS, HIT, AMB = 0, 1, 2
TAU = 1e-9
PARALLEL_TOL = 1e-4     # orthogonal eligibility tolerance on n . a (reading R8 of oracle.c)


def build(force=False):
    """Compile ``oracle.c`` into ``liboracle.so`` next to it (gcc, -O2,
    -ffp-contract=off so no multiply-add is fused)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
                           "-fno-fast-math", "-fPIC", "-shared", "-pthread", src, "-o", tmp, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            lib.or_splitmix64.argtypes = [ctypes.c_uint64]
            lib.or_splitmix64.restype = ctypes.c_uint64
            lib.or_face_prep.argtypes = [P, P, i64, P, P, P]
            lib.or_sample_area.argtypes = [P, P, i64, i64, ctypes.c_uint64, P, P, P]
            lib.or_sample_area.restype = ctypes.c_int
            lib.or_sample_on_faces.argtypes = [P, P, i64, i64, ctypes.c_uint64, ctypes.c_int, P, P, P]
            lib.or_sample_on_faces.restype = i64
            lib.or_direction_table.argtypes = [i32, P, P]
            lib.or_ray_dirs.argtypes = [P, P, i32, P]
            lib.or_ray_origin.argtypes = [P, P, f64, P]
            lib.or_pair_f32.argtypes = [P, P, P, P, P]
            lib.or_pair_f32.restype = ctypes.c_int
            lib.or_bvh_build.argtypes = [P, i64, P, i64]
            lib.or_bvh_build.restype = P
            lib.or_bvh_free.argtypes = [P]
            lib.or_bvh_nodes.argtypes = [P]
            lib.or_bvh_nodes.restype = i64
            lib.or_cast_rays.argtypes = [P, P, P, i64, P, P, i64, P, ctypes.c_int]
            lib.or_hemisphere.argtypes = [P, P, P, i64, P, P, i64, i32, f64, P, P, P, ctypes.c_int]
            lib.or_orthogonal.argtypes = [P, P, P, i64, P, P, i64, P, f64, f64, P, P, ctypes.c_int]
            lib.or_variability.argtypes = [P, P, i64, i32, P, P, P]
            lib.or_num_cores.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def num_cores():
    return _L().or_num_cores()


def splitmix64(x):
    """The splitmix64 mixer (Steele, Lea, Flood 2014)."""
    return int(_L().or_splitmix64(ctypes.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


# ---------------------------------------------------------------------------
# Section 3.1: geometry preparation, sampling, directions, rays
# ---------------------------------------------------------------------------

def face_prep(V, F):
    """Per-face fp32 unit normal, FP64 area and fp32 centroid (Section 3.1)."""
    V, F = _c(V, np.float32), _c(F, np.int32)
    T = len(F)
    n = np.zeros((T, 3), np.float32)
    a = np.zeros(T, np.float64)
    c = np.zeros((T, 3), np.float32)
    _L().or_face_prep(_p(V), _p(F), T, _p(n), _p(a), _p(c))
    return n, a, c


def sample_centroid(V, F):
    """The paper's sampling: one point per face at its centroid, weighted by
    the face area (Section 3.1)."""
    n, a, c = face_prep(V, F)
    return c, n, np.arange(len(F), dtype=np.int32), a


def sample_area(V, F, n, seed=0):
    """Seeded area-weighted random points with their face normals (reading
    R7 of ``oracle.c``); weight 1 each."""
    V, F = _c(V, np.float32), _c(F, np.int32)
    P = np.zeros((n, 3), np.float32)
    Nn = np.zeros((n, 3), np.float32)
    fc = np.zeros(n, np.int32)
    rc = _L().or_sample_area(_p(V), _p(F), len(F), n, ctypes.c_uint64(seed), _p(P), _p(Nn), _p(fc))
    if rc != 0:
        raise ValueError("part has no positive-area face")
    return P, Nn, fc, np.ones(n, np.float64)


def sample_on_faces(V, F, face, seed=0, centroid=False):
    """Points kept on the given faces (reading R9 of ``oracle.c``): point i
    on face[i] at the position its own counter-based u1, u2 give (area
    mode), or at the face centroid; with the face normals."""
    V, F = _c(V, np.float32), _c(F, np.int32)
    face = _c(face, np.int32)
    n = len(face)
    P = np.zeros((n, 3), np.float32)
    Nn = np.zeros((n, 3), np.float32)
    bad = _L().or_sample_on_faces(_p(V), _p(F), len(F), n, ctypes.c_uint64(seed), int(bool(centroid)), _p(face),
                                  _p(P), _p(Nn))
    if bad >= 0:
        raise ValueError("face of point %d out of range" % bad)
    return P, Nn


def direction_table(N):
    """Fibonacci hemisphere (Section 3.1, Fig. 1; reading R2): FP64 and fp32."""
    h64 = np.zeros((N, 3), np.float64)
    h32 = np.zeros((N, 3), np.float32)
    _L().or_direction_table(N, _p(h64), _p(h32))
    return h64, h32


def ray_dirs(normal, N):
    """World directions of one point's hemisphere rays (reading R3)."""
    _, h32 = direction_table(N)
    d = np.zeros((N, 3), np.float32)
    _L().or_ray_dirs(_p(_c(normal, np.float32)), _p(h32), N, _p(d))
    return d


def rays_at(P, Nrm, N, i, j, eps=1e-4):
    """Origins and directions of selected hemisphere rays (readings R3, R4):
    ray k is direction j[k] of point i[k] (the same fp32 rays the
    hemisphere cast traces)."""
    _, h32 = direction_table(N)
    P, Nrm = _c(P, np.float32), _c(Nrm, np.float32)
    i = np.asarray(i, np.int64)
    j = np.asarray(j, np.int64)
    O = np.zeros((len(i), 3), np.float32)
    D = np.zeros((len(i), 3), np.float32)
    lib = _L()
    for k in range(len(i)):
        lib.or_ray_origin(_p(P[i[k]]), _p(Nrm[i[k]]), float(eps), _p(O[k]))
        lib.or_ray_dirs(_p(Nrm[i[k]]), _p(h32[j[k]]), 1, _p(D[k]))
    return O, D


def ray_origins(P, Nrm, eps):
    """o = fl32(p + eps*n) in FP64 (reading R4)."""
    P, Nrm = _c(P, np.float32), _c(Nrm, np.float32)
    o = np.zeros_like(P)
    lib = _L()
    for i in range(len(P)):
        lib.or_ray_origin(_p(P[i]), _p(Nrm[i]), float(eps), _p(o[i]))
    return o


def pair(o, d, A, B, C):
    """Classify one ray/triangle pair: 0 MISS, 1 HIT, 2 AMBIGUOUS."""
    a = [_c(x, np.float32) for x in (o, d, A, B, C)]
    return _L().or_pair_f32(*[_p(x) for x in a])


# ---------------------------------------------------------------------------
# acceleration structure
# ---------------------------------------------------------------------------

class Mesh:
    """A part held by the oracle: fp32 vertices, int32 faces and (unless
    ``brute``) a plain median-split FP64 BVH over them."""

    def __init__(self, V, F, brute=False):
        self.V = _c(V, np.float32)
        self.F = _c(F, np.int32)
        self.T = len(self.F)
        self.brute = brute
        self._h = None
        if not brute:
            self._h = _L().or_bvh_build(_p(self.V), len(self.V), _p(self.F), self.T)

    def __del__(self):
        if getattr(self, "_h", None):
            _L().or_bvh_free(self._h)
            self._h = None

    @property
    def handle(self):
        return None if self.brute else self._h

    def cast_rays(self, O, D, threads=0):
        """Per-ray state 0 MISS / 1 HIT / 2 AMBIGUOUS (readings R5, R6)."""
        O, D = _c(O, np.float32), _c(D, np.float32)
        st = np.zeros(len(O), np.int8)
        _L().or_cast_rays(self.handle, _p(self.V), _p(self.F), self.T, _p(O), _p(D), len(O),
                          _p(st), threads)
        return st

    def hemisphere(self, P, Nrm, N, eps=1e-4, threads=0):
        """Section 3.1: visibility bits (1 = unobstructed), ambiguity bits and
        per-point unobstructed counts for ``N`` directions per point."""
        P, Nrm = _c(P, np.float32), _c(Nrm, np.float32)
        n = len(P)
        W = (N + 31) // 32
        bits = np.zeros((n, W), np.uint32)
        amb = np.zeros((n, W), np.uint32)
        cnt = np.zeros(n, np.int32)
        _L().or_hemisphere(self.handle, _p(self.V), _p(self.F), self.T, _p(P), _p(Nrm), n, N,
                           float(eps), _p(bits), _p(amb), _p(cnt), threads)
        return bits, amb, cnt

    def orthogonal(self, P, Nrm, frame=None, eps=1e-4, threads=0, parallel_tol=PARALLEL_TOL):
        """Section 3.2: six-direction accessibility mask (bit a set = axis a
        eligible -- n . a >= -parallel_tol -- and unobstructed) plus the
        ambiguity mask."""
        P, Nrm = _c(P, np.float32), _c(Nrm, np.float32)
        axes = frame_axes(frame)
        n = len(P)
        m = np.zeros(n, np.uint8)
        am = np.zeros(n, np.uint8)
        _L().or_orthogonal(self.handle, _p(self.V), _p(self.F), self.T, _p(P), _p(Nrm), n,
                           _p(axes), float(eps), float(parallel_tol), _p(m), _p(am), threads)
        return m, am


def frame_axes(frame=None):
    """Six fp32 machining directions +X', -X', +Y', -Y', +Z', -Z': the
    columns of the row-major 3x3 ``frame`` and their negatives (Section 3.2)."""
    R = np.eye(3, dtype=np.float32) if frame is None else _c(frame, np.float32).reshape(3, 3)
    ax = np.zeros((6, 3), np.float32)
    for k in range(3):
        ax[2 * k] = R[:, k]
        ax[2 * k + 1] = -R[:, k]
    return ax


# ---------------------------------------------------------------------------
# Section 3.3: directional variability and classification indicators
# ---------------------------------------------------------------------------

Q40 = float(2 ** 40)


def variability(bits, Nrm, N, conc_mode=0):
    """Per point: fixed-point visible-direction sum M (int64 [n,3]), dominant
    axis (argmax |M_k|, ties to the lower axis; -1 if nothing is visible) and
    concentration (Section 3.3, 'how exclusively each face is accessible from
    its dominant axis').  conc_mode 0: share of visible rays whose largest
    component is the dominant axis; conc_mode 1: |M_dom| / (2^40 count)."""
    bits = _c(bits, np.uint32)
    Nrm = _c(Nrm, np.float32)
    n = len(Nrm)
    M = np.zeros((n, 3), np.int64)
    ac = np.zeros((n, 3), np.int32)
    dom = np.zeros(n, np.int8)
    _L().or_variability(_p(bits), _p(Nrm), n, N, _p(M), _p(ac), _p(dom))
    cnt = np.unpackbits(bits.view(np.uint8), axis=1).sum(1).astype(np.int64)
    conc = np.zeros(n, np.float64)
    ok = cnt > 0
    idx = np.flatnonzero(ok)
    if conc_mode == 0:
        conc[idx] = ac[idx, dom[idx]].astype(np.float64) / cnt[idx].astype(np.float64)
    else:
        conc[idx] = np.abs(M[idx, dom[idx]]).astype(np.float64) / (Q40 * cnt[idx].astype(np.float64))
    return M, ac, dom, conc, cnt


def summary(cnt, dom, conc, N, weight=None):
    """Part-level indicators (Sections 3.1 and 3.3).

    - overall accessibility: the area-weighted mean of the per-point
      unobstructed fractions, sum w_i count_i / (N sum w_i), in FP64 with
      no quantisation (Section 3.1's area-weighted score; unit weights give
      the plain mean over the points);
    - dominant-axis distribution: share of points with count > 0 whose
      dominant axis is x, y, z (sums to 1);
    - mean axis concentration over the same points, summed as
      round(conc_i * 2^40) in integers."""
    cnt = np.asarray(cnt, np.int64)
    n = len(cnt)
    w = np.ones(n, np.float64) if weight is None else np.asarray(weight, np.float64)
    num = float(np.sum(w * cnt.astype(np.float64)))
    den = float(np.sum(w)) * N
    overall = num / den if den else 0.0
    ok = cnt > 0
    nc = int(ok.sum())
    share = [float(int((dom[ok] == k).sum())) / nc if nc else 0.0 for k in range(3)]
    csum = sum(int(np.rint(c * Q40)) for c in np.asarray(conc)[ok])
    mean_conc = float(csum) / (Q40 * nc) if nc else 0.0
    unweighted = float(cnt.sum()) / float(n * N) if n else 0.0
    return {
        "overall_access": overall,
        "overall_access_unweighted": unweighted,
        "axis_share": share,
        "mean_conc": mean_conc,
        "n_points": n,
        "n_counted": nc,
        "n_zero_visible": n - nc,
    }


def classify(s, t_acc=0.60, t_share=0.45, t_conc=0.41):
    """Section 3.3: multi-axis (1) if any indicator crosses its threshold --
    overall accessibility below t_acc, largest dominant-axis share below
    t_share (no clear dominant axis), or mean concentration above t_conc --
    else 3-axis (0)."""
    multi = (s["overall_access"] < t_acc) or (max(s["axis_share"]) < t_share) or \
        (s["mean_conc"] > t_conc)
    return 1 if multi else 0


# ---------------------------------------------------------------------------
# Section 3.3: reachability, fixture faces, face classes, setups
# ---------------------------------------------------------------------------

def _frame_coords(X, R):
    """Coordinates along the frame's columns, FP64, summed in x, y, z order."""
    X = np.asarray(X, np.float64)
    R = np.asarray(R, np.float64)
    out = np.empty_like(X)
    for k in range(3):
        s = X[:, 0] * R[0, k] + X[:, 1] * R[1, k]
        out[:, k] = s + X[:, 2] * R[2, k]
    return out


def travel(V, P, frame=None):
    """Tool travel (Section 3.3, reading: distance from the point to the
    part's bounding-box face along each axis, in the machining frame):
    fp32 [n, 6] in the order +X', -X', +Y', -Y', +Z', -Z'."""
    R = np.eye(3, dtype=np.float32) if frame is None else _c(frame, np.float32).reshape(3, 3)
    Vq = _frame_coords(V, R)
    lo, hi = Vq.min(0), Vq.max(0)
    Pq = _frame_coords(P, R)
    t = np.empty((len(P), 6), np.float32)
    for k in range(3):
        t[:, 2 * k] = (hi[k] - Pq[:, k]).astype(np.float32)
        t[:, 2 * k + 1] = (Pq[:, k] - lo[k]).astype(np.float32)
    return t


def fixture_faces(V, F, frame=None, rel_tol=1e-6):
    """Section 3.3: 'bounding box faces are excluded as fixture surfaces'.
    A face is a fixture face when its three vertices lie within
    rel_tol*diag of one bounding-box plane (machining frame) and its normal
    points out through that plane to within rel_tol."""
    R = np.eye(3, dtype=np.float32) if frame is None else _c(frame, np.float32).reshape(3, 3)
    Vq = _frame_coords(V, R)
    lo, hi = Vq.min(0), Vq.max(0)
    diag = float(np.sqrt(((hi - lo) ** 2).sum()))
    tol = rel_tol * diag
    n, _, _ = face_prep(V, F)
    nq = _frame_coords(n, R)
    F = np.asarray(F, np.int64)
    out = np.zeros(len(F), bool)
    for k in range(3):
        c = Vq[:, k][F]
        on_hi = (np.abs(c - hi[k]) <= tol).all(1) & (nq[:, k] >= 1.0 - rel_tol)
        on_lo = (np.abs(c - lo[k]) <= tol).all(1) & (nq[:, k] <= -(1.0 - rel_tol))
        out |= on_hi | on_lo
    return out


def face_classes(mask, trav, face, fixture, tool_length):
    """Section 3.3 face classes: 0 viable (some accessible axis with travel
    <= tool length), 1 over-threshold (accessible only beyond it), 2 fully
    inaccessible, 3 fixture (excluded).  Returns (class, reach mask)."""
    mask = np.asarray(mask, np.uint8)
    reach = np.zeros_like(mask)
    for a in range(6):
        ok = ((mask >> a) & 1).astype(bool) & (np.asarray(trav)[:, a] <= np.float32(tool_length))
        reach |= (ok.astype(np.uint8) << a)
    cls = np.where(reach != 0, 0, np.where(mask != 0, 1, 2)).astype(np.uint8)
    cls[np.asarray(fixture)[np.asarray(face)]] = 3
    return cls, reach


def setups_exact(reach_masks):
    """Smallest set S of the six axes with S & m != 0 for every viable mask m
    (the 'theoretical minimum', Section 5); ties to the smallest bitmask."""
    ms = sorted(set(int(m) for m in reach_masks))
    if not ms:
        return 0, 0
    for size in range(1, 7):
        for S in range(1, 64):
            if bin(S).count("1") != size:
                continue
            if all(S & m for m in ms):
                return size, S
    raise AssertionError("unreachable: viable masks are non-zero")


def setups_greedy(reach_masks):
    """Greedy set cover over the six axes (Section 3.3): repeatedly take the
    axis covering the most uncovered viable points, ties to the lower axis."""
    left = [int(m) for m in reach_masks]
    S = 0
    while left:
        best, bc = -1, -1
        for a in range(6):
            if S >> a & 1:
                continue
            c = sum(1 for m in left if m >> a & 1)
            if c > bc:
                best, bc = a, c
        S |= 1 << best
        left = [m for m in left if not (m >> best & 1)]
    return bin(S).count("1"), S
