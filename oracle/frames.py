"""Automatic machining frame -- TEST INFRASTRUCTURE ONLY.

Part of the FP64 CPU oracle: only the test suite, ``__graft_entry__.smoke()``
and the CPU legs of ``bench.py`` may import it; the library never does.  Plain
numpy and Python floats; the orthogonal cast and the setup cover come from the
oracle's own functions in ``oracle/__init__.py``.

Section 3.2 of the paper puts the part in a canonical frame whose axes X', Y',
Z' are the machine axes, and Section 3.3 counts setups in that frame; how the
frame is found is not stated.  The readings taken here (and by the library, in
its own code) are:

F1  Principal axes.  The area second moment of the surface about its area
    centroid, M = sum_f int_f (x - c)(x - c)^T dA, using the exact triangle
    integral int_f x x^T dA = A_f / 12 (a a^T + b b^T + c c^T + s s^T) with
    s = a + b + c.  Eigenvectors by descending eigenvalue give X' and Y';
    Z' = X' x Y'.  When two adjacent eigenvalues (descending) differ by at most
    1e-3 times the largest one the axes are not determined and this candidate
    is absent.
F2  Dominant normals.  Face normals are binned as lines (n and -n together)
    on a cube map of 3 x 32 x 32 cells, weighted by the quantised face areas
    llround(A_f / A_max * 2^32).  Z' is the normal of the largest face of the
    heaviest cell.  X' is the normal of the largest face of the heaviest cell
    whose centre direction w has |w . Z'| <= 0.2 |w|, made orthogonal to Z'.
    Y' = Z' x X'.  Ties go to the lower cell index, then the lower face id.
F3  Box-minimising rotation of a base frame.  Each column of the base frame
    in turn is held and the other two are turned about it by theta with
    tan(theta / 2) = j / 128, j = 0 .. 127 (0 to 90 degrees; cos and sin are
    the rational (1 - t^2) / (1 + t^2) and 2t / (1 + t^2)).  The rotation
    whose frame bounding box of the vertices has the smallest volume wins;
    ties go to the lower column, then the lower j.
F4  Snapping.  The axis vectors of F1 and F2 are rounded to multiples of
    2^-20 per component, their sign is fixed so that the largest-magnitude
    component is positive, and the pair is orthonormalised (Gram-Schmidt) in
    FP64 and rounded to fp32.  Two computations of the same axes that agree
    to ~1e-12 thus give the same frame.
F5  Candidates, in this order: the given frame, its box rotation, the
    principal frame, its box rotation, the normals frame, its box rotation,
    each rounded to fp32 with negative zeros made positive; a candidate whose
    three axes are, up to sign and order, those of an earlier one (fp32
    values equal) is dropped -- it has the same six machining directions.
F6  Selection.  The candidate with the fewest setups (the exact cover of
    Section 3.3) wins; ties go to the one with fewer over-threshold plus
    inaccessible points, then to the smaller bounding-box volume (less stock
    to remove), then to the lower index.

All FP64 expressions are evaluated left to right, one rounding per operation
(numpy element-wise operations and Python floats do not fuse).
"""
from __future__ import annotations

import math

import numpy as np

from . import Mesh, face_prep, face_classes, fixture_faces, setups_exact, setups_greedy, travel

SNAP = 2.0 ** 20
CELLS = 32
BOX_STEPS = 128
GAP = 1e-3
ORTHO = 0.2

GIVEN, PRINCIPAL, NORMALS = 0, 1, 2
BOX = 3          # + base source


# ---------------------------------------------------------------------------
# F1: principal axes of the surface
# ---------------------------------------------------------------------------

def surface_moments(V, F, ref=None):
    """Area moments of the surface (F1) relative to ``ref`` (default: the
    vertex bounding-box midpoint): S0 = sum A_f, S1 = sum A_f g_f and
    S2 = sum A_f / 12 (a a^T + b b^T + c c^T + s s^T)."""
    V64 = np.asarray(V, np.float64)
    F = np.asarray(F, np.int64)
    r = 0.5 * (V64.min(0) + V64.max(0)) if ref is None else np.asarray(ref, np.float64)
    _, A, _ = face_prep(V, F)
    a, b, c = V64[F[:, 0]] - r, V64[F[:, 1]] - r, V64[F[:, 2]] - r
    s = a + b + c
    S0 = A.sum()
    S1 = (A[:, None] * s / 3.0).sum(0)
    outer = lambda u: u[:, :, None] * u[:, None, :]
    S2 = ((A / 12.0)[:, None, None] * (outer(a) + outer(b) + outer(c) + outer(s))).sum(0)
    return S0, S1, S2, r


def central_second_moment(V, F):
    """M = S2 - S0 c c^T with the area centroid c = S1 / S0 (F1)."""
    S0, S1, S2, r = surface_moments(V, F)
    cen = S1 / S0
    return S2 - S0 * np.outer(cen, cen), cen + r


def principal_axes(V, F):
    """Eigenvalues (descending) and unit eigenvectors (columns) of M."""
    M, _ = central_second_moment(V, F)
    w, U = np.linalg.eigh(M)
    order = np.argsort(-w, kind="stable")
    return w[order], U[:, order]


# ---------------------------------------------------------------------------
# F4: snapping, Gram-Schmidt, cross products
# ---------------------------------------------------------------------------

def _dot(u, v):
    return (u[0] * v[0] + u[1] * v[1]) + u[2] * v[2]


def _unit(u):
    n = math.sqrt((u[0] * u[0] + u[1] * u[1]) + u[2] * u[2])
    return [u[0] / n, u[1] / n, u[2] / n]


def _cross(u, v):
    return [u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]]


def snap(u):
    """Components rounded to multiples of 2^-20 (half to even; -0 becomes
    +0), sign such that the largest-magnitude component (lowest index on
    ties) is positive."""
    w = [float(np.rint(float(x) * SNAP)) / SNAP + 0.0 for x in u]     # + 0.0: no negative zeros
    k = 0
    for i in (1, 2):
        if abs(w[i]) > abs(w[k]):
            k = i
    if w[k] < 0.0:
        w = [-x for x in w]
    return w


def frame_from(col_a, u, col_b, v):
    """Right-handed orthonormal FP64 frame (row-major 3x3, columns X', Y', Z')
    with column ``col_a`` along snap(u) and column ``col_b`` along snap(v)
    made orthogonal to it (F4)."""
    ea = _unit(snap(u))
    w = snap(v)
    d = _dot(w, ea)
    eb = _unit([w[0] - d * ea[0], w[1] - d * ea[1], w[2] - d * ea[2]])
    col_c = 3 - col_a - col_b
    ec = _cross(ea, eb) if (col_a + 1) % 3 == col_b else _cross(eb, ea)
    R = np.zeros((3, 3), np.float64)
    R[:, col_a], R[:, col_b], R[:, col_c] = ea, eb, ec
    return R


def principal_frame(V, F):
    """F1 + F4: X' along the largest-eigenvalue axis, Y' the second; None
    when two eigenvalues are within GAP of the largest."""
    w, U = principal_axes(V, F)
    if not w[0] > 0.0 or (w[0] - w[1]) <= GAP * w[0] or (w[1] - w[2]) <= GAP * w[0]:
        return None, w
    return frame_from(0, U[:, 0], 1, U[:, 1]), w


# ---------------------------------------------------------------------------
# F2: dominant normals
# ---------------------------------------------------------------------------

def quantised_areas(area):
    """llround(A_f / A_max * 2^32), exact (the sampler's quantisation)."""
    A = np.asarray(area, np.float64)
    amax = A.max() if len(A) else 0.0
    if not amax > 0.0:
        return np.zeros(len(A), np.int64)
    x = (A / amax) * 4294967296.0
    fl = np.floor(x)
    return (fl + (x - fl >= 0.5)).astype(np.int64)


def normal_cells(normals):
    """Cube-map cell of each normal taken as a line (F2): major axis k
    (lowest on ties), sign flipped so n_k > 0, the other two components in
    (k+1, k+2) order divided by n_k, 32 cells per side."""
    n = np.asarray(normals, np.float32).astype(np.float64)
    k = np.argmax(np.abs(n), axis=1)
    rows = np.arange(len(n))
    nk = n[rows, k]
    sgn = np.where(nk < 0.0, -1.0, 1.0)
    m = np.abs(nk)
    u = (n[rows, (k + 1) % 3] * sgn) / m
    v = (n[rows, (k + 2) % 3] * sgn) / m
    half = CELLS / 2.0
    i = np.clip(np.floor((u + 1.0) * half), 0, CELLS - 1).astype(np.int64)
    j = np.clip(np.floor((v + 1.0) * half), 0, CELLS - 1).astype(np.int64)
    return (k * CELLS + i) * CELLS + j, sgn


def _cell_centre(cell):
    k, rem = divmod(int(cell), CELLS * CELLS)
    i, j = divmod(rem, CELLS)
    w = [0.0, 0.0, 0.0]
    w[k] = 1.0
    w[(k + 1) % 3] = (i + 0.5) / (CELLS / 2.0) - 1.0
    w[(k + 2) % 3] = (j + 0.5) / (CELLS / 2.0) - 1.0
    return w


def _largest_face(cells, qa, cell):
    idx = np.flatnonzero((cells == cell) & (qa > 0))
    best = idx[np.argmax(qa[idx])]          # first maximum: lowest face id
    return int(best)


def normals_frame(V, F):
    """F2 + F4: Z' from the heaviest normal cell, X' from the heaviest cell
    nearly orthogonal to it; None when no such second cell exists."""
    nrm, A, _ = face_prep(V, F)
    qa = quantised_areas(A)
    cells, sgn = normal_cells(nrm)
    H = np.zeros(3 * CELLS * CELLS, np.int64)
    np.add.at(H, cells, qa)
    if not (H > 0).any():
        return None
    c1 = int(np.argmax(H))
    f1 = _largest_face(cells, qa, c1)
    u1 = [float(x) * sgn[f1] for x in nrm[f1].astype(np.float64)]
    e1 = _unit(snap(u1))
    best, c2 = -1, -1
    for c in np.flatnonzero(H > 0):
        w = _cell_centre(c)
        nw = math.sqrt((w[0] * w[0] + w[1] * w[1]) + w[2] * w[2])
        if abs(_dot(w, e1)) <= ORTHO * nw and H[c] > best:
            best, c2 = int(H[c]), int(c)
    if c2 < 0:
        return None
    f2 = _largest_face(cells, qa, c2)
    u2 = [float(x) * sgn[f2] for x in nrm[f2].astype(np.float64)]
    return frame_from(2, u1, 0, u2)


# ---------------------------------------------------------------------------
# F3: box-minimising rotations
# ---------------------------------------------------------------------------

def box_volume(V, G):
    """Volume of the vertices' bounding box in the FP64 frame G (columns)."""
    X = np.asarray(V, np.float64)
    ext = []
    for k in range(3):
        q = (X[:, 0] * G[0, k] + X[:, 1] * G[1, k]) + X[:, 2] * G[2, k]
        ext.append(q.max() - q.min())
    return (ext[0] * ext[1]) * ext[2]


def box_rotations(B):
    """The 3 x BOX_STEPS rotated FP64 frames of base frame B (F3), column
    ``a`` held, in (a, j) order."""
    B = np.asarray(B, np.float32).astype(np.float64).reshape(3, 3)
    out = []
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        for j in range(BOX_STEPS):
            t = j / float(BOX_STEPS)
            t2 = t * t
            den = 1.0 + t2
            cs = (1.0 - t2) / den
            sn = (2.0 * t) / den
            G = B.copy()
            G[:, b] = cs * B[:, b] + sn * B[:, c]
            G[:, c] = cs * B[:, c] - sn * B[:, b]
            out.append((a, j, G))
    return out


def box_search(V, B):
    """Best rotation of base frame B (F3): (axis, step, FP64 frame, volume)."""
    best = None
    for a, j, G in box_rotations(B):
        vol = box_volume(V, G)
        if best is None or vol < best[3]:
            best = (a, j, G, vol)
    return best


# ---------------------------------------------------------------------------
# F5 / F6: candidates and selection
# ---------------------------------------------------------------------------

def frame_candidates(V, F, frame=None):
    """Candidate frames (F5): list of dicts with ``source``, ``frame`` (fp32
    row-major [9]), ``box_axis``, ``box_step`` (-1 unless a box rotation)
    and ``volume`` (vertex bounding-box volume in the candidate's fp32 frame,
    evaluated in FP64)."""
    base0 = np.eye(3, dtype=np.float32) if frame is None else np.asarray(frame, np.float32).reshape(3, 3)
    bases = [(GIVEN, base0)]
    P, _ = principal_frame(V, F)
    if P is not None:
        bases.append((PRINCIPAL, P.astype(np.float32)))
    Nf = normals_frame(V, F)
    if Nf is not None:
        bases.append((NORMALS, Nf.astype(np.float32)))
    out = []

    def same_axes(A, B):
        return all(any(np.array_equal(A[:, k], B[:, j]) or np.array_equal(A[:, k], -B[:, j]) for j in range(3))
                   for k in range(3))

    def add(src, f, a, j):
        f32 = np.asarray(f, np.float32).reshape(3, 3) + np.float32(0.0)     # no negative zeros
        if any(same_axes(f32, c["frame"].reshape(3, 3)) for c in out):
            return
        out.append({"source": src, "frame": f32.reshape(9), "box_axis": a, "box_step": j,
                    "volume": box_volume(V, f32.astype(np.float64))})

    for src, B in bases:
        a, j, G, vol = box_search(V, B)
        add(src, B, -1, -1)
        add(BOX + src, G.astype(np.float32), a, j)
    return out


def evaluate_frame(mesh, V, F, P, Nn, face, frame, tool_length, eps=1e-4):
    """Orthogonal cast, classes and setups of the points in one frame
    (Sections 3.2 and 3.3) with the oracle's own masks."""
    m, am = mesh.orthogonal(P, Nn, frame=frame, eps=eps)
    tr = travel(V, P, frame=frame)
    fx = fixture_faces(V, F, frame=frame)
    cls, reach = face_classes(m, tr, face, fx, tool_length)
    viable = reach[cls == 0]
    se, ce = setups_exact(viable)
    sg, cg = setups_greedy(viable)
    counts = [int((cls == k).sum()) for k in range(4)]
    return {"mask": m, "amb": am, "travel": tr, "cls": cls, "setups_exact": se, "chosen_exact": ce,
            "setups_greedy": sg, "chosen_greedy": cg, "class_counts": counts}


def select_frame(cands, evals):
    """F6: fewest setups, then fewest over-threshold + inaccessible points,
    then the smallest box volume, then the lowest index."""
    keys = [(e["setups_exact"], e["class_counts"][1] + e["class_counts"][2], c["volume"], i)
            for i, (c, e) in enumerate(zip(cands, evals))]
    return min(keys)[3]


def auto_frame(V, F, P, Nn, face, tool_length, frame=None, eps=1e-4):
    """Candidates (F5), their evaluation and the selection (F6)."""
    cands = frame_candidates(V, F, frame)
    mesh = Mesh(V, F)
    evals = [evaluate_frame(mesh, V, F, P, Nn, face, c["frame"], tool_length, eps) for c in cands]
    return cands, evals, select_frame(cands, evals)
