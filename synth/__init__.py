"""Seeded synthetic parts: the input meshes for tests and benchmarks.

This module produces triangle meshes and nothing else.  It holds none of the
ray-casting method's arithmetic (no normals, areas, sampling, directions or
intersection tests); both the CPU oracle and the CUDA library consume its
output.  Every mesh is returned as ``(V, F)`` with ``V`` float32 ``[nV, 3]``
(millimetres) and ``F`` int32 ``[T, 3]``, wound counter-clockwise when seen
from outside the material (outward right-hand normals), watertight.

Generators
----------
- :func:`pocket_block` -- the paper's prismatic class at its simplest: an
  axis-aligned block with one centred square pocket, an explicit polyhedron
  refined by conforming 1->4 midpoint subdivision (all coordinates stay
  dyadic, hence exact in fp32).
- :func:`prismatic` -- block with a T-slot, four oblique through-holes and two
  side pockets, meshed from a signed distance function by marching
  tetrahedra (stand-in for the housing of the paper's second case study,
  Section 4.2).
- :func:`impeller` -- hub with twelve wrapped, twisted blades meshed the same
  way (stand-in for the impeller of the first case study, Section 4.1).
- :func:`cube`, :func:`icosphere` -- convex solids (every hemisphere ray from
  their surface escapes).
- :func:`cavity_box` -- block with a sealed internal void (every ray from the
  void's surface is blocked).
- :func:`deep_hole` -- block with one narrow deep square hole.
- :func:`rotate90` -- exact 90-degree rotation / axis permutation of a mesh.
- :func:`bump` -- a local smooth bump of a mesh (vertices within a radius
  pushed along a direction; the triangle list is unchanged): a local edit.
- :func:`rotation`, :func:`rotate` -- a rotation matrix from Euler angles and
  a mesh turned by it (vertices rounded to fp32): parts that do not sit in
  their machining frame.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "pocket_block", "prismatic", "impeller", "cube", "icosphere", "cavity_box",
    "deep_hole", "box_with_pockets", "rotate90", "subdivide", "marching_tets",
    "part_family", "perturbed_part", "rotation", "rotate", "bump",
]


# ---------------------------------------------------------------------------
# explicit polyhedra
# ---------------------------------------------------------------------------

def _quad(a, b, c, d):
    """Two triangles of the planar quad a-b-c-d given counter-clockwise."""
    return [(a, b, c), (a, c, d)]


def _mesh_from_tris(tris):
    """Index a list of triangles given as float64 vertex triples."""
    pts = np.asarray(tris, dtype=np.float64).reshape(-1, 3)
    uniq, inv = np.unique(pts, axis=0, return_inverse=True)
    return uniq, inv.reshape(-1, 3).astype(np.int64)


def subdivide(V, F, levels):
    """Conforming 1->4 midpoint subdivision, in float64 (midpoints of shared
    edges are computed identically, so the result stays watertight)."""
    V = np.asarray(V, dtype=np.float64)
    F = np.asarray(F, dtype=np.int64)
    for _ in range(levels):
        e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
        key = np.sort(e, axis=1)
        uk, inv = np.unique(key, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        mids = 0.5 * (V[uk[:, 0]] + V[uk[:, 1]])
        base = len(V)
        V = np.concatenate([V, mids])
        T = len(F)
        m01 = base + inv[0:T]
        m12 = base + inv[T:2 * T]
        m20 = base + inv[2 * T:3 * T]
        a, b, c = F[:, 0], F[:, 1], F[:, 2]
        F = np.concatenate([
            np.stack([a, m01, m20], 1),
            np.stack([m01, b, m12], 1),
            np.stack([m20, m12, c], 1),
            np.stack([m01, m12, m20], 1),
        ])
    return V, F


def _finish(V, F):
    return np.ascontiguousarray(V, dtype=np.float32), np.ascontiguousarray(F, dtype=np.int32)


def _box_tris(lo, hi, inward=False):
    """12 triangles of an axis-aligned box, outward (or inward) wound."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    p = {
        (i, j, k): (x1 if i else x0, y1 if j else y0, z1 if k else z0)
        for i in (0, 1) for j in (0, 1) for k in (0, 1)
    }
    faces = [
        # -z bottom, seen from below: counter-clockwise
        (p[0, 0, 0], p[0, 1, 0], p[1, 1, 0], p[1, 0, 0]),
        # +z top
        (p[0, 0, 1], p[1, 0, 1], p[1, 1, 1], p[0, 1, 1]),
        # -y
        (p[0, 0, 0], p[1, 0, 0], p[1, 0, 1], p[0, 0, 1]),
        # +y
        (p[0, 1, 0], p[0, 1, 1], p[1, 1, 1], p[1, 1, 0]),
        # -x
        (p[0, 0, 0], p[0, 0, 1], p[0, 1, 1], p[0, 1, 0]),
        # +x
        (p[1, 0, 0], p[1, 1, 0], p[1, 1, 1], p[1, 0, 1]),
    ]
    tris = []
    for q in faces:
        if inward:
            q = q[::-1]
        tris += _quad(*q)
    return tris


def cube(size=20.0, subdiv=2, origin=(0.0, 0.0, 0.0)):
    """Axis-aligned cube ``[origin, origin+size]^3`` (convex)."""
    lo = np.asarray(origin, dtype=np.float64)
    V, F = _mesh_from_tris(_box_tris(lo, lo + size))
    return _finish(*subdivide(V, F, subdiv))


def cavity_box(outer=40.0, inner=(10.0, 30.0), subdiv=2):
    """Solid block with a sealed cubic void.  The void's surface is wound so
    its normals point into the void (away from the material); every ray
    leaving that surface is blocked by the void's other walls."""
    tris = _box_tris((0.0, 0.0, 0.0), (outer,) * 3)
    a, b = inner
    tris += _box_tris((a, a, a), (b, b, b), inward=True)
    V, F = _mesh_from_tris(tris)
    return _finish(*subdivide(V, F, subdiv))


def box_with_pockets(size=(100.0, 60.0, 40.0), pockets=(("+z", (35.0, 65.0), (15.0, 45.0), 15.0),),
                     subdiv=0):
    """Axis-aligned block with rectangular pockets sunk into chosen faces.

    Each pocket is ``(face, (u0, u1), (v0, v1), depth)`` where ``face`` is one
    of ``+x -x +y -y +z -z`` and ``(u, v)`` are the face's two in-plane axes in
    x<y<z order.  The face around each opening is triangulated as a conforming
    ring of four trapezoids, so the mesh has no T-junctions."""
    L = np.asarray(size, dtype=np.float64)
    by_face = {}
    for pk in pockets:
        by_face.setdefault(pk[0], []).append(pk)
    tris = []
    for axis in range(3):
        for sign in (+1, -1):
            name = ("+" if sign > 0 else "-") + "xyz"[axis]
            u_ax, v_ax = [k for k in range(3) if k != axis]
            w = L[axis] if sign > 0 else 0.0

            def P(u, v, ww=w):
                p = [0.0, 0.0, 0.0]
                p[axis] = ww
                p[u_ax] = u
                p[v_ax] = v
                return tuple(p)

            # counter-clockwise in (u, v) seen from +axis is (u,v) order for
            # u<v cyclic ordering when (u_ax, v_ax, axis) is even.
            even = (u_ax, v_ax, axis) in ((0, 1, 2), (1, 2, 0), (2, 0, 1))
            flip = (sign > 0) != even

            def add(q):
                q = list(q)
                if flip:
                    q = q[::-1]
                tris.extend(_quad(*q))

            U, Vv = L[u_ax], L[v_ax]
            pk = by_face.get(name, [])
            if not pk:
                add([P(0, 0), P(U, 0), P(U, Vv), P(0, Vv)])
                continue
            assert len(pk) == 1, "one pocket per face"
            _, (u0, u1), (v0, v1), depth = pk[0]
            o = [P(0, 0), P(U, 0), P(U, Vv), P(0, Vv)]
            i = [P(u0, v0), P(u1, v0), P(u1, v1), P(u0, v1)]
            for k in range(4):
                add([o[k], o[(k + 1) % 4], i[(k + 1) % 4], i[k]])
            wf = w - sign * depth
            f = [P(u0, v0, wf), P(u1, v0, wf), P(u1, v1, wf), P(u0, v1, wf)]
            # floor faces the same way as the outer face
            add(f)
            # walls: from the opening rim down to the floor, facing inwards
            for k in range(4):
                add([i[k], i[(k + 1) % 4], f[(k + 1) % 4], f[k]])
    V, F = _mesh_from_tris(tris)
    return _finish(*subdivide(V, F, subdiv))


def pocket_block(subdiv=3, size=(100.0, 60.0, 40.0), width=30.0, depth=15.0):
    """Block ``size`` (mm, corner at the origin) with one centred square
    pocket ``width`` x ``width`` x ``depth`` in its top (+z) face; 28 base
    triangles, times ``4**subdiv`` (subdiv=3 gives 1,792 triangles)."""
    cx, cy = size[0] / 2, size[1] / 2
    h = width / 2
    return box_with_pockets(size, (("+z", (cx - h, cx + h), (cy - h, cy + h), depth),), subdiv)


def deep_hole(width=2.0, depth=38.0, size=(20.0, 20.0, 40.0), subdiv=0):
    """Block with one narrow square blind hole in its top face."""
    cx, cy = size[0] / 2, size[1] / 2
    h = width / 2
    return box_with_pockets(size, (("+z", (cx - h, cx + h), (cy - h, cy + h), depth),), subdiv)


def icosphere(radius=10.0, subdiv=3):
    """Triangulated sphere.  The vertices are rounded to fp32 first and the
    mesh is the convex hull of exactly those points, so the polytope is
    convex in the coordinates that are actually stored."""
    from scipy.spatial import ConvexHull

    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]])
    V, F = subdivide(v, f, subdiv)
    V = V / np.linalg.norm(V, axis=1, keepdims=True) * radius
    V32 = V.astype(np.float32)
    hull = ConvexHull(V32.astype(np.float64))
    F = hull.simplices.astype(np.int64)
    # orient every facet outward using the hull's plane normals
    P = V32.astype(np.float64)
    n = np.cross(P[F[:, 1]] - P[F[:, 0]], P[F[:, 2]] - P[F[:, 0]])
    flip = np.einsum("ij,ij->i", n, hull.equations[:, :3]) < 0
    F[flip] = F[flip][:, ::-1]
    return _finish(V32, F)


def rotate90(V, axis, k=1):
    """Rotate a mesh by ``k`` quarter turns about coordinate ``axis``; exact
    in fp32 (only swaps and sign flips)."""
    V = np.asarray(V, dtype=np.float32).copy()
    a, b = [(1, 2), (2, 0), (0, 1)][axis]
    for _ in range(k % 4):
        va, vb = V[:, a].copy(), V[:, b].copy()
        V[:, a], V[:, b] = -vb, va
    return V


def bump(V, centre, radius, height, direction=(0.0, 0.0, 1.0)):
    """Vertices within ``radius`` of ``centre`` moved by height * (1 -
    (d / radius)^2)^2 along ``direction`` (FP64, rounded to fp32); the others
    are unchanged bit for bit."""
    V64 = np.asarray(V, np.float64)
    d = np.linalg.norm(V64 - np.asarray(centre, np.float64), axis=1)
    w = np.where(d < radius, (1.0 - (d / radius) ** 2) ** 2, 0.0)
    u = np.asarray(direction, np.float64)
    u = u / np.linalg.norm(u)
    out = np.asarray(V, np.float32).copy()
    sel = w > 0
    out[sel] = (V64[sel] + height * w[sel, None] * u).astype(np.float32)
    return out


def rotation(rx_deg=0.0, ry_deg=0.0, rz_deg=0.0):
    """FP64 rotation matrix Rz @ Ry @ Rx (angles in degrees)."""
    ax, ay, az = (math.radians(x) for x in (rx_deg, ry_deg, rz_deg))
    Rx = np.array([[1, 0, 0], [0, math.cos(ax), -math.sin(ax)], [0, math.sin(ax), math.cos(ax)]])
    Ry = np.array([[math.cos(ay), 0, math.sin(ay)], [0, 1, 0], [-math.sin(ay), 0, math.cos(ay)]])
    Rz = np.array([[math.cos(az), -math.sin(az), 0], [math.sin(az), math.cos(az), 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def rotate(V, R, centre=None):
    """Vertices turned by the 3x3 matrix ``R`` about ``centre`` (default: the
    bounding-box midpoint), computed in FP64 and rounded to fp32.  The
    triangle list is unchanged, so the winding stays outward."""
    V64 = np.asarray(V, np.float64)
    c = 0.5 * (V64.min(0) + V64.max(0)) if centre is None else np.asarray(centre, np.float64)
    return ((V64 - c) @ np.asarray(R, np.float64).T + c).astype(np.float32)


# ---------------------------------------------------------------------------
# marching tetrahedra
# ---------------------------------------------------------------------------

# Freudenthal decomposition of the unit cube into six tetrahedra sharing the
# 000-111 diagonal; it tiles space consistently, so neighbouring cells agree
# on every shared face diagonal and the extracted surface is watertight.
_CORNERS = np.array([(i, j, k) for i in (0, 1) for j in (0, 1) for k in (0, 1)])
_TETS = []
for _perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
    _p = [0, 0, 0]
    _path = [tuple(_p)]
    for _ax in _perm:
        _p[_ax] = 1
        _path.append(tuple(_p))
    _TETS.append([int(np.flatnonzero((_CORNERS == c).all(1))[0]) for c in _path])
_TETS = np.array(_TETS)


def marching_tets(sdf, lo, hi, h, chunk=24):
    """Mesh the zero set of ``sdf`` (negative inside) on a regular grid.

    ``sdf(x, y, z)`` takes broadcastable float64 arrays.  The grid starts at
    ``lo`` and has spacing ``h``.  Surface points are interpolated along
    grid edges with the lower grid index first, so a crossing shared by
    several tetrahedra is computed once and reused."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    n = np.ceil((hi - lo) / h).astype(int) + 1
    nx, ny, nz = (int(a) for a in n)
    xs = lo[0] + h * np.arange(nx)
    ys = lo[1] + h * np.arange(ny)
    zs = lo[2] + h * np.arange(nz)
    f = np.empty((nx, ny, nz), dtype=np.float64)
    for k0 in range(0, nz, chunk):
        k1 = min(nz, k0 + chunk)
        f[:, :, k0:k1] = sdf(xs[:, None, None], ys[None, :, None], zs[None, None, k0:k1])
    inside = f < 0
    # candidate cells: corners disagree
    cnt = np.zeros((nx - 1, ny - 1, nz - 1), dtype=np.int8)
    for (i, j, k) in _CORNERS:
        cnt += inside[i:nx - 1 + i, j:ny - 1 + j, k:nz - 1 + k]
    ci, cj, ck = np.nonzero((cnt > 0) & (cnt < 8))
    del cnt
    strides = np.array([ny * nz, nz, 1], dtype=np.int64)
    base = ci.astype(np.int64) * strides[0] + cj * strides[1] + ck
    corner_off = (_CORNERS * strides).sum(1)
    gidx = base[:, None] + corner_off[None, :]           # [M, 8]
    tet = gidx[:, _TETS].reshape(-1, 4)                   # [6M, 4]
    ff = f.reshape(-1)
    val = ff[tet]
    ins = val < 0
    nin = ins.sum(1)
    keep = (nin > 0) & (nin < 4)
    tet, val, ins, nin = tet[keep], val[keep], ins[keep], nin[keep]

    def gpos(g):
        i = g // strides[0]
        j = (g // strides[1]) % ny
        k = g % nz
        return np.stack([xs[i], ys[j], zs[k]], -1)

    # order the four corners of each tet: inside ones first
    order = np.argsort(~ins, axis=1, kind="stable")
    tet = np.take_along_axis(tet, order, 1)
    edges = []   # per triangle: 3 (ga, gb) pairs
    ref_in = []  # per triangle: an inside corner and an outside corner centroid
    ref_out = []
    # 1 inside: p | q1 q2 q3
    m = nin == 1
    t1 = tet[m]
    if len(t1):
        edges.append(np.stack([t1[:, [0, 1]], t1[:, [0, 2]], t1[:, [0, 3]]], 1))
        ref_in.append(t1[:, [0]])
        ref_out.append(t1[:, 1:])
    # 3 inside: p1 p2 p3 | q
    m = nin == 3
    t3 = tet[m]
    if len(t3):
        edges.append(np.stack([t3[:, [0, 3]], t3[:, [1, 3]], t3[:, [2, 3]]], 1))
        ref_in.append(t3[:, :3])
        ref_out.append(t3[:, [3]])
    # 2 inside: p1 p2 | q1 q2 -> quad (p1q1, p1q2, p2q2, p2q1)
    m = nin == 2
    t2 = tet[m]
    if len(t2):
        e11, e12, e22, e21 = t2[:, [0, 2]], t2[:, [0, 3]], t2[:, [1, 3]], t2[:, [1, 2]]
        edges.append(np.stack([e11, e12, e22], 1))
        edges.append(np.stack([e11, e22, e21], 1))
        ref_in += [t2[:, :2], t2[:, :2]]
        ref_out += [t2[:, 2:], t2[:, 2:]]
    E = np.concatenate(edges)                             # [T, 3, 2]
    E = np.sort(E, axis=2)                                # lower grid index first
    keys = E[..., 0] * (nx * ny * nz) + E[..., 1]
    uk, inv = np.unique(keys.reshape(-1), return_inverse=True)
    ga, gb = uk // (nx * ny * nz), uk % (nx * ny * nz)
    fa, fb = ff[ga], ff[gb]
    t = fa / (fa - fb)
    pa, pb = gpos(ga), gpos(gb)
    P = pa + t[:, None] * (pb - pa)
    F = inv.reshape(-1, 3).astype(np.int64)
    # orient: normal towards the outside corners
    rin = np.concatenate([gpos(r).mean(1) if r.shape[1] > 1 else gpos(r[:, 0]) for r in ref_in])
    rout = np.concatenate([gpos(r).mean(1) if r.shape[1] > 1 else gpos(r[:, 0]) for r in ref_out])
    nrm = np.cross(P[F[:, 1]] - P[F[:, 0]], P[F[:, 2]] - P[F[:, 0]])
    flip = np.einsum("ij,ij->i", nrm, rout - rin) < 0
    F[flip] = F[flip][:, ::-1]
    return _finish(P, F)


# ---------------------------------------------------------------------------
# signed distance functions
# ---------------------------------------------------------------------------

def _sd_box(x, y, z, lo, hi):
    """Signed 'max of slabs' function of an axis-aligned box (exact zero set)."""
    return np.maximum(np.maximum(np.maximum(lo[0] - x, x - hi[0]),
                                 np.maximum(lo[1] - y, y - hi[1])),
                      np.maximum(lo[2] - z, z - hi[2]))


def _sd_cyl_inf(x, y, z, p0, axis, r):
    """Distance to an infinite cylinder of radius r around line p0 + s*axis."""
    ax = np.asarray(axis, dtype=np.float64)
    ax = ax / np.linalg.norm(ax)
    dx, dy, dz = x - p0[0], y - p0[1], z - p0[2]
    s = dx * ax[0] + dy * ax[1] + dz * ax[2]
    qx, qy, qz = dx - s * ax[0], dy - s * ax[1], dz - s * ax[2]
    return np.sqrt(qx * qx + qy * qy + qz * qz) - r


def prismatic(h=1.67, size=(150.0, 100.0, 50.0), scale=1.0):
    """Prismatic part with an undercut (about 200k triangles at h=1.67):
    a ``size`` block with a T-slot along x (12 mm neck over a 24 x 8 mm
    head, open at both ends), four through-holes of diameter 8 mm tilted 20
    degrees from z, and one rectangular pocket in each of the +y and -y
    faces (undercuts with respect to +z and -z)."""
    L = np.asarray(size, dtype=np.float64) * scale
    sx, sy, sz = L
    cy = sy / 2

    def sdf(x, y, z):
        d = _sd_box(x, y, z, (0.0, 0.0, 0.0), L)
        big = 10.0 * sx
        neck = _sd_box(x, y, z, (-big, cy - 6 * scale, sz - 10 * scale), (big, cy + 6 * scale, big))
        head = _sd_box(x, y, z, (-big, cy - 12 * scale, sz - 18 * scale), (big, cy + 12 * scale, sz - 10 * scale))
        d = np.maximum(d, -np.minimum(neck, head))
        tilt = math.radians(20.0)
        ax = (math.sin(tilt), 0.0, math.cos(tilt))
        for hx in (0.2 * sx, 0.8 * sx):
            for hy in (0.2 * sy, 0.8 * sy):
                d = np.maximum(d, -_sd_cyl_inf(x, y, z, (hx, hy, sz / 2), ax, 4.0 * scale))
        for y0, y1 in ((-big, 15 * scale), (sy - 15 * scale, big)):
            pk = _sd_box(x, y, z, (0.37 * sx, y0, 0.2 * sz), (0.63 * sx, y1, 0.6 * sz))
            d = np.maximum(d, -pk)
        return d

    # grid offset by an irrational fraction of h so that no grid point lies
    # on an axis-aligned face (no zero-area slivers from exact zeros)
    off = h * 0.3819660112501051
    lo = -np.array([off, off * 1.1, off * 0.9]) - 2 * h
    hi = L + 2 * h
    return marching_tets(sdf, lo, hi, h)


def impeller(h=0.69, r_hub=40.0, r_tip=70.0, height=40.0, blades=12, wrap_deg=90.0,
             twist_deg=35.0, tip_gap=0.8, scale=1.0):
    """Axial impeller: a hub cylinder of radius ``r_hub`` carrying ``blades``
    helical blades out to ``r_tip``.  Each blade's mid-surface wraps
    ``wrap_deg`` about the axis over its height and twists ``twist_deg``
    from root to tip; the blade thickness is chosen so that the clear gap
    between neighbouring blades at the tip is ``tip_gap``.  About 2M
    triangles at h=0.69."""
    r_hub, r_tip, height = r_hub * scale, r_tip * scale, height * scale
    z0, z1 = 0.125 * height, 0.875 * height
    beta = math.radians(wrap_deg) / (z1 - z0)          # rad per mm along z
    gam = math.radians(twist_deg) / (r_tip - r_hub)    # rad per mm along r
    pitch = 2 * math.pi / blades
    # perpendicular spacing of neighbouring mid-surfaces at the tip radius
    spacing = r_tip * pitch / math.sqrt(1.0 + (r_tip * beta) ** 2 + (r_tip * gam) ** 2)
    thick = spacing - tip_gap * scale

    def sdf(x, y, z):
        r = np.sqrt(x * x + y * y)
        th = np.arctan2(y, x)
        hub = np.maximum(r - r_hub, np.maximum(-z, z - height))
        phase = th - beta * (z - z0) - gam * (r - r_hub)
        dphi = (phase / pitch + 0.5) % 1.0 - 0.5
        perp = r * dphi * pitch / np.sqrt(1.0 + (r * beta) ** 2 + (r * gam) ** 2)
        blade = np.abs(perp) - thick / 2
        blade = np.maximum(blade, np.maximum(r - r_tip, (r_hub - 1.0) - r))
        blade = np.maximum(blade, np.maximum(z0 - z, z - z1))
        return np.minimum(hub, blade)

    off = h * 0.3819660112501051
    ext = r_tip + 2 * h
    lo = np.array([-ext - off, -ext - off * 1.1, -2 * h - off * 0.9])
    hi = np.array([ext, ext, height + 2 * h])
    return marching_tets(sdf, lo, hi, h)


# ---------------------------------------------------------------------------
# families for batched / served workloads
# ---------------------------------------------------------------------------

def part_family(family, target_tris, rng):
    """One randomly sized part of ``family`` (0 pocket block, 1 prismatic,
    2 impeller) with each dimension scaled by U(0.7, 1.3) and a resolution
    chosen so that its triangle count is near ``target_tris``."""
    s = rng.uniform(0.7, 1.3, size=3)
    if family == 0:
        size = (100.0 * s[0], 60.0 * s[1], 40.0 * s[2])
        lv = max(0, int(round(math.log(max(target_tris, 28) / 28.0, 4))))
        w = 30.0 * min(s[0], s[1])
        return pocket_block(lv, size=size, width=w, depth=15.0 * s[2])
    if family == 1:
        sc = float(np.cbrt(s.prod()))
        # about 203k triangles at h = 1.67 mm and unit scale, T ~ 1/h^2
        return prismatic(h=1.67 * sc * math.sqrt(203000.0 / max(target_tris, 1000)), scale=sc)
    sc = float(np.cbrt(s.prod()))
    # about 1.93M triangles at h = 0.69 mm and unit scale
    return impeller(h=0.69 * sc * math.sqrt(1.93e6 / max(target_tris, 1000)), scale=sc)


def perturbed_part(subdiv, shift_mm, size=(100.0, 60.0, 40.0), width=30.0, depth=15.0, deepen_mm=0.0):
    """Pocket block whose pocket is moved ``shift_mm`` along x and sunk
    ``deepen_mm`` deeper.  The mesh has the same triangle list ``F`` as the
    unedited block, so a BVH built for one can be refitted to the other.
    Moving the pocket moves every vertex of the top face's ring around it;
    deepening moves only the pocket's walls and floor."""
    cx, cy = size[0] / 2 + shift_mm, size[1] / 2
    h = width / 2
    return box_with_pockets(size, (("+z", (cx - h, cx + h), (cy - h, cy + h), depth + deepen_mm),), subdiv)
