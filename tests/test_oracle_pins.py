"""Pins for the CPU oracle: each test checks it against something other than
itself -- published values, closed forms, exact rational arithmetic,
invariants, or brute force -- so that a dropped term, a wrong sign or index
or a transposed operand in the oracle fails here.  CPU only."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# helpers: exact arithmetic on fp32 inputs
# ---------------------------------------------------------------------------

def _fr(v):
    return [Fraction(float(x)) for x in np.asarray(v, np.float32)]


def _sub(a, b):
    return [x - y for x, y in zip(a, b)]


def _cross(u, v):
    return [u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]]


def _dot(u, v):
    return sum(x * y for x, y in zip(u, v))


def exact_pair(o, d, A, B, C):
    """Exact answer of 'does o + t d, t > 0, meet the closed triangle ABC'
    in rational arithmetic: returns True / False, or None on a boundary
    (the line through an edge or vertex, the crossing at the origin, or the
    ray lying in the plane)."""
    o, d, A, B, C = map(_fr, (o, d, A, B, C))
    a, b, c = _sub(A, o), _sub(B, o), _sub(C, o)
    U = _dot(_cross(b, c), d)
    V = _dot(_cross(c, a), d)
    W = _dot(_cross(a, b), d)
    s = [U, V, W]
    if any(x > 0 for x in s) and any(x < 0 for x in s):
        return False
    N = _cross(_sub(B, A), _sub(C, A))
    nd, na = _dot(N, d), _dot(N, a)
    if any(x == 0 for x in s):
        if nd != 0 and (na / nd) < 0:
            return False
        return None
    if nd == 0:
        return None
    t = na / nd
    if t == 0:
        return None
    return t > 0


# ---------------------------------------------------------------------------
# published values
# ---------------------------------------------------------------------------

def test_splitmix64_published_outputs(orc):
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "splitmix64.txt"))
            if ln.strip() and not ln.startswith("#")]
    g = 0x9E3779B97F4A7C15
    for k, val in rows:
        assert orc.splitmix64((int(k) * g) % 2 ** 64) == int(val, 16)


def test_classify_reproduces_paper_table_labels(orc):
    """Tables 1 and 2 print the indicators and the resulting label; the
    default thresholds must give the same labels."""
    for ln in open(os.path.join(GOLDEN, "paper_tables.txt")):
        if not ln.strip() or ln.startswith("#"):
            continue
        _, acc, sx, sy, sz, conc, label = ln.split()
        s = {"overall_access": float(acc), "axis_share": [float(sx), float(sy), float(sz)],
             "mean_conc": float(conc)}
        assert orc.classify(s) == (1 if label == "multi" else 0)


# ---------------------------------------------------------------------------
# Section 3.1: face preparation and direction set
# ---------------------------------------------------------------------------

def test_face_prep_right_hand_rule_and_area(orc):
    V = np.array([[0, 0, 0], [2, 0, 0], [0, 3, 0], [0, 0, 5]], np.float32)
    F = np.array([[0, 1, 2], [0, 2, 1], [0, 3, 1]], np.int32)
    n, a, c = orc.face_prep(V, F)
    assert np.array_equal(n[0], [0, 0, 1]) and np.array_equal(n[1], [0, 0, -1])
    assert np.array_equal(n[2], [0, 1, 0])          # (0,0,5)x(2,0,0) = (0,10,0)
    assert a[0] == 3.0 and a[2] == 5.0
    assert np.allclose(c[0], [2 / 3, 1.0, 0.0])


def test_direction_table_uniform_hemisphere(orc):
    N = 1024
    h64, h32 = orc.direction_table(N)
    assert np.allclose(np.linalg.norm(h64, axis=1), 1.0, atol=1e-15)
    assert np.allclose(np.linalg.norm(h32.astype(np.float64), axis=1), 1.0, atol=3e-7)
    z = h64[:, 2]
    assert np.all(z > 0) and np.all(z < 1) and np.all(np.diff(z) < 0)
    # z uniform on (0,1): the mean of z over the set is exactly 1/2, and any
    # z-band holds N*band points up to one (equal-area by Archimedes)
    assert abs(z.mean() - 0.5) < 1e-12
    for lo, hi in ((0.0, 0.25), (0.3, 0.7), (0.9, 1.0)):
        k = int(((z >= lo) & (z < hi)).sum())
        assert abs(k - N * (hi - lo)) <= 1
    # azimuth steps by the golden angle pi*(3-sqrt5)
    phi = np.unwrap(np.arctan2(h64[:, 1], h64[:, 0]))
    ga = math.pi * (3 - math.sqrt(5))
    assert np.allclose(np.diff(phi) % (2 * math.pi), ga, atol=1e-9)


def test_ray_directions_rotate_hemisphere_to_normal(orc):
    rng = np.random.default_rng(1)
    N = 256
    h64, _ = orc.direction_table(N)
    for _ in range(20):
        n = rng.normal(size=3)
        n = (n / np.linalg.norm(n)).astype(np.float32)
        d = orc.ray_dirs(n, N).astype(np.float64)
        # the local z component is the direction's projection on the normal
        assert np.allclose(d @ n.astype(np.float64), h64[:, 2], atol=2e-6)
        assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=2e-6)
        # angles between directions are preserved (a rotation)
        assert np.allclose(d @ d.T, h64 @ h64.T, atol=5e-6)
        # and it is a rotation, not a reflection: the map h -> d fitted over
        # the set has determinant +1 and takes the local z axis to n
        Q = np.linalg.lstsq(h64, d, rcond=None)[0].T
        assert abs(np.linalg.det(Q) - 1.0) < 1e-5
        assert np.allclose(Q[:, 2], n, atol=2e-6)
    # axis-aligned normal +z maps the table to itself up to a reflection
    d = orc.ray_dirs(np.array([0, 0, 1], np.float32), N)
    assert np.allclose(np.abs(d), np.abs(h64), atol=1e-7)


def test_origin_offset(orc):
    P = np.array([[10, 20, 30]], np.float32)
    n = np.array([[0, 0, 1]], np.float32)
    o = orc.ray_origins(P, n, 1e-4)
    assert o[0, 2] == np.float32(30.0 + 1e-4) and o[0, 0] == 10 and o[0, 1] == 20


# ---------------------------------------------------------------------------
# the occlusion predicate against exact rational arithmetic
# ---------------------------------------------------------------------------

def test_pair_matches_exact_rational_predicate(orc):
    rng = np.random.default_rng(7)
    checked = amb = 0
    for it in range(3000):
        A, B, C = rng.uniform(-5, 5, size=(3, 3)).astype(np.float32)
        o = rng.uniform(-8, 8, size=3).astype(np.float32)
        if it % 2:
            # aim at a point of the triangle's plane near (inside or just
            # outside) the triangle: many near-edge cases
            w = rng.uniform(-0.1, 1.1, size=3)
            w /= w.sum()
            tgt = w[0] * A + w[1] * B + w[2] * C
            d = (tgt - o).astype(np.float32)
            if it % 4 == 1:
                d = -d
        else:
            d = rng.normal(size=3).astype(np.float32)
        r = orc.pair(o, d, A, B, C)
        ex = exact_pair(o, d, A, B, C)
        if r == orc.AMB:
            amb += 1
            continue
        checked += 1
        assert ex is not None, (o, d, A, B, C)
        assert (r == orc.HIT) == ex, (r, ex, o, d, A, B, C)
    assert checked > 2900 and amb < 10


def test_pair_boundary_cases_are_ambiguous(orc):
    A = np.array([0, 0, 0], np.float32)
    B = np.array([4, 0, 0], np.float32)
    C = np.array([0, 4, 0], np.float32)
    down = np.array([0, 0, -1], np.float32)
    # exactly through an edge midpoint, a vertex, the hypotenuse
    for p in ([2, 0, 0], [0, 0, 0], [2, 2, 0], [0, 3, 0]):
        o = np.array(p, np.float32) + np.array([0, 0, 3], np.float32)
        assert exact_pair(o, down, A, B, C) is None
        assert orc.pair(o, down, A, B, C) == orc.AMB
    # clear interior hit, clear outside, hit behind the origin
    assert orc.pair(np.array([1, 1, 3], np.float32), down, A, B, C) == orc.HIT
    assert orc.pair(np.array([3, 3, 3], np.float32), down, A, B, C) == orc.MISS
    assert orc.pair(np.array([1, 1, -3], np.float32), down, A, B, C) == orc.MISS
    # origin on the plane inside the triangle: crossing at t = 0
    assert orc.pair(np.array([1, 1, 0], np.float32), down, A, B, C) == orc.AMB
    # the band (reading R6, tau*R = 4e-9 here since R = 4): a line within it
    # of an edge line is ambiguous on either side, one farther is decided;
    # the same for a crossing within it of the origin along the ray
    for p, expect in (([2, 1e-9, 3], orc.AMB), ([2, -1e-9, 3], orc.AMB), ([2, 1e-7, 3], orc.HIT),
                      ([2, -1e-7, 3], orc.MISS), ([1, 1, 1e-9], orc.AMB), ([1, 1, 1e-6], orc.HIT)):
        assert orc.pair(np.array(p, np.float32), down, A, B, C) == expect, p
    # ray in the plane of the triangle
    assert orc.pair(np.array([-1, 1, 0], np.float32), np.array([1, 0, 0], np.float32),
                    A, B, C) == orc.AMB
    # parallel and offset: clear miss
    assert orc.pair(np.array([-1, 1, 1e-3], np.float32), np.array([1, 0, 0], np.float32),
                    A, B, C) == orc.MISS


def test_bvh_matches_brute_force(orc):
    rng = np.random.default_rng(3)
    parts = [synth.pocket_block(2), synth.prismatic(h=6.0), synth.impeller(h=3.0),
             synth.icosphere(10.0, 2), synth.cavity_box(subdiv=1)]
    for V, F in parts:
        lo, hi = V.min(0), V.max(0)
        nr = 4000
        O = rng.uniform(lo - 5, hi + 5, size=(nr, 3)).astype(np.float32)
        D = rng.normal(size=(nr, 3)).astype(np.float32)
        # also rays from sampled surface points (the method's own rays)
        P, Nn, _, _ = orc.sample_area(V, F, 200, seed=5)
        Oh = orc.ray_origins(P, Nn, 1e-4)
        Dh = np.concatenate([orc.ray_dirs(Nn[i], 16) for i in range(200)])
        O = np.concatenate([O, np.repeat(Oh, 16, axis=0)])
        D = np.concatenate([D, Dh])
        s1 = orc.Mesh(V, F).cast_rays(O, D)
        s2 = orc.Mesh(V, F, brute=True).cast_rays(O, D)
        assert np.array_equal(s1, s2)
        assert (s1 == orc.HIT).any() and (s1 == orc.MISS).any()


# ---------------------------------------------------------------------------
# closed forms on whole parts
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("part", ["cube", "icosphere"])
def test_convex_part_fully_accessible(orc, part):
    """Offset origin strictly outside the supporting plane, direction into
    the open half-space, polytope behind the plane: every ray escapes."""
    V, F = synth.cube(20.0, 2) if part == "cube" else synth.icosphere(10.0, 3)
    P, Nn, _, _ = orc.sample_area(V, F, 300, seed=11)
    bits, amb, cnt = orc.Mesh(V, F).hemisphere(P, Nn, 128)
    assert (cnt == 128).all() and not amb.any()


def test_sealed_cavity_fully_blocked(orc):
    V, F = synth.cavity_box(subdiv=1)
    n, a, _ = orc.face_prep(V, F)
    P, Nn, fc, _ = orc.sample_area(V, F, 400, seed=2)
    inner = (P.min(1) > 5) & (P.max(1) < 35)          # points on the void's faces
    assert inner.sum() > 50
    bits, amb, cnt = orc.Mesh(V, F).hemisphere(P[inner], Nn[inner], 64)
    assert (cnt == 0).all() and not amb.any()


def _pocket_expected(o, d, rect, ztop):
    """Exact visibility of a ray from inside a box pocket whose opening is
    the rectangle ``rect`` at height ztop: it escapes iff it crosses the
    top plane strictly inside the opening.  None on the rim."""
    ox, oy, oz = (Fraction(float(x)) for x in o)
    dx, dy, dz = (Fraction(float(x)) for x in d)
    if dz <= 0:
        return False
    t = (Fraction(ztop) - oz) / dz
    x, y = ox + t * dx, oy + t * dy
    (x0, x1), (y0, y1) = rect
    if x0 < x < x1 and y0 < y < y1:
        return True
    if x0 <= x <= x1 and y0 <= y <= y1:
        return None
    return False


def test_pocket_block_matches_exact_visibility(orc):
    """The whole visibility bitmask of the pocket block (configuration 1
    geometry) is analytic: points on the outer faces see their entire
    hemisphere; points on the pocket floor and walls see exactly the
    directions that leave through the opening."""
    V, F = synth.pocket_block(3)
    N = 256
    P, Nn, fc, _ = orc.sample_area(V, F, 1000, seed=0)
    bits, amb, cnt = orc.Mesh(V, F).hemisphere(P, Nn, N)
    O = orc.ray_origins(P, Nn, 1e-4)
    rect = ((35.0, 65.0), (15.0, 45.0))
    in_pocket = (P[:, 2] < 40) & (P[:, 2] >= 25) & (P[:, 0] >= 35) & (P[:, 0] <= 65) & \
        (P[:, 1] >= 15) & (P[:, 1] <= 45) & ~((P[:, 2] == 0))
    assert in_pocket.sum() > 20
    n_amb = n_cmp = 0
    for i in range(len(P)):
        row = np.unpackbits(bits[i].view(np.uint8), bitorder="little")[:N].astype(bool)
        arow = np.unpackbits(amb[i].view(np.uint8), bitorder="little")[:N].astype(bool)
        if not in_pocket[i]:
            assert row.all() and not arow.any()
            continue
        D = orc.ray_dirs(Nn[i], N)
        for j in range(N):
            ex = _pocket_expected(O[i], D[j], rect, 40.0)
            if arow[j]:
                n_amb += 1
                continue
            n_cmp += 1
            assert ex is not None and row[j] == ex, (i, j)
    assert n_cmp > 5000 and n_amb <= 3


def test_area_weighted_accessibility_equals_exact_rational(orc):
    """Section 3.1's area-weighted overall accessibility, pinned on the
    pocket block in the paper's centroid mode: every face is axis-aligned,
    so its exact area is |(B-A) x (C-A)| / 2 with one non-zero component,
    and every ray's visibility is the exact rational test through the
    opening.  The weighted mean sum A_f c_f / (N sum A_f) is then an exact
    rational number; the oracle's summary must give it in FP64, and its
    whole chain (cast + summary) within the 1e-4 accessibility bar.  The
    unweighted mean and the n*N denominator both miss it by far, so
    ignoring the weights or the weight sum fails here."""
    V, F = synth.pocket_block(2)
    N = 64
    P, Nn, fc, w = orc.sample_centroid(V, F)
    O = orc.ray_origins(P, Nn, 1e-4)
    rect = ((35.0, 65.0), (15.0, 45.0))
    Vq = [[Fraction(float(x)) for x in v] for v in V]
    areas, counts = [], []
    for f in range(len(F)):
        A, B, C = (Vq[int(k)] for k in F[f])
        c = _cross(_sub(B, A), _sub(C, A))
        nz = [x for x in c if x != 0]
        assert len(nz) == 1
        areas.append(abs(nz[0]) / 2)
        assert abs(float(areas[-1]) - w[f]) <= 1e-12 * float(areas[-1])
        x, y, z = (float(t) for t in P[f])
        if not (25.0 <= z < 40.0 and 35.0 <= x <= 65.0 and 15.0 <= y <= 45.0):
            counts.append(N)
            continue
        D = orc.ray_dirs(Nn[f], N)
        ex = [_pocket_expected(O[f], D[j], rect, 40.0) for j in range(N)]
        assert all(e is not None for e in ex)
        counts.append(sum(1 for e in ex if e))
    cnt = np.array(counts, np.int64)
    assert 0 < (cnt < N).sum() < len(F)
    exact = sum(a * c for a, c in zip(areas, counts)) / (N * sum(areas))
    zero = np.zeros(len(F))
    s = orc.summary(cnt, np.zeros(len(F), np.int8), zero, N, weight=w)
    assert abs(s["overall_access"] - float(exact)) <= 1e-12
    # the pin discriminates: no weights, or n*N as the denominator
    assert abs(float(Fraction(int(cnt.sum()), N * len(F))) - float(exact)) > 1e-2
    assert abs(float(sum(a * c for a, c in zip(areas, counts)) / (N * len(F))) - float(exact)) > 1e-2
    # the oracle's own chain: its cast's counts through the same summary
    _, amb, ocnt = orc.Mesh(V, F).hemisphere(P, Nn, N)
    so = orc.summary(ocnt, np.zeros(len(F), np.int8), zero, N, weight=w)
    assert abs(so["overall_access"] - float(exact)) <= 1e-4


def test_pocket_floor_centre_cone_fraction(orc):
    """Floor centre of a square pocket of width w and depth D: the visible
    cone has solid angle 4*asin(w^2/(w^2+4D^2)) (the square-pyramid
    formula), so the visible fraction of the hemisphere tends to
    4*asin(w^2/(w^2+4D^2))/(2*pi); for w = 2D this is exactly 1/3."""
    for w, D in ((30.0, 15.0), (20.0, 25.0)):
        V, F = synth.box_with_pockets((100.0, 60.0, 40.0),
                                      (("+z", (50 - w / 2, 50 + w / 2), (30 - w / 2, 30 + w / 2), D),))
        P = np.array([[50.0, 30.0, 40.0 - D]], np.float32)
        Nn = np.array([[0, 0, 1]], np.float32)
        N = 65536
        bits, amb, cnt = orc.Mesh(V, F).hemisphere(P, Nn, N)
        frac = cnt[0] / N
        expect = 4 * math.asin(w * w / (w * w + 4 * D * D)) / (2 * math.pi)
        assert abs(frac - expect) < 1e-3, (frac, expect)
    assert abs(4 * math.asin(0.5) / (2 * math.pi) - 1 / 3) < 1e-15


# ---------------------------------------------------------------------------
# sampling
# ---------------------------------------------------------------------------

def test_area_sampling_on_faces_and_proportional_to_area(orc):
    V, F = synth.box_with_pockets((4.0, 2.0, 1.0), ())
    n_f, area, _ = orc.face_prep(V, F)
    P, Nn, fc, w = orc.sample_area(V, F, 60000, seed=3)
    # each point lies on its face: barycentric coordinates >= 0 (up to fp32)
    A, B, C = (V[F[fc, k]].astype(np.float64) for k in range(3))
    p = P.astype(np.float64)
    e1, e2, q = B - A, C - A, p - A
    d00, d01, d11 = (e1 * e1).sum(1), (e1 * e2).sum(1), (e2 * e2).sum(1)
    d20, d21 = (q * e1).sum(1), (q * e2).sum(1)
    den = d00 * d11 - d01 * d01
    v = (d11 * d20 - d01 * d21) / den
    ww = (d00 * d21 - d01 * d20) / den
    assert (v > -1e-6).all() and (ww > -1e-6).all() and (v + ww < 1 + 1e-6).all()
    # uniform within the triangle: each barycentric coordinate has density
    # 2(1 - u) on [0, 1], so a quarter of the points lie where it exceeds 1/2
    # (the corner triangle cut off by the mid-edges); 5 sigma at 60,000 points
    for u in (1.0 - v - ww, v, ww):
        assert abs((u > 0.5).mean() - 0.25) < 5 * math.sqrt(0.25 * 0.75 / len(P))
    assert np.array_equal(Nn, n_f[fc])
    # chi-square of per-face counts against the area distribution
    cnt = np.bincount(fc, minlength=len(F))
    exp = len(P) * area / area.sum()
    chi2 = ((cnt - exp) ** 2 / exp).sum()
    assert chi2 < len(F) + 6 * math.sqrt(2 * len(F))
    # deterministic in the seed
    P2, _, fc2, _ = orc.sample_area(V, F, 60000, seed=3)
    assert np.array_equal(P, P2) and np.array_equal(fc, fc2)
    P3, _, _, _ = orc.sample_area(V, F, 60000, seed=4)
    assert not np.array_equal(P, P3)


def test_centroid_sampling(orc):
    V, F = synth.pocket_block(1)
    P, Nn, fc, w = orc.sample_centroid(V, F)
    assert len(P) == len(F) and np.array_equal(fc, np.arange(len(F)))
    ref = V[F].astype(np.float64).mean(1)
    assert np.allclose(P, ref, atol=1e-5)
    assert abs(w.sum() - (2 * (100 * 60 + 100 * 40 + 60 * 40) + 4 * 30 * 15)) < 1e-6


# ---------------------------------------------------------------------------
# Section 3.3: variability, classification, setups
# ---------------------------------------------------------------------------

def test_open_flat_face_axis_and_concentration(orc):
    """Open face with normal +z: dominant axis z; mode-0 concentration tends
    to 1/3 (the +z cube-face region is 1/3 of the hemisphere's area), mode-1
    concentration to 1/2 (mean height of a uniform hemisphere)."""
    N = 8192
    Nn = np.array([[0, 0, 1]], np.float32)
    bits = np.full((1, N // 32), 0xFFFFFFFF, np.uint32)
    M, ac, dom, conc0, cnt = orc.variability(bits, Nn, N, conc_mode=0)
    _, _, _, conc1, _ = orc.variability(bits, Nn, N, conc_mode=1)
    assert dom[0] == 2 and cnt[0] == N
    assert abs(conc0[0] - 1 / 3) < 2e-3 and abs(conc1[0] - 0.5) < 1e-4
    # tilted normals: the dominant axis follows the largest normal component
    for n in ([1, 0, 0], [0, -1, 0], [0.6, 0.0, -0.8]):
        Nn = np.array([n], np.float32)
        _, _, dom, _, _ = orc.variability(bits, Nn, N)
        assert dom[0] == int(np.argmax(np.abs(n)))
    # a normal along another axis sees the same two limits (a permutation of
    # the axes maps the +z hemisphere onto it)
    for n in ([1, 0, 0], [0, -1, 0]):
        Nn = np.array([n], np.float32)
        _, _, _, c0, _ = orc.variability(bits, Nn, N, conc_mode=0)
        _, _, _, c1, _ = orc.variability(bits, Nn, N, conc_mode=1)
        assert abs(c0[0] - 1 / 3) < 2e-3 and abs(c1[0] - 0.5) < 1e-4
    # only a cone of half-angle 30 degrees about the normal visible: in every
    # visible direction the normal's axis is the largest component (cos 30 >
    # sin 30), so the mode-0 concentration is exactly 1, and the mode-1 one
    # is the mean height of the cone's directions
    h64, _ = orc.direction_table(N)
    cone = h64[:, 2] > math.cos(math.pi / 6)
    cbits = np.packbits(cone.astype(np.uint8), bitorder="little").view(np.uint32)[None, :]
    for n, axis in (([1, 0, 0], 0), ([0, -1, 0], 1)):
        Nn = np.array([n], np.float32)
        _, _, dom, c0, cnt = orc.variability(cbits, Nn, N, conc_mode=0)
        _, _, _, c1, _ = orc.variability(cbits, Nn, N, conc_mode=1)
        assert dom[0] == axis and cnt[0] == cone.sum() and c0[0] == 1.0
        assert abs(c1[0] - h64[cone, 2].mean()) < 1e-6


def test_deep_hole_concentration_tends_to_one(orc):
    V, F = synth.deep_hole(width=2.0, depth=38.0)
    P = np.array([[10.0, 10.0, 2.0]], np.float32)
    Nn = np.array([[0, 0, 1]], np.float32)
    N = 4096
    bits, amb, cnt = orc.Mesh(V, F).hemisphere(P, Nn, N)
    assert 0 < cnt[0] < N * 0.01
    _, _, dom, conc, _ = orc.variability(bits, Nn, N)
    assert dom[0] == 2 and conc[0] == 1.0


def test_summary_shares_sum_to_one(orc):
    V, F = synth.pocket_block(2)
    P, Nn, fc, w = orc.sample_area(V, F, 500, seed=1)
    bits, amb, cnt = orc.Mesh(V, F).hemisphere(P, Nn, 64)
    M, ac, dom, conc, c2 = orc.variability(bits, Nn, 64)
    assert np.array_equal(c2, cnt)
    s = orc.summary(cnt, dom, conc, 64)
    assert abs(sum(s["axis_share"]) - 1.0) < 1e-12
    assert s["n_counted"] + s["n_zero_visible"] == 500
    assert abs(s["overall_access"] - cnt.sum() / (500 * 64)) < 1e-15


def test_summary_worked_example(orc):
    """Four points, N = 8, one with nothing visible: the shares and the mean
    concentration are over the three counted points, the accessibility over
    all four (weighted: sum w c / (N sum w))."""
    cnt = np.array([0, 6, 3, 8], np.int64)
    dom = np.array([-1, 2, 0, 2], np.int8)
    conc = np.array([0.0, 0.5, 1.0, 0.25])
    s = orc.summary(cnt, dom, conc, 8)
    assert s["axis_share"] == [1 / 3, 0.0, 2 / 3]
    assert s["mean_conc"] == 1.75 / 3 and s["n_counted"] == 3 and s["n_zero_visible"] == 1
    assert s["overall_access"] == 17 / 32 and s["overall_access_unweighted"] == 17 / 32
    sw = orc.summary(cnt, dom, conc, 8, weight=np.array([1.0, 2.0, 3.0, 4.0]))
    assert abs(sw["overall_access"] - 53 / 80) <= 1e-15 and sw["overall_access_unweighted"] == 17 / 32


def test_classify_any_indicator_suffices(orc):
    """Section 3.3: the part is multi-axis if any one threshold is crossed."""
    base = {"overall_access": 0.70, "axis_share": [0.50, 0.25, 0.25], "mean_conc": 0.30}
    assert orc.classify(base) == 0
    for key, val in (("overall_access", 0.59), ("axis_share", [0.44, 0.28, 0.28]), ("mean_conc", 0.42)):
        s = dict(base)
        s[key] = val
        assert orc.classify(s) == 1, key


def test_travel_closed_form(orc):
    """Tool travel to the bounding box along each machining direction: the
    box [0,100] x [0,60] x [0,40] and the point (10, 20, 30), in the part's
    frame and in a frame whose axes X', Y', Z' are the part's y, z, x."""
    V = np.array([[x, y, z] for x in (0, 100) for y in (0, 60) for z in (0, 40)], np.float32)
    P = np.array([[10, 20, 30]], np.float32)
    assert np.array_equal(orc.travel(V, P)[0], [90, 10, 40, 20, 10, 30])
    frame = np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]], np.float32)      # columns: y, z, x
    assert np.array_equal(orc.travel(V, P, frame=frame.ravel())[0], [40, 20, 10, 30, 90, 10])


def test_face_classes_worked_example(orc):
    """Section 3.3: directions whose travel exceeds the tool length are
    discarded (travel equal to it is kept); a face with a kept direction is
    viable, one whose accessible directions were all discarded
    over-threshold, one with none fully inaccessible; fixture faces are
    excluded whatever their access."""
    mask = np.array([0b000001, 0b000001, 0, 0b010000, 0b100010], np.uint8)
    trav = np.full((5, 6), 99.0, np.float32)
    trav[0, 0], trav[1, 0], trav[3, 4], trav[4, 1], trav[4, 5] = 10.0, 10.5, 1.0, 20.0, 5.0
    face = np.array([0, 1, 2, 3, 4], np.int32)
    fixture = np.array([False, False, False, True, False])
    cls, reach = orc.face_classes(mask, trav, face, fixture, 10.0)
    assert cls.tolist() == [0, 1, 2, 3, 0]
    assert reach[0] == 0b000001 and reach[1] == 0 and reach[4] == 0b100000


def test_cover_tie_rules(orc):
    """Readings of the covers' ties: the exact cover takes the smallest
    bitmask among the smallest sets, the greedy cover the lower axis."""
    assert orc.setups_exact([0b011, 0b011]) == (1, 0b001)
    assert orc.setups_exact([0b0110, 0b1100]) == (1, 0b0100)
    assert orc.setups_greedy([0b011]) == (1, 0b001)
    assert orc.setups_greedy([0b0011, 0b1100]) == (2, 0b0101)


def test_setups_on_hand_built_parts(orc):
    # a cube: every face lies on the bounding box -> all fixture -> 0 setups
    V, F = synth.cube(20.0, 1)
    fx = orc.fixture_faces(V, F)
    assert fx.all()
    # pocket block: outer faces are fixture faces; pocket floor and walls
    # are reachable from +Z only -> one setup (+Z, bit 4)
    for V, F, expect in ((*synth.pocket_block(2), 1),
                         (*synth.box_with_pockets((100.0, 60.0, 40.0), (
                             ("+z", (35.0, 65.0), (15.0, 45.0), 15.0),
                             ("+x", (10.0, 50.0), (10.0, 30.0), 10.0))), 2)):
        P, Nn, fc, w = orc.sample_centroid(V, F)
        m, am = orc.Mesh(V, F).orthogonal(P, Nn)
        trav = orc.travel(V, P)
        fx = orc.fixture_faces(V, F)
        cls, reach = orc.face_classes(m, trav, fc, fx, tool_length=50.0)
        viable = reach[cls == 0]
        assert (cls != 2).all()
        k, S = orc.setups_exact(viable)
        assert k == expect
        if expect == 1:
            assert S == 1 << 4
        g, _ = orc.setups_greedy(viable)
        assert g >= k
    # a tool shorter than the pocket depth makes its floor over-threshold
    V, F = synth.pocket_block(1)
    P, Nn, fc, w = orc.sample_centroid(V, F)
    m, _ = orc.Mesh(V, F).orthogonal(P, Nn)
    cls, reach = orc.face_classes(m, orc.travel(V, P), fc, orc.fixture_faces(V, F), 10.0)
    floor = (np.abs(P[:, 2] - 25.0) < 1e-6)
    assert (cls[floor] == 1).all()


def test_greedy_cover_can_exceed_exact(orc):
    masks = [0b011, 0b011, 0b101, 0b101, 0b010, 0b100]
    assert orc.setups_exact(masks) == (2, 0b110)
    assert orc.setups_greedy(masks)[0] == 3


def test_orthogonal_masks_permute_under_quarter_turns(orc):
    """A quarter turn about z maps +X->+Y, +Y->-X; the six-axis masks of the
    rotated part are the permuted masks of the original, exactly."""
    V, F = synth.box_with_pockets((100.0, 60.0, 40.0), (
        ("+z", (35.0, 65.0), (15.0, 45.0), 15.0), ("-y", (20.0, 40.0), (5.0, 15.0), 10.0)), subdiv=1)
    P, Nn, fc, w = orc.sample_centroid(V, F)
    m0, a0 = orc.Mesh(V, F).orthogonal(P, Nn)
    Vr = synth.rotate90(V, 2)
    Pr, Nr, _, _ = orc.sample_centroid(Vr, F)
    m1, a1 = orc.Mesh(Vr, F).orthogonal(Pr, Nr)
    # rotation about z: x' = -y, y' = x.  +X(0)->+Y(2), -X(1)->-Y(3),
    # +Y(2)->-X(1), -Y(3)->+X(0), Z unchanged
    perm = {0: 2, 1: 3, 2: 1, 3: 0, 4: 4, 5: 5}
    ok = (a0 == 0) & (a1 == 0)
    mapped = np.zeros_like(m0)
    for s, t in perm.items():
        mapped |= ((m0 >> s) & 1) << t
    assert ok.mean() > 0.95
    assert np.array_equal(mapped[ok], m1[ok])


def test_accessibility_rotation_invariant(orc):
    V, F = synth.pocket_block(2)
    Vr = synth.rotate90(V, 0)
    out = []
    for VV in (V, Vr):
        P, Nn, fc, w = orc.sample_centroid(VV, F)
        _, _, cnt = orc.Mesh(VV, F).hemisphere(P, Nn, 1024)
        out.append(orc.summary(cnt, np.zeros(len(cnt), np.int8), np.zeros(len(cnt)), 1024, w))
    assert abs(out[0]["overall_access"] - out[1]["overall_access"]) < 5e-3


# ---------------------------------------------------------------------------
# points kept on their faces (re-analysis of an edited part)
# ---------------------------------------------------------------------------

def test_points_on_faces_reproduce_sampling_and_follow_the_edit(orc):
    V0, F = synth.perturbed_part(2, 0.0)
    V1, F1 = synth.perturbed_part(2, 3.0)
    assert np.array_equal(F, F1) and not np.array_equal(V0, V1)
    P, Nn, f, _ = orc.sample_area(V0, F, 3000, seed=7)
    # on the unedited part: exactly the sampler's points
    Q, Qn = orc.sample_on_faces(V0, F, f, seed=7)
    assert np.array_equal(Q, P) and np.array_equal(Qn, Nn)
    # on the edited part: same barycentric position on the moved triangle
    R, Rn = orc.sample_on_faces(V1, F, f, seed=7)
    tri = V1.astype(np.float64)[F[f]]
    e1, e2, d = tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0], R.astype(np.float64) - tri[:, 0]
    # barycentrics by least squares: both within [0, 1] and summing to <= 1
    G = np.stack([e1, e2], axis=2)
    lam = np.linalg.lstsq(G[0], d[0], rcond=None)[0]
    for k in range(0, len(f), 97):
        lam = np.linalg.lstsq(G[k], d[k], rcond=None)[0]
        assert lam.min() >= -1e-5 and lam.sum() <= 1 + 1e-5
    moved = (V0[F[f]] != V1[F[f]]).any(axis=(1, 2))
    assert moved.any() and (~moved).any()
    assert np.array_equal(R[~moved], P[~moved]) and not np.array_equal(R[moved], P[moved])
    n1, _, _ = orc.face_prep(V1, F)
    assert np.array_equal(Rn, n1[f])
    # centroid mode: the moved centroids
    C, Cn = orc.sample_on_faces(V1, F, np.arange(len(F), dtype=np.int32), centroid=True)
    c1, cn1, _, _ = orc.sample_centroid(V1, F)
    assert np.array_equal(C, c1) and np.array_equal(Cn, cn1)
    with pytest.raises(ValueError):
        orc.sample_on_faces(V1, F, np.array([0, len(F)], np.int32))
