"""Pins for the oracle's automatic-frame functions (oracle/frames.py) against
closed forms, exact rotations and brute force -- nothing here re-types the
oracle's formulas."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import frames as fr


def _lines_match(A, B, tol):
    """Columns of A equal columns of B up to sign and order."""
    M = np.abs(np.asarray(A, np.float64).T @ np.asarray(B, np.float64))
    return np.allclose(np.sort(M, axis=1)[:, -1], 1.0, atol=tol) and \
        sorted(np.argmax(M, axis=1).tolist()) == [0, 1, 2]


def test_triangle_second_moment_closed_form():
    # unit right triangle: int x^2 = int y^2 = 1/12, int xy = 1/24, area 1/2
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    F = np.array([[0, 1, 2]], np.int32)
    S0, S1, S2, r = fr.surface_moments(V, F, ref=np.zeros(3))
    assert S0 == 0.5
    assert np.allclose(S1, [1 / 6, 1 / 6, 0], rtol=0, atol=1e-15)
    assert np.allclose(S2, [[1 / 12, 1 / 24, 0], [1 / 24, 1 / 12, 0], [0, 0, 0]], rtol=0, atol=1e-15)
    # about its centroid (1/3, 1/3, 0) -- away from the bounding-box midpoint
    # the moments are taken from -- by the parallel-axis theorem:
    # 1/12 - (1/2)(1/3)^2 = 1/36 and 1/24 - (1/2)(1/3)(1/3) = -1/72
    M, cen = fr.central_second_moment(V, F)
    assert np.allclose(cen, [1 / 3, 1 / 3, 0], rtol=0, atol=1e-15)
    assert np.allclose(M, [[1 / 36, -1 / 72, 0], [-1 / 72, 1 / 36, 0], [0, 0, 0]], rtol=0, atol=1e-15)


@pytest.mark.parametrize("subdiv", [0, 2])
def test_box_surface_moment_closed_form(subdiv):
    # box [-a,a] x [-b,b] x [-c,c]: int over the surface of x^2 dA =
    # 8 a^2 b c + 8 a^3 (b + c) / 3, and cyclically; no products of inertia
    V, F = synth.box_with_pockets((100.0, 60.0, 40.0), pockets=(), subdiv=subdiv)
    M, cen = fr.central_second_moment(V, F)
    a, b, c = 50.0, 30.0, 20.0
    want = [8 * a * a * b * c + 8 * a ** 3 * (b + c) / 3,
            8 * b * b * a * c + 8 * b ** 3 * (a + c) / 3,
            8 * c * c * a * b + 8 * c ** 3 * (a + b) / 3]
    assert np.allclose(np.diag(M), want, rtol=1e-12)
    assert np.abs(M - np.diag(np.diag(M))).max() <= 1e-9 * want[0]
    assert np.allclose(cen, [50.0, 30.0, 20.0], rtol=0, atol=1e-9)


def test_principal_frame_follows_a_rotation():
    V, F = synth.box_with_pockets((100.0, 60.0, 40.0), pockets=(), subdiv=1)
    R = synth.rotation(25.0, -40.0, 70.0)
    P, w = fr.principal_frame(synth.rotate(V, R), F)
    assert P is not None                             # three distinct eigenvalues
    # columns = rotated x, y, z (largest extent first), eigenvalues invariant
    assert np.allclose(np.abs(np.sum(P * R, axis=0)), 1.0, atol=2e-6)
    a, b, c = 50.0, 30.0, 20.0
    want = [8 * a * a * b * c + 8 * a ** 3 * (b + c) / 3, 8 * b * b * a * c + 8 * b ** 3 * (a + c) / 3,
            8 * c * c * a * b + 8 * c ** 3 * (a + b) / 3]
    assert np.allclose(w, want, rtol=1e-5)
    assert abs(np.linalg.det(P) - 1.0) < 1e-12 and np.allclose(P.T @ P, np.eye(3), atol=1e-12)


def test_principal_frame_absent_when_undetermined():
    V, F = synth.cube(20.0, 1)                       # three equal eigenvalues
    assert fr.principal_frame(V, F)[0] is None
    V, F = synth.box_with_pockets((60.0, 60.0, 20.0), pockets=(), subdiv=1)   # two equal
    assert fr.principal_frame(V, F)[0] is None


def test_normals_frame_of_a_rotated_box():
    # largest faces are the z faces (100 x 60), then the y faces (100 x 40)
    V, F = synth.box_with_pockets((100.0, 60.0, 40.0), pockets=(), subdiv=1)
    R = synth.rotation(-15.0, 35.0, 10.0)
    Nf = fr.normals_frame(synth.rotate(V, R), F)
    assert Nf is not None
    assert abs(abs(Nf[:, 2] @ R[:, 2]) - 1.0) < 1e-6     # Z' along the rotated z
    assert abs(abs(Nf[:, 0] @ R[:, 1]) - 1.0) < 1e-6     # X' along the rotated y
    assert abs(np.linalg.det(Nf) - 1.0) < 1e-12


def test_normal_cells_brute_force():
    rng = np.random.default_rng(3)
    n = rng.normal(size=(400, 3))
    n /= np.linalg.norm(n, axis=1)[:, None]
    n = n.astype(np.float32)
    cells, _ = fr.normal_cells(n)
    for v, c in zip(n.astype(np.float64), cells):
        # the cell is a function of the line: -n falls in the same cell
        k = int(np.argmax(np.abs(v)))
        u = v if v[k] > 0 else -v
        uu = Fraction(float(u[(k + 1) % 3])) / Fraction(float(u[k]))
        vv = Fraction(float(u[(k + 2) % 3])) / Fraction(float(u[k]))
        i = min(31, math.floor((uu + 1) * 16))
        j = min(31, math.floor((vv + 1) * 16))
        assert c == (k * 32 + i) * 32 + j or abs(float(uu) * 16 + 16 - round(float(uu) * 16 + 16)) < 1e-12 \
            or abs(float(vv) * 16 + 16 - round(float(vv) * 16 + 16)) < 1e-12
    assert np.array_equal(fr.normal_cells(-n)[0], cells)


def test_quantised_areas_are_llround():
    rng = np.random.default_rng(5)
    A = np.concatenate([rng.random(200) * 10.0, [10.0, 0.0, 5.0, 2.5 / 2 ** 32 * 10.0]])
    q = fr.quantised_areas(A)
    amax = Fraction(float(A.max()))
    for a, qq in zip(A, q):
        # x = fl(fl(a / amax) * 2^32); llround rounds halves away from zero
        x = Fraction(float(np.float64(a) / np.float64(A.max()))) * 2 ** 32
        want = math.floor(x + Fraction(1, 2))
        assert qq == want
    assert q.max() == 2 ** 32 and amax > 0


def test_snap_and_frame_from_are_orthonormal_right_handed():
    rng = np.random.default_rng(9)
    for _ in range(50):
        u, v = rng.normal(size=3), rng.normal(size=3)
        for ca, cb in ((0, 1), (2, 0), (1, 2), (1, 0)):
            R = fr.frame_from(ca, u, cb, v)
            assert np.allclose(R.T @ R, np.eye(3), atol=1e-14)
            assert abs(np.linalg.det(R) - 1.0) < 1e-14
            # column ca along u (as a line), within the 2^-20 snapping
            assert abs(abs(R[:, ca] @ u / np.linalg.norm(u)) - 1.0) < 1e-10
    # the snapped vector's largest component is positive; -u gives the same
    w = fr.snap([-0.3, 0.9, -0.1])
    assert w[1] > 0 and fr.snap([0.3, -0.9, 0.1]) == w


def test_box_search_recovers_a_rational_rotation():
    # turn a box about z by exactly the angle of step j0 (tan(theta/2) = j0/128)
    V, F = synth.box_with_pockets((100.0, 60.0, 40.0), pockets=(), subdiv=0)
    for j0 in (0, 1, 37, 90, 127):
        t = Fraction(j0, 128)
        cs, sn = float((1 - t * t) / (1 + t * t)), float(2 * t / (1 + t * t))
        R = np.array([[cs, -sn, 0.0], [sn, cs, 0.0], [0.0, 0.0, 1.0]])
        Vr = synth.rotate(V, R)
        a, j, G, vol = fr.box_search(Vr, np.eye(3))
        assert (a, j) == ((0, 0) if j0 == 0 else (2, j0))
        assert abs(vol - 240000.0) <= 1e-4 * 240000.0


def test_box_search_is_the_brute_force_minimum():
    V, F = synth.prismatic(h=8.0)
    B = synth.rotation(5.0, 10.0, 20.0)
    a, j, G, vol = fr.box_search(V, B)
    # independent evaluation: numpy matrix products and trig of the angle
    best = None
    for aa in range(3):
        for jj in range(128):
            th = 2.0 * math.atan(jj / 128.0)
            b, c = (aa + 1) % 3, (aa + 2) % 3
            Bf = np.asarray(B, np.float32).astype(np.float64)
            Gm = Bf.copy()
            Gm[:, b] = math.cos(th) * Bf[:, b] + math.sin(th) * Bf[:, c]
            Gm[:, c] = math.cos(th) * Bf[:, c] - math.sin(th) * Bf[:, b]
            q = V.astype(np.float64) @ Gm
            v = float(np.prod(q.max(0) - q.min(0)))
            if best is None or v < best[0] * (1 - 1e-9):
                best = (v, aa, jj)
    assert (a, j) == best[1:] and abs(vol - best[0]) <= 1e-9 * best[0]


def test_select_frame_order():
    """F6 on hand-made scores: fewest setups first, then fewest over-threshold
    plus inaccessible points, then the smallest box volume, then the lowest
    index."""
    def pick(vol, setups, bad):
        cands = [{"volume": v} for v in vol]
        evals = [{"setups_exact": k, "class_counts": [0, b, 0, 0]} for k, b in zip(setups, bad)]
        return fr.select_frame(cands, evals)
    assert pick([1.0, 9.0, 8.0], [2, 1, 1], [0, 4, 2]) == 2        # setups, then flagged points
    assert pick([1.0, 9.0, 8.0], [2, 1, 1], [0, 1, 2]) == 1        # flagged points before volume
    assert pick([5.0, 3.0, 4.0], [1, 1, 1], [0, 0, 0]) == 1        # then volume
    assert pick([3.0, 3.0, 3.0], [1, 1, 1], [2, 2, 2]) == 0        # then the index


def test_auto_frame_undoes_a_rotation():
    # a rotated pocket block: the chosen frame gives the setups, classes and
    # fixture exclusion of the unrotated block in the identity frame
    V, F = synth.pocket_block(2)
    P0, N0, f0, _ = oracle.sample_area(V, F, 600, seed=0)
    ref = fr.evaluate_frame(oracle.Mesh(V, F), V, F, P0, N0, f0, None, 100.0)
    for ang in ((30.0, 0.0, 20.0), (10.0, 45.0, 0.0)):
        R = synth.rotation(*ang)
        Vr = synth.rotate(V, R)
        P, Nn, f, _ = oracle.sample_area(Vr, F, 600, seed=0)
        cands, evals, best = fr.auto_frame(Vr, F, P, Nn, f, 100.0)
        e = evals[best]
        assert cands[0]["source"] == fr.GIVEN
        assert e["setups_exact"] == ref["setups_exact"] == 1
        assert e["class_counts"][1] + e["class_counts"][2] == 0
        assert evals[0]["setups_exact"] > e["setups_exact"]
        assert _lines_match(cands[best]["frame"].reshape(3, 3), R, 1e-5)


def test_eligibility_tolerance_keeps_side_milling_in_a_rotated_frame():
    # a wall parallel to Z' is eligible for +-Z' in the exact frame (n.a = 0);
    # after rotation n.a is a rounding residue, and only the tolerance keeps it
    V, F = synth.pocket_block(2)
    R = synth.rotation(30.0, 0.0, 20.0)
    Vr = synth.rotate(V, R)
    P, Nn, f, _ = oracle.sample_area(Vr, F, 600, seed=0)
    Rf = R.astype(np.float32).reshape(9)
    m = oracle.Mesh(Vr, F)
    with_tol, _ = m.orthogonal(P, Nn, frame=Rf)
    exact, _ = m.orthogonal(P, Nn, frame=Rf, parallel_tol=0.0)
    assert ((exact & ~with_tol) == 0).all()            # the tolerance only adds axes
    assert (with_tol != exact).sum() > 0
