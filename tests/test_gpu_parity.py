"""Parity of the CUDA library (through the C ABI) with the FP64 oracle.

Bar: bit-exact for the integer / bit / index outputs (sample points, face
ids, visibility bits outside the oracle's ambiguous rays, counts, dominant
axes, masks, classes, setup counts); accessibility fractions within 1e-4
absolute.  Run on a GB300 with ``pytest -m gpu``."""
import math

import numpy as np
import pytest

import oracle
import synth
from common import setup_outcomes, gpu_outcome, compare_bits, gpu_cast, gpu_mesh, unpack

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_05467_gb300 as rc
    rc.load()
    return rc


def _build(rc, V, F):
    Vt, Ft = gpu_mesh(V, F)
    return rc.Bvh(Vt, Ft)


def _points(V, F, n, params):
    """Sample points from the oracle's sampler (the library's own sampler is
    compared with it bit for bit in test_sampling_bit_exact), so that no
    GPU output is an input of the oracle's casts."""
    if params.sample_mode == 1:
        return oracle.sample_centroid(V, F)
    return oracle.sample_area(V, F, n, seed=params.seed)


def _sample(rc, bvh, n, params):
    P = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    N = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    f = torch.zeros(n, dtype=torch.int32, device="cuda")
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc.rc_sample_points(bvh.h, n, params, P, N, f, w)
    torch.cuda.synchronize()
    return P.cpu().numpy(), N.cpu().numpy(), f.cpu().numpy(), w.cpu().numpy()


PARTS = {
    "pocket": lambda: synth.pocket_block(3),
    "cube": lambda: synth.cube(20.0, 2),
    "icosphere": lambda: synth.icosphere(10.0, 3),
    "cavity": lambda: synth.cavity_box(subdiv=2),
    "prismatic_coarse": lambda: synth.prismatic(h=4.0),
    "impeller_coarse": lambda: synth.impeller(h=2.5),
    "multi_pocket": lambda: synth.box_with_pockets((100.0, 60.0, 40.0), (
        ("+z", (35.0, 65.0), (15.0, 45.0), 15.0), ("+x", (10.0, 50.0), (10.0, 30.0), 10.0),
        ("-y", (20.0, 40.0), (5.0, 15.0), 10.0)), subdiv=2),
}


# ---------------------------------------------------------------------------
# Section 3.1 face data and sampling: bit-exact
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["pocket", "prismatic_coarse", "impeller_coarse"])
def test_sampling_bit_exact(rc, name):
    V, F = PARTS[name]()
    bvh = _build(rc, V, F)
    for n, seed in ((1, 0), (1000, 0), (4099, 12345)):
        p = rc.rc_params_default(seed=seed)
        P, N, f, w = _sample(rc, bvh, n, p)
        oP, oN, of, ow = oracle.sample_area(V, F, n, seed=seed)
        assert np.array_equal(P.view(np.uint32), oP.view(np.uint32))
        assert np.array_equal(N.view(np.uint32), oN.view(np.uint32))
        assert np.array_equal(f, of) and np.all(w == 1.0)
    p = rc.rc_params_default(sample_mode=rc.RC_SAMPLE_FACE_CENTROID)
    P, N, f, w = _sample(rc, bvh, len(F), p)
    oP, oN, of, ow = oracle.sample_centroid(V, F)
    assert np.array_equal(P.view(np.uint32), oP.view(np.uint32))
    assert np.array_equal(N.view(np.uint32), oN.view(np.uint32))
    assert np.array_equal(w.view(np.uint64), ow.view(np.uint64))
    bvh.close()


def test_direction_table_matches_oracle(rc):
    for N in (32, 256, 1024, 2048, 65536):
        _, h32 = oracle.direction_table(N)
        assert np.array_equal(rc.rc_direction_table(N).view(np.uint32), h32.view(np.uint32))


# ---------------------------------------------------------------------------
# Section 3.1 hemispherical cast: visibility bits exact outside ambiguity
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,n,N", [
    ("pocket", 1000, 256),          # configuration-1 geometry and sizes
    ("pocket", 37, 32),
    ("pocket", 300, 150),           # the paper's 150 directions (last word padded)
    ("prismatic_coarse", 333, 150),
    ("cube", 50, 1),
    ("cavity", 100, 7),
    ("impeller_coarse", 120, 1000),
    ("cube", 200, 64),
    ("icosphere", 300, 96),
    ("cavity", 300, 64),
    ("prismatic_coarse", 777, 160),
    ("impeller_coarse", 500, 128),
    ("multi_pocket", 400, 256),
])
def test_hemisphere_parity(rc, name, n, N):
    V, F = PARTS[name]()
    bvh = _build(rc, V, F)
    p = rc.rc_params_default(n_dirs=N)
    P, Nn, f, w = _points(V, F, n, p)
    gb, gc, ctr = gpu_cast(rc, bvh.h, P, Nn, p)
    ob, oa, oc = oracle.Mesh(V, F).hemisphere(P, Nn, N)
    cmp_, amb = compare_bits(gb, gc, ob, oa, oc, N)
    assert cmp_ + amb == n * N
    assert amb <= max(1, 1e-5 * n * N) + 2
    assert ctr[0] == n * N and ctr[3] == 0
    # accessibility fractions within 1e-4
    assert abs(gc.sum() - oc.sum()) / (n * N) <= 1e-4
    bvh.close()


@pytest.mark.parametrize("mode", ["binary", "index_order", "launch_per_point"])
@pytest.mark.parametrize("name,n,N", [("pocket", 1000, 256), ("prismatic_coarse", 777, 160),
                                       ("impeller_coarse", 500, 128), ("cavity", 300, 64),
                                       ("prismatic_coarse", 333, 150), ("pocket", 90, 13)])
def test_hemisphere_parity_other_traversals(rc, name, n, N, mode):
    """The binary-tree walk, index-order points and directions, and the grid
    sized to the work give the oracle's bits too."""
    V, F = PARTS[name]()
    bvh = _build(rc, V, F)
    if mode == "binary":
        p = rc.rc_params_default(n_dirs=N, tree_width=2)
    elif mode == "index_order":
        p = rc.rc_params_default(n_dirs=N, point_order=1, tile_mode=1)
    else:
        p = rc.rc_params_default(n_dirs=N, launch_mode=1)
    P, Nn, f, w = _points(V, F, n, p)
    gb, gc, ctr = gpu_cast(rc, bvh.h, P, Nn, p)
    ob, oa, oc = oracle.Mesh(V, F).hemisphere(P, Nn, N)
    compare_bits(gb, gc, ob, oa, oc, N)
    assert ctr[0] == n * N and ctr[3] == 0
    bvh.close()


def test_hemisphere_closed_forms_on_gpu(rc):
    """Convex parts: every ray escapes; sealed cavity: every ray is blocked."""
    for V, F, expect in ((*synth.cube(20.0, 2), 1), (*synth.icosphere(10.0, 3), 1)):
        bvh = _build(rc, V, F)
        p = rc.rc_params_default(n_dirs=128)
        P, Nn, f, w = _points(V, F, 500, p)
        gb, gc, ctr = gpu_cast(rc, bvh.h, P, Nn, p)
        assert (gc == 128).all()
        bvh.close()
    V, F = synth.cavity_box(subdiv=1)
    bvh = _build(rc, V, F)
    p = rc.rc_params_default(n_dirs=64)
    P, Nn, f, w = _points(V, F, 600, p)
    inner = (P.min(1) > 5) & (P.max(1) < 35)
    gb, gc, ctr = gpu_cast(rc, bvh.h, P[inner], Nn[inner], p)
    assert (gc == 0).all()
    bvh.close()


def test_pocket_floor_centre_fraction_on_gpu(rc):
    V, F = synth.pocket_block(3)
    bvh = _build(rc, V, F)
    p = rc.rc_params_default(n_dirs=65536)
    P = np.array([[50.0, 30.0, 25.0]], np.float32)
    Nn = np.array([[0, 0, 1]], np.float32)
    gb, gc, ctr = gpu_cast(rc, bvh.h, P, Nn, p)
    assert abs(gc[0] / 65536 - 1 / 3) < 1e-3
    ob, oa, oc = oracle.Mesh(V, F).hemisphere(P, Nn, 65536)
    compare_bits(gb, gc, ob, oa, oc, 65536)
    bvh.close()


def _funnel(K, r=20.0, h=20.0):
    """Concave funnel: K side triangles from the apex (origin) to a rim of
    radius r at height h, wound so that their normals face the hollow."""
    th = 2 * np.pi * np.arange(K) / K
    V = np.concatenate([[[0.0, 0.0, 0.0]], np.stack([r * np.cos(th), r * np.sin(th), np.full(K, h)], 1)])
    F = np.array([[0, 1 + (i + 1) % K, 1 + i] for i in range(K)], np.int32)
    a, b, c = V[F[0, 0]], V[F[0, 1]], V[F[0, 2]]
    if np.cross(b - a, c - a)[2] < 0:
        F = F[:, [0, 2, 1]]
    return V.astype(np.float32), F


@pytest.mark.parametrize("K", [64, 128])
def test_points_whose_frontier_does_not_fit(rc, K):
    """Points at and near the apex of a concave funnel: more than 12 triangles have
    boxes that contain the ray origin and are not wholly below the point's
    tangent plane, so the per-point frontier (12 local triangles at most)
    does not fit and the warp walks from the root instead.  The premise is
    checked on the host; the bits must still be the oracle's."""
    V, F = _funnel(K)
    Vd = V.astype(np.float64)
    P, Nn = [], []
    for f in F:
        a, b, c = Vd[f]
        n = np.cross(b - a, c - a)
        n /= np.linalg.norm(n)
        for s in (0.0, 0.002, 0.01, 0.03):     # s = 0: the apex itself, shared by every face
            P.append(a + s * (b - a) + s * (c - a))
            Nn.append(n)
    P = np.array(P, np.float32)
    Nn = np.array(Nn, np.float32)
    lo, hi = Vd[F].min(1), Vd[F].max(1)
    for o, n in zip(P.astype(np.float64) + 1e-4 * Nn, Nn.astype(np.float64)):
        inside = ((lo <= o) & (o <= hi)).all(1)
        below = ((Vd[F] - o) @ n < 0).all(1)
        assert (inside & ~below).sum() > 12
    N = 256
    bvh = _build(rc, V, F)
    p = rc.rc_params_default(n_dirs=N)
    gb, gc, ctr = gpu_cast(rc, bvh.h, P, Nn, p)
    ob, oa, oc = oracle.Mesh(V, F).hemisphere(P, Nn, N)
    cmp_, amb = compare_bits(gb, gc, ob, oa, oc, N)
    assert cmp_ + amb == len(P) * N
    assert ctr[0] == len(P) * N and ctr[3] == 0
    assert 0 < gc.sum() < len(P) * N
    bvh.close()


@pytest.mark.parametrize("scale", [2.0, 0.5, "mixed"])
def test_normals_that_are_not_unit(rc, scale):
    """The cast takes the caller's normals as given: a normal that is not of
    unit length gives a basis whose directions can dip below the point's
    tangent plane, so the walk must not drop the triangles and boxes below
    that plane for such a point.  The bits must still be the oracle's for
    the rays as defined (offset origin and directions from the given
    normal)."""
    V, F = PARTS["pocket"]()
    p = rc.rc_params_default(n_dirs=256)
    P, Nn, f, w = _points(V, F, 400, p)
    if scale == "mixed":
        k = np.random.default_rng(3).uniform(0.3, 3.0, size=(len(Nn), 1))
        k[::3] = 1.0
        Nn = (Nn * k).astype(np.float32)
    else:
        Nn = (Nn * np.float32(scale)).astype(np.float32)
    bvh = _build(rc, V, F)
    gb, gc, ctr = gpu_cast(rc, bvh.h, P, Nn, p)
    ob, oa, oc = oracle.Mesh(V, F).hemisphere(P, Nn, 256)
    cmp_, amb = compare_bits(gb, gc, ob, oa, oc, 256)
    assert cmp_ + amb == len(P) * 256
    assert ctr[0] == len(P) * 256 and ctr[3] == 0
    bvh.close()


def test_cast_is_deterministic(rc):
    V, F = PARTS["prismatic_coarse"]()
    bvh = _build(rc, V, F)
    p = rc.rc_params_default(n_dirs=256)
    P, Nn, f, w = _points(V, F, 2000, p)
    a = gpu_cast(rc, bvh.h, P, Nn, p)
    b = gpu_cast(rc, bvh.h, P, Nn, p)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    bvh.close()


# ---------------------------------------------------------------------------
# Section 3.3 variability, classification
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N", [256, 150])
@pytest.mark.parametrize("conc_mode", [0, 1])
@pytest.mark.parametrize("mode", ["area", "centroid"])
def test_variability_parity(rc, conc_mode, mode, N):
    V, F = PARTS["multi_pocket"]()
    bvh = _build(rc, V, F)
    if mode == "area":
        p = rc.rc_params_default(n_dirs=N, conc_mode=conc_mode)
        P, Nn, f, w = _points(V, F, 3000, p)
        wt = None
    else:
        p = rc.rc_params_default(n_dirs=N, conc_mode=conc_mode, sample_mode=rc.RC_SAMPLE_FACE_CENTROID)
        P, Nn, f, w = _points(V, F, len(F), p)
        wt = torch.from_numpy(w).cuda()
    gb, gc, ctr = gpu_cast(rc, bvh.h, P, Nn, p)
    ob, oa, oc = oracle.Mesh(V, F).hemisphere(P, Nn, N)
    compare_bits(gb, gc, ob, oa, oc, N)
    n = len(P)
    # both sides reduce the oracle's bits (its ambiguous rays as it took them)
    bits = torch.from_numpy(ob.view(np.int32).copy()).cuda()
    Nt = torch.from_numpy(Nn).cuda()
    acc = torch.zeros(n, dtype=torch.float32, device="cuda")
    dom = torch.zeros(n, dtype=torch.int8, device="cuda")
    conc = torch.zeros(n, dtype=torch.float32, device="cuda")
    dira = torch.zeros(N, dtype=torch.float64, device="cuda")
    s = rc.rc_direction_variability(bits, Nt, p, weight=wt, acc=acc, dom=dom, conc=conc, dir_area=dira)
    M, ac, odom, oconc, ocnt = oracle.variability(ob, Nn, N, conc_mode=conc_mode)
    assert np.array_equal(dom.cpu().numpy(), odom)
    assert np.array_equal(conc.cpu().numpy(), oconc.astype(np.float32))
    assert np.array_equal(acc.cpu().numpy(), (ocnt / N).astype(np.float32))
    os_ = oracle.summary(ocnt, odom, oconc, N, weight=None if wt is None else w)
    if wt is None:
        assert s.overall_access == os_["overall_access"]
    else:
        # FP64 sums in another order than the oracle's: far inside the 1e-4 bar
        assert abs(s.overall_access - os_["overall_access"]) <= 1e-12
        assert abs(s.weight_sum - float(np.sum(w))) <= 1e-12 * float(np.sum(w))
    assert list(s.axis_share) == os_["axis_share"]
    assert s.mean_conc == os_["mean_conc"]
    assert s.n_counted == os_["n_counted"] and s.n_zero_visible == os_["n_zero_visible"]
    lab = rc.rc_classify(s, p)
    assert lab == oracle.classify(os_)
    # per-direction visible weight
    wv = np.ones(n) if wt is None else w
    expect = (unpack(ob, N) * wv[:, None]).sum(0).astype(np.float64)
    if wt is None:
        assert np.array_equal(dira.cpu().numpy(), expect)
    else:
        assert np.allclose(dira.cpu().numpy(), expect, rtol=1e-12, atol=0)
    bvh.close()


# ---------------------------------------------------------------------------
# Sections 3.2 / 3.3: orthogonal cast, classes, setups
# ---------------------------------------------------------------------------

FRAMES = {
    "identity": None,
    "quarter_z": [0, -1, 0, 1, 0, 0, 0, 0, 1],
    "tilted": [0.8, -0.6, 0, 0.6, 0.8, 0, 0, 0, 1],
    # neither orthogonal nor unit columns: G = F^T F has off-diagonal terms
    # of 0.1-0.6, which the frame-space box test must widen its band by
    "sheared": [1.0, 0.3, 0.0, 0.0, 2.0, 0.25, 0.1, 0.0, 0.5],
}


@pytest.mark.parametrize("frame", list(FRAMES))
@pytest.mark.parametrize("name", ["pocket", "multi_pocket", "prismatic_coarse"])
def test_orthogonal_and_setups_parity(rc, name, frame):
    V, F = PARTS[name]()
    bvh = _build(rc, V, F)
    fr = FRAMES[frame]
    kw = {} if fr is None else {"frame": fr}
    for mode in (rc.RC_SAMPLE_FACE_CENTROID, rc.RC_SAMPLE_AREA_RANDOM):
        p = rc.rc_params_default(sample_mode=mode, tool_length=30.0, **kw)
        n = len(F) if mode == rc.RC_SAMPLE_FACE_CENTROID else 2500
        P, Nn, f, w = _points(V, F, n, p)
        Pt, Nt = torch.from_numpy(P).cuda(), torch.from_numpy(Nn).cuda()
        mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
        trav = torch.zeros((n, 6), dtype=torch.float32, device="cuda")
        ctr = torch.zeros(4, dtype=torch.int64, device="cuda")
        rc.rc_orthogonal_cast(bvh.h, Pt, Nt, p, mask, trav, ctr)
        ft = torch.from_numpy(f).cuda()
        cls = torch.zeros(n, dtype=torch.uint8, device="cuda")
        su = rc.rc_min_setups(bvh.h, mask, trav, ft, p, cls)
        gm = mask.cpu().numpy()
        gt = trav.cpu().numpy()
        om, oam = oracle.Mesh(V, F).orthogonal(P, Nn, frame=fr)
        ot = oracle.travel(V, P, frame=fr)
        assert np.array_equal(gt.view(np.uint32), ot.view(np.uint32))
        clean = oam == 0
        assert np.array_equal(gm[clean], om[clean])
        if mode == rc.RC_SAMPLE_AREA_RANDOM:
            # centroid rays on these dyadic meshes meet other faces' edges
            # exactly by construction, so only random points get the budget
            assert (~clean).sum() <= max(2, 1e-5 * 6 * n)
        fx = oracle.fixture_faces(V, F, frame=fr)
        # classes and covers from the oracle's own masks; its ambiguous axis
        # rays are taken either way
        outs, ocls_clean, oclean = setup_outcomes(om, oam, ot, f, fx, 30.0)
        assert np.array_equal(cls.cpu().numpy()[oclean], ocls_clean)
        if outs is not None:
            assert gpu_outcome(su) in outs
        else:
            # centroid rays on dyadic meshes: too many ambiguous rays to
            # enumerate; the covers are compared when the GPU took every
            # ambiguous ray as the oracle's FP64 rule did
            if np.array_equal(gm, om):
                ocls, oreach = oracle.face_classes(om, ot, f, fx, 30.0)
                viable = oreach[ocls == 0]
                assert (su.setups_exact, su.chosen_exact) == oracle.setups_exact(viable)
                assert su.setups_greedy == oracle.setups_greedy(viable)[0]
        assert ctr.cpu().numpy()[3] == 0
    bvh.close()


@pytest.mark.parametrize("point_order", [0, 1])
def test_orthogonal_small_counts(rc, point_order):
    # work items are (axis, 32 points): counts below, at and just past a
    # multiple of 32, in Morton and in index order
    V, F = PARTS["multi_pocket"]()
    bvh = _build(rc, V, F)
    p = rc.rc_params_default(tool_length=30.0, point_order=point_order)
    Pall, Nall, _, _ = _points(V, F, 97, p)
    om_all, oam_all = oracle.Mesh(V, F).orthogonal(Pall, Nall)
    ot_all = oracle.travel(V, Pall)
    for n in (1, 31, 32, 33, 97):
        Pt, Nt = torch.from_numpy(Pall[:n].copy()).cuda(), torch.from_numpy(Nall[:n].copy()).cuda()
        mask = torch.full((n,), 0xFF, dtype=torch.uint8, device="cuda")
        trav = torch.zeros((n, 6), dtype=torch.float32, device="cuda")
        ctr = torch.zeros(4, dtype=torch.int64, device="cuda")
        rc.rc_orthogonal_cast(bvh.h, Pt, Nt, p, mask, trav, ctr)
        clean = oam_all[:n] == 0
        assert np.array_equal(mask.cpu().numpy()[clean], om_all[:n][clean])
        assert np.array_equal(trav.cpu().numpy().view(np.uint32), ot_all[:n].view(np.uint32))
        c = ctr.cpu().numpy()
        assert c[3] == 0 and 0 < c[0] <= 6 * n
    bvh.close()


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def test_edge_cases(rc):
    # single triangle and tiny parts (single-leaf root)
    for T in (1, 2, 4, 5):
        V, F = synth.cube(10.0, 0)
        F = F[:T]
        bvh = _build(rc, V, F)
        p = rc.rc_params_default(n_dirs=64)
        P, Nn, f, w = _points(V, F, 50, p)
        gb, gc, ctr = gpu_cast(rc, bvh.h, P, Nn, p)
        ob, oa, oc = oracle.Mesh(V, F).hemisphere(P, Nn, 64)
        compare_bits(gb, gc, ob, oa, oc, 64)
        bvh.close()
    V, F = synth.pocket_block(1)
    bvh = _build(rc, V, F)
    p = rc.rc_params_default(n_dirs=64)
    # n == 0 is a no-op
    e = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    rc.rc_hemisphere_cast(bvh.h, e, e, p, torch.zeros((0, 2), dtype=torch.int32, device="cuda"),
                          torch.zeros(0, dtype=torch.int32, device="cuda"))
    # bad n_dirs
    for bad_n in (0, -3, 65537):
        with pytest.raises(rc.RcError) as ei:
            rc.rc_hemisphere_cast(bvh.h, e, e, rc.rc_params_default(n_dirs=bad_n), e, e)
        assert ei.value.status == 1
    bvh.close()
    # invalid meshes are rejected
    Vt, Ft = gpu_mesh(V, F)
    bad = Ft.clone()
    bad[3, 1] = len(V)
    with pytest.raises(rc.RcError):
        rc.rc_build_bvh(Vt, bad)
    Vn = Vt.clone()
    Vn[5, 2] = float("nan")
    with pytest.raises(rc.RcError):
        rc.rc_build_bvh(Vn, Ft)
    # zero-area part cannot be sampled
    Vz = torch.zeros((3, 3), dtype=torch.float32, device="cuda")
    Fz = torch.tensor([[0, 1, 2]], dtype=torch.int32, device="cuda")
    h = rc.rc_build_bvh(Vz, Fz)
    with pytest.raises(rc.RcError) as ei:
        P = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
        rc.rc_sample_points(h, 4, rc.rc_params_default(), P, P.clone(), torch.zeros(4, dtype=torch.int32, device="cuda"))
    assert ei.value.status == 5
    rc.rc_destroy_bvh(h)


def test_refit_matches_rebuild(rc):
    V0, F = synth.perturbed_part(2, 0.0)
    V1, F1 = synth.perturbed_part(2, 3.5)
    assert np.array_equal(F, F1)
    Vt0, Ft = gpu_mesh(V0, F)
    Vt1, _ = gpu_mesh(V1, F)
    a = rc.Bvh(Vt0, Ft)
    rc.rc_refit_bvh(a.h, Vt1)
    b = rc.Bvh(Vt1, Ft)
    p = rc.rc_params_default(n_dirs=128)
    P, Nn, f, w = _sample(rc, b, 800, p)
    ra = gpu_cast(rc, a.h, P, Nn, p)
    rb = gpu_cast(rc, b.h, P, Nn, p)
    assert np.array_equal(ra[0], rb[0])
    Pa, Na, fa, wa = _sample(rc, a, 800, p)
    assert np.array_equal(Pa, P) and np.array_equal(fa, f)
    a.close()
    b.close()


# ---------------------------------------------------------------------------
# full-size workloads, sampled outputs (the benchmark's launch configuration)
# ---------------------------------------------------------------------------

def _popcount_rows(bits):
    """Unobstructed count of every row of a uint32 [n, W] bit array (in
    chunks, so a 1M x 2,048 array never becomes 2e9 booleans)."""
    out = np.zeros(len(bits), np.int64)
    for a in range(0, len(bits), 65536):
        blk = np.ascontiguousarray(bits[a:a + 65536], np.uint32).view(np.uint8)
        out[a:a + 65536] = np.unpackbits(blk, axis=1).sum(1)
    return out


def test_full_size_prismatic(rc):
    """Prismatic part: ~200k triangles, 100k points x 1,024 directions, in
    the benchmark's launch configuration; every one of the 1.02e8 rays is
    compared with the oracle (bit for bit outside its ambiguous rays)."""
    V, F = synth.prismatic()
    assert 150_000 < len(F) < 260_000
    n, N = 100_000, 1024
    bvh = _build(rc, V, F)
    p = rc.rc_params_default(n_dirs=N)
    P, Nn, f, w = _points(V, F, n, p)
    gb, gc, ctr = gpu_cast(rc, bvh.h, P, Nn, p)
    assert ctr[0] == n * N and ctr[3] == 0
    ob, oa, oc = oracle.Mesh(V, F).hemisphere(P, Nn, N)
    cmp_, amb = compare_bits(gb, gc, ob, oa, oc, N)
    assert cmp_ + amb == n * N and amb <= 1e-5 * n * N
    bvh.close()


@pytest.mark.slow
def test_full_size_impeller(rc):
    """Freeform impeller: ~2M triangles, 1M points x 2,048 directions (2.05e9
    rays) in the benchmark's launch configuration.  Compared with the
    oracle: every ray of 5,000 random points (1.02e7 rays), and every ray
    whose walk re-tested a pair in FP64 (listed by the instrumented copy of
    the traversal, whose bits must equal the plain cast's); counts equal
    the rows' popcounts everywhere."""
    V, F = synth.impeller()
    n, N = 1_000_000, 2048
    bvh = _build(rc, V, F)
    p = rc.rc_params_default(n_dirs=N)
    P, Nn, f, w = _points(V, F, n, p)
    gb, gc, ctr = gpu_cast(rc, bvh.h, P, Nn, p)
    assert ctr[0] == n * N and ctr[3] == 0
    assert np.array_equal(_popcount_rows(gb), gc)
    m = oracle.Mesh(V, F)
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(n, size=5000, replace=False))
    ob, oa, oc = m.hemisphere(P[idx], Nn[idx], N)
    cmp_, amb = compare_bits(gb[idx], gc[idx], ob, oa, oc, N)
    assert cmp_ + amb == 5000 * N and amb <= max(2, 1e-5 * 5000 * N)
    # the rays an FP64 re-test took part in
    cap = 1 << 22
    Pt, Nt = torch.from_numpy(P).cuda(), torch.from_numpy(Nn).cuda()
    b2 = torch.zeros((n, N // 32), dtype=torch.int32, device="cuda")
    c2 = torch.zeros(n, dtype=torch.int32, device="cuda")
    ctr8 = torch.zeros(8, dtype=torch.int64, device="cuda")
    lst = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    rc.rc_hemisphere_cast_retests(bvh.h, Pt, Nt, p, b2, c2, ctr8, lst)
    torch.cuda.synchronize()
    c8 = ctr8.cpu().numpy()
    total = int(c8[6])
    assert 0 < total <= cap and c8[0] == n * N and c8[3] == 0
    assert np.array_equal(b2.cpu().numpy().view(np.uint32), gb) and np.array_equal(c2.cpu().numpy(), gc)
    codes = lst[:total].cpu().numpy()
    i, j = codes >> 16, codes & 0xFFFF
    assert (i < n).all() and (j < N).all() and len(np.unique(codes)) == total
    O, D = oracle.rays_at(P, Nn, N, i, j)
    st = m.cast_rays(O, D)
    gbit = (gb[i, j >> 5] >> (j & 31).astype(np.uint32)) & 1
    ok = st != oracle.AMB
    bad = ok & (gbit != (st == oracle.MISS))
    assert not bad.any(), "%d re-tested rays differ from the oracle" % int(bad.sum())
    assert int((~ok).sum()) <= max(2, 1e-5 * n * N)
    bvh.close()


# ---------------------------------------------------------------------------
# the PLOC binary tree (rc_build_bvh_ex): same results as the Karras tree
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,n,N", [("pocket", 500, 256), ("prismatic_coarse", 600, 150),
                                       ("impeller_coarse", 300, 128), ("cavity", 200, 64), ("cube", 3, 32)])
def test_ploc_tree_parity(rc, name, n, N):
    V, F = PARTS[name]()
    Vt, Ft = gpu_mesh(V, F)
    bvh = rc.Bvh(Vt, Ft, builder=rc.RC_BUILDER_PLOC)
    info = rc.rc_bvh_get_info(bvh.h)
    assert info.n_tris == len(F)
    for width in (4, 2):
        p = rc.rc_params_default(n_dirs=N, tree_width=width)
        P, Nn, f, w = _points(V, F, n, p)
        gb, gc, ctr = gpu_cast(rc, bvh.h, P, Nn, p)
        ob, oa, oc = oracle.Mesh(V, F).hemisphere(P, Nn, N)
        compare_bits(gb, gc, ob, oa, oc, N)
        assert ctr[0] == n * N and ctr[3] == 0
    bvh.close()


def test_ploc_tree_refit_and_tiny_parts(rc):
    V0, F = synth.perturbed_part(2, 0.0)
    V1, _ = synth.perturbed_part(2, 3.5)
    Vt0, Ft = gpu_mesh(V0, F)
    Vt1, _ = gpu_mesh(V1, F)
    a = rc.Bvh(Vt0, Ft, builder=rc.RC_BUILDER_PLOC)
    rc.rc_refit_bvh(a.h, Vt1)
    b = rc.Bvh(Vt1, Ft, builder=rc.RC_BUILDER_PLOC)
    p = rc.rc_params_default(n_dirs=128)
    P, Nn, f, w = _points(V1, F, 700, p)
    assert np.array_equal(gpu_cast(rc, a.h, P, Nn, p)[0], gpu_cast(rc, b.h, P, Nn, p)[0])
    a.close()
    b.close()
    for T in (1, 2, 3, 5):
        V, F = synth.cube(10.0, 0)
        bvh = rc.Bvh(*gpu_mesh(V, F[:T]), builder=rc.RC_BUILDER_PLOC)
        p = rc.rc_params_default(n_dirs=64)
        P, Nn, f, w = _points(V, F[:T], 40, p)
        gb, gc, ctr = gpu_cast(rc, bvh.h, P, Nn, p)
        ob, oa, oc = oracle.Mesh(V, F[:T]).hemisphere(P, Nn, 64)
        compare_bits(gb, gc, ob, oa, oc, 64)
        bvh.close()
    with pytest.raises(rc.RcError):
        rc.rc_build_bvh_ex(*gpu_mesh(V, F), 7)


# ---------------------------------------------------------------------------
# device-side index checks of the built trees (in place of a memory checker)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["pocket", "cube", "prismatic_coarse", "impeller_coarse", "multi_pocket"])
def test_built_trees_pass_the_index_checks(rc, name):
    V, F = PARTS[name]()
    for builder in (0, 1):
        Vt, Ft = gpu_mesh(V, F)
        h = rc.rc_build_bvh_ex(Vt, Ft, builder)
        c = rc.rc_bvh_validate(h)
        assert c["nodes_seen"] >= 1
        assert {k: v for k, v in c.items() if k != "nodes_seen"} == dict.fromkeys(
            ("wide_child", "wide_leaf", "wide_box", "binary_child", "tri_face"), 0), c
        rc.rc_destroy_bvh(h)


def test_tiny_and_refitted_trees_pass_the_index_checks(rc):
    V, F = synth.cube(10.0, 0)
    for T in (1, 2, 3, 5):
        Vt, Ft = gpu_mesh(V, F[:T])
        h = rc.rc_build_bvh(Vt, Ft)
        c = rc.rc_bvh_validate(h)
        assert c["nodes_seen"] >= 1 and sum(v for k, v in c.items() if k != "nodes_seen") == 0, (T, c)
        rc.rc_destroy_bvh(h)
    V0, F0 = synth.perturbed_part(2, 0.0)
    V1, _ = synth.perturbed_part(2, 3.5)
    bvh = _build(rc, V0, F0)
    rc.rc_refit_bvh(bvh.h, torch.from_numpy(V1).cuda())
    c = rc.rc_bvh_validate(bvh.h)
    assert sum(v for k, v in c.items() if k != "nodes_seen") == 0, c
    bvh.close()


def test_translation_by_an_exact_offset(rc):
    # the pocket block's vertices lie on a dyadic grid, so adding (64, -32, 128)
    # is exact; the cast of the translated part from the translated centroids
    # must agree with the original: only the origin offset is rounded at a
    # different magnitude, which may move a grazing ray across an edge
    V, F = synth.pocket_block(3)
    off = np.array([64.0, -32.0, 128.0], np.float32)
    Vt = (V + off).astype(np.float32)
    assert np.array_equal((Vt - off).astype(np.float32), V)
    p = rc.rc_params_default(n_dirs=256)
    P, Nn, _, _ = oracle.sample_centroid(V, F)
    Pt, Nt, _, _ = oracle.sample_centroid(Vt, F)
    assert np.array_equal(Nt, Nn)
    b0 = _build(rc, V, F)
    b1 = _build(rc, Vt, F)
    g0, c0, _ = gpu_cast(rc, b0.h, P, Nn, p)
    g1, c1, _ = gpu_cast(rc, b1.h, Pt, Nt, p)
    same = np.unpackbits(g0.view(np.uint8)) == np.unpackbits(g1.view(np.uint8))
    assert same.mean() > 0.999
    assert abs(c0.sum() - c1.sum()) <= 1e-3 * c0.sum()
    b0.close()
    b1.close()


def test_turned_frame_after_a_refit_that_grows_the_part(rc):
    """A refit to vertices far outside the old bounding box, then the
    orthogonal cast in a turned frame (frame-space boxes, whose band
    tolerance scales with the part's reach): masks equal the oracle's on
    the refitted geometry outside its ambiguous axes."""
    V0, F = PARTS["multi_pocket"]()
    Vt0, Ft = gpu_mesh(V0, F)
    bvh = rc.Bvh(Vt0, Ft)
    V1 = (V0.astype(np.float64) * 2.5 + np.array([300.0, -120.0, 75.0])).astype(np.float32)
    rc.rc_refit_bvh(bvh.h, torch.from_numpy(V1).cuda())
    info = rc.rc_bvh_get_info(bvh.h)
    assert np.allclose(info.scene_lo, V1.min(0)) and np.allclose(info.scene_hi, V1.max(0))
    frame = [0.8, -0.6, 0, 0.6, 0.8, 0, 0, 0, 1]
    p = rc.rc_params_default(frame=frame)
    P, Nn, f, w = _points(V1, F, 3000, p)
    Pt, Nt = torch.from_numpy(P).cuda(), torch.from_numpy(Nn).cuda()
    mask = torch.zeros(len(P), dtype=torch.uint8, device="cuda")
    trav = torch.zeros((len(P), 6), dtype=torch.float32, device="cuda")
    rc.rc_orthogonal_cast(bvh.h, Pt, Nt, p, mask, trav)
    om, oam = oracle.Mesh(V1, F).orthogonal(P, Nn, frame=frame)
    gm = mask.cpu().numpy()
    assert np.array_equal(gm & ~oam, om & ~oam)
    bvh.close()
