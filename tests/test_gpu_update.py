"""Re-analysis after an edit that keeps the triangle list: points kept on
their faces (bit for bit the oracle's), changed faces and their box, and the
updated visibility equal to a full re-cast of the edited part and to the
oracle's cast at the same points."""
import numpy as np
import pytest

import oracle
import synth

from common import compare_bits, gpu_mesh

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_05467_gb300 as rc
    rc.load()
    return rc


def _cast(rc, h, P, Nn, p):
    n = P.shape[0]
    W = (p.n_dirs + 31) // 32
    bits = torch.zeros((n, W), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    ctr = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc.rc_hemisphere_cast(h, P, Nn, p, bits, cnt, ctr)
    return bits, cnt, ctr


def _edit(rc, V0, V1, F, n, p, centroid):
    Vt0, Ft = gpu_mesh(V0, F)
    Vt1, _ = gpu_mesh(V1, F)
    b0, b1 = rc.Bvh(Vt0, Ft), rc.Bvh(Vt1, Ft)
    if centroid:
        n = len(F)
    P0 = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    N0 = torch.zeros_like(P0)
    f = torch.zeros(n, dtype=torch.int32, device="cuda")
    rc.rc_sample_points(b0.h, n, p, P0, N0, f)
    bits, cnt, _ = _cast(rc, b0.h, P0, N0, p)
    changed = torch.zeros(len(F), dtype=torch.uint8, device="cuda")
    nc, box = rc.rc_changed_faces(Vt0, Vt1, Ft, changed)
    P1 = torch.zeros_like(P0)
    N1 = torch.zeros_like(P0)
    rc.rc_sample_points_on_faces(b1.h, p, f, P1, N1)
    ctr = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc.rc_hemisphere_update(b1.h, P1, N1, f, changed, box, p, bits, cnt, ctr)
    full_bits, full_cnt, full_ctr = _cast(rc, b1.h, P1, N1, p)
    torch.cuda.synchronize()
    out = dict(nc=nc, box=box, changed=changed.cpu().numpy(), f=f.cpu().numpy(), P1=P1.cpu().numpy(),
               N1=N1.cpu().numpy(), bits=bits.cpu().numpy().view(np.uint32), cnt=cnt.cpu().numpy(),
               ctr=ctr.cpu().numpy(), full_bits=full_bits.cpu().numpy().view(np.uint32),
               full_cnt=full_cnt.cpu().numpy(), full_ctr=full_ctr.cpu().numpy())
    b0.close()
    b1.close()
    return out


@pytest.mark.parametrize("centroid", [False, True])
@pytest.mark.parametrize("shift,deepen,N", [(2.5, 0.0, 256), (0.75, 0.0, 150), (4.0, 0.0, 64), (0.0, 2.0, 256),
                                            (1.5, 3.0, 96)])
def test_update_equals_full_recast_and_oracle(rc, shift, deepen, N, centroid):
    V0, F = synth.perturbed_part(3, 0.0)
    V1, F1 = synth.perturbed_part(3, shift, deepen_mm=deepen)
    assert np.array_equal(F, F1)
    seed = 5
    p = rc.rc_params_default(n_dirs=N, seed=seed,
                             sample_mode=rc.RC_SAMPLE_FACE_CENTROID if centroid else rc.RC_SAMPLE_AREA_RANDOM)
    n = 2000
    r = _edit(rc, V0, V1, F, n, p, centroid)
    # changed faces and their box, by brute force
    moved = (V0[F] != V1[F]).any(axis=(1, 2))
    assert np.array_equal(r["changed"].astype(bool), moved) and r["nc"] == int(moved.sum())
    both = np.concatenate([V0[F[moved]].reshape(-1, 3), V1[F[moved]].reshape(-1, 3)])
    assert np.array_equal(np.array(r["box"], np.float32), np.concatenate([both.min(0), both.max(0)]))
    # points kept on their faces: the oracle's own chain gives the same bits
    if centroid:
        oP1, oN1 = oracle.sample_on_faces(V1, F, np.arange(len(F), dtype=np.int32), centroid=True)
    else:
        _, _, of, _ = oracle.sample_area(V0, F, n, seed=seed)
        oP1, oN1 = oracle.sample_on_faces(V1, F, of, seed=seed)
    assert np.array_equal(r["P1"].view(np.uint32), oP1.view(np.uint32))
    assert np.array_equal(r["N1"].view(np.uint32), oN1.view(np.uint32))
    # the update equals the full re-cast (up to rays decided by ambiguous pairs)
    diff = int(np.unpackbits((r["bits"] ^ r["full_bits"]).view(np.uint8)).sum())
    assert diff <= int(r["ctr"][1] + r["full_ctr"][1])
    if diff == 0:
        assert np.array_equal(r["cnt"], r["full_cnt"])
    assert r["ctr"][3] == 0 and 0 < r["ctr"][0] < len(r["P1"]) * N
    # and the oracle's cast at the same points
    ob, oa, oc = oracle.Mesh(V1, F).hemisphere(oP1, oN1, N)
    compare_bits(r["bits"], r["cnt"], ob, oa, oc, N)


def test_update_with_normals_that_are_not_unit(rc):
    """A caller's normals of other than unit length: the update must not skip
    a point because the changed box lies behind its tangent plane (its
    directions can dip below that plane), and its bits must equal the full
    re-cast with the same normals and the oracle's cast."""
    V0, F = synth.perturbed_part(3, 0.0)
    V1, _ = synth.perturbed_part(3, 2.5)
    p = rc.rc_params_default(n_dirs=128, seed=2)
    n = 1500
    Vt0, Ft = gpu_mesh(V0, F)
    Vt1, _ = gpu_mesh(V1, F)
    b0, b1 = rc.Bvh(Vt0, Ft), rc.Bvh(Vt1, Ft)
    P0 = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    N0 = torch.zeros_like(P0)
    f = torch.zeros(n, dtype=torch.int32, device="cuda")
    rc.rc_sample_points(b0.h, n, p, P0, N0, f)
    k = torch.from_numpy(np.random.default_rng(9).uniform(0.4, 2.5, size=(n, 1)).astype(np.float32)).cuda()
    bits, cnt, _ = _cast(rc, b0.h, P0, N0 * k, p)
    changed = torch.zeros(len(F), dtype=torch.uint8, device="cuda")
    nc, box = rc.rc_changed_faces(Vt0, Vt1, Ft, changed)
    P1 = torch.zeros_like(P0)
    N1 = torch.zeros_like(P0)
    rc.rc_sample_points_on_faces(b1.h, p, f, P1, N1)
    N1k = N1 * k
    ctr = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc.rc_hemisphere_update(b1.h, P1, N1k, f, changed, box, p, bits, cnt, ctr)
    full_bits, full_cnt, full_ctr = _cast(rc, b1.h, P1, N1k, p)
    torch.cuda.synchronize()
    gb = bits.cpu().numpy().view(np.uint32)
    diff = int(np.unpackbits((gb ^ full_bits.cpu().numpy().view(np.uint32)).view(np.uint8)).sum())
    assert diff <= int(ctr[1].item() + full_ctr[1].item())
    hP1, hN1k = P1.cpu().numpy(), N1k.cpu().numpy()
    ob, oa, oc = oracle.Mesh(V1, F).hemisphere(hP1, hN1k, 128)
    compare_bits(gb, cnt.cpu().numpy(), ob, oa, oc, 128)
    b0.close()
    b1.close()


def test_update_without_and_with_everything_changed(rc):
    V0, F = synth.perturbed_part(2, 0.0)
    p = rc.rc_params_default(n_dirs=128, seed=1)
    r = _edit(rc, V0, V0.copy(), F, 700, p, False)
    assert r["nc"] == 0 and r["box"][0] > r["box"][3] and r["ctr"][0] == 0
    assert np.array_equal(r["bits"], r["full_bits"]) and np.array_equal(r["cnt"], r["full_cnt"])
    Vs = V0 + np.float32(1.0)                      # every face moves
    r = _edit(rc, V0, Vs, F, 700, p, False)
    assert r["nc"] == len(F) and r["ctr"][0] == 700 * 128
    assert np.array_equal(r["bits"], r["full_bits"])


def test_update_argument_errors(rc):
    V0, F = synth.perturbed_part(1, 0.0)
    Vt, Ft = gpu_mesh(V0, F)
    b = rc.Bvh(Vt, Ft)
    p = rc.rc_params_default(n_dirs=64)
    f = torch.tensor([0, len(F)], dtype=torch.int32, device="cuda")
    P = torch.zeros((2, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(rc.RcError) as ei:
        rc.rc_sample_points_on_faces(b.h, p, f, P, P.clone())
    assert ei.value.status == 1 and "outside" in str(ei.value)
    bad = Ft.clone()
    bad[2, 0] = len(V0) + 3
    with pytest.raises(rc.RcError):
        rc.rc_changed_faces(Vt, Vt, bad, torch.zeros(len(F), dtype=torch.uint8, device="cuda"))
    with pytest.raises(rc.RcError):
        rc.rc_hemisphere_update(b.h, P, P, f, torch.zeros(len(F), dtype=torch.uint8, device="cuda"),
                                [0, 0, 0, float("inf"), 1, 1], p, torch.zeros((2, 2), dtype=torch.int32, device="cuda"),
                                torch.zeros(2, dtype=torch.int32, device="cuda"))
    b.close()


def test_update_after_a_local_bump_on_a_blade(rc):
    V0, F = synth.impeller(h=2.5)
    r = np.hypot(V0[:, 0], V0[:, 1])
    c = V0[np.argmin(np.abs(r - 55.0) + np.abs(V0[:, 2] - 25.0))].astype(np.float64)
    V1 = synth.bump(V0, c, 6.0, 0.5, direction=(-c[1], c[0], 0.0))
    p = rc.rc_params_default(n_dirs=256, seed=2)
    n = 3000
    res = _edit(rc, V0, V1, F, n, p, False)
    assert 0 < res["nc"] < len(F) // 20
    _, _, of, _ = oracle.sample_area(V0, F, n, seed=2)
    oP1, oN1 = oracle.sample_on_faces(V1, F, of, seed=2)
    assert np.array_equal(res["P1"].view(np.uint32), oP1.view(np.uint32))
    assert np.array_equal(res["bits"], res["full_bits"]) and np.array_equal(res["cnt"], res["full_cnt"])
    assert res["ctr"][0] < 0.2 * n * 256                  # a local edit: few rays cast again
    ob, oa, oc = oracle.Mesh(V1, F).hemisphere(oP1, oN1, 256)
    compare_bits(res["bits"], res["cnt"], ob, oa, oc, 256)
