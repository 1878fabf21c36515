"""Automatic machining frame on the GPU against the oracle (oracle/frames.py):
candidate frames bit for bit, per-frame setups and the choice exactly (the
oracle's ambiguous axis rays enumerated either way)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import frames as ofr

from common import gpu_mesh, gpu_outcome, setup_outcomes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_05467_gb300 as rc
    rc.load()
    return rc


def _pocket_rot(ang):
    V, F = synth.pocket_block(2)
    return synth.rotate(V, synth.rotation(*ang)), F


PARTS = {
    "pocket_30_0_20": lambda: _pocket_rot((30.0, 0.0, 20.0)),
    "pocket_10_45_0": lambda: _pocket_rot((10.0, 45.0, 0.0)),
    "pocket_0_0_33": lambda: _pocket_rot((0.0, 0.0, 33.0)),
    "pocket_axis_aligned": lambda: synth.pocket_block(2),
    "box_rot": lambda: (synth.rotate(synth.box_with_pockets((100.0, 60.0, 40.0), pockets=(), subdiv=1)[0],
                                     synth.rotation(-15.0, 35.0, 10.0)),
                        synth.box_with_pockets((100.0, 60.0, 40.0), pockets=(), subdiv=1)[1]),
    "cube": lambda: synth.cube(20.0, 1),
    "prismatic_rot": lambda: (synth.rotate(synth.prismatic(h=5.0)[0], synth.rotation(12.0, -7.0, 25.0)),
                              synth.prismatic(h=5.0)[1]),
    "impeller_coarse": lambda: synth.impeller(h=3.0),
}


def _frames_from_oracle(rc, cands):
    fr = rc.Frames()
    fr.k = len(cands)
    fr.best = -1
    for c, cand in enumerate(cands):
        for i in range(9):
            fr.frame[c][i] = float(cand["frame"][i])
    return fr


def _check_candidates(rc, V, F, fr, cands):
    assert fr.k == len(cands) and fr.best == -1
    for c, cand in enumerate(cands):
        assert fr.source[c] == cand["source"]
        assert (fr.box_axis[c], fr.box_step[c]) == (cand["box_axis"], cand["box_step"])
        assert np.array_equal(fr.frame_array(c).view(np.uint32), cand["frame"].view(np.uint32)), c
        assert fr.volume[c] == cand["volume"]
    w, _ = ofr.principal_axes(V, F)
    assert np.allclose(list(fr.principal), w, rtol=1e-9, atol=1e-9 * abs(w[0]))


@pytest.mark.parametrize("name", list(PARTS))
def test_frame_candidates_match_oracle(rc, name):
    V, F = PARTS[name]()
    Vt, Ft = gpu_mesh(V, F)
    bvh = rc.Bvh(Vt, Ft)
    fr = rc.rc_frame_candidates(bvh.h, rc.rc_params_default())
    _check_candidates(rc, V, F, fr, ofr.frame_candidates(V, F))
    bvh.close()


def _select_and_compare(rc, V, F, bvh, P, Nn, f, cands, p):
    fr = _frames_from_oracle(rc, cands)
    ctr = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc.rc_frame_select(bvh.h, torch.from_numpy(P).cuda(), torch.from_numpy(Nn).cuda(), torch.from_numpy(f).cuda(),
                       p, fr, ctr)
    mesh = oracle.Mesh(V, F)
    allowed = []
    for c, cand in enumerate(cands):
        ev = ofr.evaluate_frame(mesh, V, F, P, Nn, f, cand["frame"], p.tool_length)
        fx = oracle.fixture_faces(V, F, frame=cand["frame"])
        outs, _, _ = setup_outcomes(ev["mask"], ev["amb"], ev["travel"], f, fx, p.tool_length)
        assert outs is not None, "too many ambiguous axis rays to enumerate"
        assert gpu_outcome(fr.setups[c]) in outs, c
        allowed.append(outs)
        assert fr.volume[c] == cand["volume"]
    # the choice: the oracle's rule applied to the GPU's (validated) outcomes
    keys = [(fr.setups[c].setups_exact, fr.setups[c].class_counts[1] + fr.setups[c].class_counts[2],
             fr.volume[c], c) for c in range(fr.k)]
    assert fr.best == min(keys)[3]
    # and, when no ambiguous ray is involved, the oracle's own choice
    if all(len(o) == 1 for o in allowed):
        evals = [ofr.evaluate_frame(mesh, V, F, P, Nn, f, c["frame"], p.tool_length) for c in cands]
        assert fr.best == ofr.select_frame(cands, evals)
    c = ctr.cpu().numpy()
    assert c[3] == 0 and c[1] <= max(2, 1e-5 * c[0])
    return fr


@pytest.mark.parametrize("name", ["pocket_30_0_20", "pocket_10_45_0", "pocket_0_0_33", "prismatic_rot",
                                  "impeller_coarse"])
def test_frame_select_matches_oracle(rc, name):
    V, F = PARTS[name]()
    Vt, Ft = gpu_mesh(V, F)
    bvh = rc.Bvh(Vt, Ft)
    p = rc.rc_params_default(tool_length=60.0)
    P, Nn, f, _ = oracle.sample_area(V, F, 1500, seed=3)
    cands = ofr.frame_candidates(V, F)
    _select_and_compare(rc, V, F, bvh, P, Nn, f, cands, p)
    bvh.close()


def test_auto_frame_end_to_end_undoes_a_rotation(rc):
    V0, F = synth.pocket_block(2)
    Vr, _ = _pocket_rot((30.0, 0.0, 20.0))
    Vt, Ft = gpu_mesh(Vr, F)
    bvh = rc.Bvh(Vt, Ft)
    p = rc.rc_params_default()
    n = 800
    P = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    Nn = torch.zeros_like(P)
    f = torch.zeros(n, dtype=torch.int32, device="cuda")
    rc.rc_sample_points(bvh.h, n, p, P, Nn, f)
    fr = rc.rc_frame_candidates(bvh.h, p)
    rc.rc_frame_select(bvh.h, P, Nn, f, p, fr)
    cands, evals, best = ofr.auto_frame(Vr, F, *oracle.sample_area(Vr, F, n, seed=0)[:3], p.tool_length)
    assert fr.best == best
    su = fr.setups[fr.best]
    assert su.setups_exact == evals[best]["setups_exact"] == 1
    assert list(su.class_counts) == evals[best]["class_counts"]
    # the unrotated block in the identity frame
    ref = ofr.evaluate_frame(oracle.Mesh(V0, F), V0, F, *oracle.sample_area(V0, F, n, seed=0)[:3], None,
                             p.tool_length)
    assert su.setups_exact == ref["setups_exact"] and list(su.class_counts)[1:3] == ref["class_counts"][1:3]
    # the chosen frame works through the ordinary entry points too
    q = rc.rc_params_default(frame=list(fr.frame[fr.best]))
    mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
    trav = torch.zeros((n, 6), dtype=torch.float32, device="cuda")
    rc.rc_orthogonal_cast(bvh.h, P, Nn, q, mask, trav)
    s2 = rc.rc_min_setups(bvh.h, mask, trav, f, q)
    assert (s2.setups_exact, list(s2.class_counts)) == (su.setups_exact, list(su.class_counts))
    bvh.close()


def test_instrumented_orthogonal_cast_changes_nothing(rc):
    V, F = PARTS["prismatic_rot"]()
    Vt, Ft = gpu_mesh(V, F)
    bvh = rc.Bvh(Vt, Ft)
    P, Nn, f, _ = oracle.sample_area(V, F, 3000, seed=1)
    Pt, Nt, ft = torch.from_numpy(P).cuda(), torch.from_numpy(Nn).cuda(), torch.from_numpy(f).cuda()
    out = []
    for stats in (0, 1):
        p = rc.rc_params_default(collect_stats=stats)
        fr = rc.rc_frame_candidates(bvh.h, p)
        ctr = torch.zeros(8, dtype=torch.int64, device="cuda")
        rc.rc_frame_select(bvh.h, Pt, Nt, ft, p, fr, ctr)
        mask = torch.zeros(len(P), dtype=torch.uint8, device="cuda")
        trav = torch.zeros((len(P), 6), dtype=torch.float32, device="cuda")
        c2 = torch.zeros(8, dtype=torch.int64, device="cuda")
        rc.rc_orthogonal_cast(bvh.h, Pt, Nt, p, mask, trav, c2)
        out.append((fr.best, [gpu_outcome(fr.setups[k]) for k in range(fr.k)], mask.cpu().numpy(),
                    ctr.cpu().numpy(), c2.cpu().numpy()))
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1] and np.array_equal(out[0][2], out[1][2])
    c, c2 = out[1][3], out[1][4]
    assert np.array_equal(c[:4], out[0][3][:4]) and c[4] >= c[0] and c[5] > 0
    assert out[0][3][4] == 0 and c2[4] >= c2[0] > 0
    with pytest.raises(rc.RcError):
        rc.rc_orthogonal_cast(bvh.h, Pt, Nt, rc.rc_params_default(collect_stats=1), mask, trav, None)
    bvh.close()


def test_frame_select_edge_cases(rc):
    V, F = synth.cube(20.0, 0)
    Vt, Ft = gpu_mesh(V, F)
    bvh = rc.Bvh(Vt, Ft)
    p = rc.rc_params_default()
    fr = rc.rc_frame_candidates(bvh.h, p)
    assert fr.source[0] == rc.RC_FRAME_GIVEN and fr.k >= 1
    # no points: every frame has zero setups; the smallest box wins
    e = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    rc.rc_frame_select(bvh.h, e, e, torch.zeros(0, dtype=torch.int32, device="cuda"), p, fr)
    assert all(fr.setups[c].setups_exact == 0 for c in range(fr.k))
    assert fr.volume[fr.best] == min(fr.volume[c] for c in range(fr.k))
    # a caller-made list of every size up to the maximum
    for k in range(1, rc.RC_MAX_FRAMES + 1):
        g = rc.Frames()
        g.k = k
        for c in range(k):
            R = synth.rotation(0.0, 0.0, 15.0 * c).astype(np.float32).reshape(9)
            for i in range(9):
                g.frame[c][i] = float(R[i])
        rc.rc_frame_select(bvh.h, e, e, torch.zeros(0, dtype=torch.int32, device="cuda"), p, g)
        assert g.best == 0          # the axis-aligned cube has the smallest box
    bvh.close()


@pytest.mark.slow
def test_full_size_prismatic_rotated(rc):
    """The prismatic part at full size (202,948 triangles, 100,000 points),
    turned off its axes: candidates bit for bit, setups per frame exactly."""
    V0, F = synth.prismatic()
    V = synth.rotate(V0, synth.rotation(12.0, -7.0, 25.0))
    Vt, Ft = gpu_mesh(V, F)
    bvh = rc.Bvh(Vt, Ft)
    p = rc.rc_params_default(tool_length=60.0)
    fr = rc.rc_frame_candidates(bvh.h, p)
    cands = ofr.frame_candidates(V, F)
    _check_candidates(rc, V, F, fr, cands)
    P, Nn, f, _ = oracle.sample_area(V, F, 100000, seed=0)
    _select_and_compare(rc, V, F, bvh, P, Nn, f, cands, p)
    bvh.close()
