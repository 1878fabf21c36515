"""Batched cast: many parts of uneven size in one graph-replayed launch give
the oracle's visibility bits (bit for bit outside its ambiguous rays) and
exactly the single-part results (bits and counts bit for bit), under every
knob the autotuner may pick and on repeated replays."""
import numpy as np
import pytest

import oracle
import synth
from common import compare_bits, gpu_outcome, setup_outcomes, unpack

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_05467_gb300 as rc
    rc.load()
    return rc


def _parts():
    return [synth.pocket_block(2), synth.prismatic(h=5.0), synth.impeller(h=3.0), synth.cube(20.0, 1),
            synth.box_with_pockets((80.0, 50.0, 30.0), (("+z", (20.0, 60.0), (10.0, 40.0), 12.0),), subdiv=1),
            synth.pocket_block(0)]


def _setup(rc, N, counts):
    """Each part with the oracle's seeded sample points (so no GPU output is
    an oracle input), the oracle's own cast of them, and the single-part
    GPU cast."""
    out = []
    for (V, F), n in zip(_parts(), counts):
        bvh = rc.Bvh(torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda())
        p = rc.rc_params_default(n_dirs=N, seed=len(out))
        hP, hN, _, _ = oracle.sample_area(V, F, n, seed=len(out))
        ob, oa, oc = oracle.Mesh(V, F).hemisphere(hP, hN, N)
        P = torch.from_numpy(hP).cuda()
        Nn = torch.from_numpy(hN).cuda()
        ref_b = torch.zeros((n, (N + 31) // 32), dtype=torch.int32, device="cuda")
        ref_c = torch.zeros(n, dtype=torch.int32, device="cuda")
        rc.rc_hemisphere_cast(bvh.h, P, Nn, p, ref_b, ref_c)
        out.append(dict(bvh=bvh, P=P, N=Nn, ref_b=ref_b, ref_c=ref_c, oracle=(ob, oa, oc), nV=len(V), T=len(F),
                        b=torch.full_like(ref_b, -1), c=torch.full_like(ref_c, -1),
                        ctr=torch.zeros(4, dtype=torch.int64, device="cuda")))
    torch.cuda.synchronize()
    return out


def _check(parts, N, against_oracle=False):
    torch.cuda.synchronize()
    for q in parts:
        if against_oracle:
            gb = q["b"].cpu().numpy().view(np.uint32)
            compare_bits(gb, q["c"].cpu().numpy(), *q["oracle"], N)
        assert torch.equal(q["b"], q["ref_b"]) and torch.equal(q["c"], q["ref_c"])
        c = q["ctr"].cpu().numpy()
        assert c[0] == q["P"].shape[0] * N and c[3] == 0


@pytest.mark.parametrize("N", [64, 512, 150])
def test_batch_equals_single_part(rc, N):
    counts = [1000, 777, 1500, 1, 333, 64]
    parts = _setup(rc, N, counts)
    p = rc.rc_params_default(n_dirs=N)
    b = rc.rc_batch_create(p)
    for q in parts:
        rc.rc_batch_add_part(b, q["bvh"].h, q["P"], q["N"], q["b"], q["c"], q["ctr"])
    rc.rc_batch_launch(b)
    _check(parts, N, against_oracle=True)
    # replays of the captured graph
    for q in parts:
        q["b"].fill_(-1)
        q["c"].fill_(-1)
    rc.rc_batch_launch(b)
    rc.rc_batch_launch(b)
    _check(parts, N)
    # every knob combination the autotuner tries gives the same answer
    for order in (0, 1):
        for tile in (0, 1):
            for ppi in (1, 3):
                q2 = rc.rc_params_default(n_dirs=N, point_order=order, tile_mode=tile, points_per_item=ppi,
                                          blocks_per_sm=4)
                rc.rc_batch_set_params(b, q2)
                for q in parts:
                    q["b"].fill_(-1)
                rc.rc_batch_launch(b)
                _check(parts, N)
    for width in (2, 4):
        rc.rc_batch_set_params(b, rc.rc_params_default(n_dirs=N, tree_width=width))
        for q in parts:
            q["b"].fill_(-1)
        rc.rc_batch_launch(b)
        _check(parts, N)
    best = rc.rc_batch_autotune(b, repeats=1)
    assert best.blocks_per_sm in (4, 6, 8) and best.points_per_item in (1, 2, 4)
    for q in parts:
        q["b"].fill_(-1)
    rc.rc_batch_launch(b)
    _check(parts, N, against_oracle=True)
    rc.rc_batch_clear(b)
    rc.rc_batch_launch(b)        # empty batch: no-op
    rc.rc_batch_destroy(b)
    for q in parts:
        q["bvh"].close()


def test_single_part_knobs_do_not_change_results(rc):
    V, F = synth.prismatic(h=4.0)
    bvh = rc.Bvh(torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda())
    N, n = 256, 1200
    p = rc.rc_params_default(n_dirs=N)
    P = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    Nn = torch.zeros_like(P)
    f = torch.zeros(n, dtype=torch.int32, device="cuda")
    rc.rc_sample_points(bvh.h, n, p, P, Nn, f)
    res = []
    for order in (0, 1):
        for tile in (0, 1):
            for per_sm, launch, width in ((0, 0, 0), (4, 0, 0), (3, 0, 2), (0, 1, 0), (0, 0, 2), (0, 1, 2)):
                q = rc.rc_params_default(n_dirs=N, point_order=order, tile_mode=tile, blocks_per_sm=per_sm,
                                         launch_mode=launch, tree_width=width)
                bits = torch.zeros((n, (N + 31) // 32), dtype=torch.int32, device="cuda")
                cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
                rc.rc_hemisphere_cast(bvh.h, P, Nn, q, bits, cnt)
                res.append((bits, cnt))
    torch.cuda.synchronize()
    for bits, cnt in res[1:]:
        assert torch.equal(bits, res[0][0]) and torch.equal(cnt, res[0][1])
    bvh.close()


def test_batch_budget_and_poll(rc):
    """A part that would take the batch past its HBM budget is refused with
    RC_E_OOM (and not added); rc_batch_poll reports 0 before the first launch
    and 1 once the launch's work has completed."""
    N = 64
    parts = _setup(rc, N, [500, 300])
    sizes = [12 * q["nV"] + 260 * q["T"] + q["P"].shape[0] * (24 + 4 * 2 + 8) + 64 for q in parts]
    b = rc.rc_batch_create(rc.rc_params_default(n_dirs=N), hbm_budget_bytes=sizes[0] + sizes[1] - 1)
    q0, q1 = parts
    pid = rc.rc_batch_add_part(b, q0["bvh"].h, q0["P"], q0["N"], q0["b"], q0["c"], q0["ctr"])
    with pytest.raises(rc.RcError) as ei:
        rc.rc_batch_add_part(b, q1["bvh"].h, q1["P"], q1["N"], q1["b"], q1["c"], q1["ctr"])
    assert ei.value.status == 3
    assert rc.rc_batch_poll(b, pid) == 0
    with pytest.raises(rc.RcError):
        rc.rc_batch_poll(b, 1)                      # the refused part was not added
    rc.rc_batch_launch(b)
    torch.cuda.synchronize()
    assert rc.rc_batch_poll(b, pid) == 1
    _check(parts[:1], N, against_oracle=True)
    rc.rc_batch_destroy(b)
    for q in parts:
        q["bvh"].close()


def _single_chain(rc, q, p):
    """The single-part entry points on the same points: reduction,
    classification, orthogonal cast, setups."""
    n = q["P"].shape[0]
    s = rc.rc_direction_variability(q["ref_b"], q["N"], p)
    lab = rc.rc_classify(s, p)
    mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
    trav = torch.zeros((n, 6), dtype=torch.float32, device="cuda")
    ctr = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc.rc_orthogonal_cast(q["bvh"].h, q["P"], q["N"], p, mask, trav, ctr)
    su = rc.rc_min_setups(q["bvh"].h, mask, trav, q["face"], p)
    return s, lab, su, mask, ctr.cpu().numpy()


@pytest.mark.parametrize("frame", [None, [0.8, -0.6, 0, 0.6, 0.8, 0, 0, 0, 1]])
def test_batch_whole_path_equals_single_part_and_oracle(rc, frame):
    """Analysis parts: one graph casts every part, then reduces, casts the six
    axes and counts classes per part.  Each part's results equal the
    single-part entry points on the same points exactly, and the oracle's
    (bits outside its ambiguous rays; indicators and label exactly when it
    saw no ambiguous ray; setups among the outcomes its ambiguous axis rays
    allow); a cast-only part in the same batch is unaffected; a replay gives
    the same results."""
    N = 128
    kw = {} if frame is None else {"frame": frame}
    p = rc.rc_params_default(n_dirs=N, tool_length=40.0, **kw)
    counts = [900, 700, 1200, 1, 333, 64]
    parts = _setup(rc, N, counts)
    meshes = _parts()
    b = rc.rc_batch_create(p)
    ids = []
    for k, q in enumerate(parts):
        V, F = meshes[k]
        _, _, f, _ = oracle.sample_area(V, F, q["P"].shape[0], seed=k)
        q["face"] = torch.from_numpy(f).cuda()
        if k == 3:
            ids.append(rc.rc_batch_add_part(b, q["bvh"].h, q["P"], q["N"], q["b"], q["c"], q["ctr"]))
        else:
            ids.append(rc.rc_batch_add_analysis(b, q["bvh"].h, q["P"], q["N"], q["face"], q["b"], q["c"]))
    rc.rc_batch_launch(b)
    res = rc.rc_batch_results(b, len(parts))
    torch.cuda.synchronize()
    for k, (q, r) in enumerate(zip(parts, res)):
        V, F = meshes[k]
        n = q["P"].shape[0]
        gb = q["b"].cpu().numpy().view(np.uint32)
        compare_bits(gb, q["c"].cpu().numpy(), *q["oracle"], N)
        assert torch.equal(q["b"], q["ref_b"]) and torch.equal(q["c"], q["ref_c"])
        if k == 3:
            assert r.setups_ran == 0 and q["ctr"].cpu().numpy()[0] == n * N
            continue
        s, lab, su, mask, octr = _single_chain(rc, q, p)
        assert r.summary.overall_access == s.overall_access and r.summary.mean_conc == s.mean_conc
        assert list(r.summary.axis_share) == list(s.axis_share) and r.label == lab
        assert r.setups_ran == 1 and (r.setups.setups_exact, r.setups.setups_greedy) == (su.setups_exact, su.setups_greedy)
        assert list(r.setups.class_counts) == list(su.class_counts) and list(r.setups.mask_hist) == list(su.mask_hist)
        assert r.cast_counters[0] == n * N and r.cast_counters[3] == 0 and r.ortho_counters[0] == octr[0]
        # against the oracle
        hP, hN = q["P"].cpu().numpy(), q["N"].cpu().numpy()
        ob, oa, oc = q["oracle"]
        n_amb = int(unpack(oa, N).sum())
        M, ac, dom, conc, c2 = oracle.variability(ob, hN, N)
        os_ = oracle.summary(c2, dom, conc, N)
        if n_amb == 0:
            assert r.summary.overall_access == os_["overall_access"] and r.label == oracle.classify(os_)
        m = oracle.Mesh(V, F)
        om, oam = m.orthogonal(hP, hN, frame=frame)
        outs, _, _ = setup_outcomes(om, oam, oracle.travel(V, hP, frame=frame), q["face"].cpu().numpy(),
                                    oracle.fixture_faces(V, F, frame=frame), p.tool_length)
        if outs is not None:
            assert gpu_outcome(r.setups) in outs
    # results refer to the last launch: after a change they wait for the next one
    rc.rc_batch_set_params(b, p)
    with pytest.raises(rc.RcError):
        rc.rc_batch_results(b, len(parts))
    # a replay of the graph gives the same results
    rc.rc_batch_launch(b)
    res2 = rc.rc_batch_results(b, len(parts))
    for r, r2 in zip(res, res2):
        assert r.summary.overall_access == r2.summary.overall_access and r.setups.setups_exact == r2.setups.setups_exact
        assert list(r.setups.mask_hist) == list(r2.setups.mask_hist)
    rc.rc_batch_destroy(b)
    for q in parts:
        q["bvh"].close()


@pytest.mark.slow
def test_full_size_batched(rc):
    """The batched configuration at full size, in the benchmark's launch: 64
    parts from the three families (10k-500k triangles, log-uniform), 2 points
    per mm^2 up to 200k, 512 directions, all added for analysis and run in
    one graph.  Every part: all 512 rays of 48 random points against the
    oracle (bit for bit outside its ambiguous rays) and its ray counter;
    four parts' part-level results against the single-part chain."""
    import bench
    from common import gpu_mesh
    rng = np.random.default_rng(0)
    N = 512
    p = rc.rc_params_default(n_dirs=N, seed=0, tool_length=60.0)
    b = rc.rc_batch_create(p)
    items = []
    for k in range(64):
        fam = int(rng.integers(3))
        t = float(np.exp(rng.uniform(np.log(1e4), np.log(5e5))))
        V, F = synth.part_family(fam, t, rng)
        n = int(min(200_000, round(2.0 * bench._area(V, F))))
        hP, hN, hf, _ = oracle.sample_area(V, F, n, seed=0)
        bvh = rc.Bvh(*gpu_mesh(V, F))
        q = dict(V=V, F=F, bvh=bvh, P=torch.from_numpy(hP).cuda(), N=torch.from_numpy(hN).cuda(),
                 face=torch.from_numpy(hf).cuda(), b=torch.zeros((n, N // 32), dtype=torch.int32, device="cuda"),
                 c=torch.zeros(n, dtype=torch.int32, device="cuda"), hP=hP, hN=hN)
        rc.rc_batch_add_analysis(b, bvh.h, q["P"], q["N"], q["face"], q["b"], q["c"])
        items.append(q)
    rc.rc_batch_launch(b)
    res = rc.rc_batch_results(b, len(items))
    torch.cuda.synchronize()
    pick = np.random.default_rng(1)
    for k, (q, r) in enumerate(zip(items, res)):
        n = q["hP"].shape[0]
        assert r.cast_counters[0] == n * N and r.cast_counters[3] == 0 and r.ortho_counters[3] == 0
        idx = np.sort(pick.choice(n, size=min(48, n), replace=False))
        gb = q["b"].cpu().numpy().view(np.uint32)
        gc = q["c"].cpu().numpy()
        ob, oa, oc = oracle.Mesh(q["V"], q["F"]).hemisphere(q["hP"][idx], q["hN"][idx], N)
        compare_bits(gb[idx], gc[idx], ob, oa, oc, N)
        if k < 4:
            q["ref_b"] = q["b"]
            s, lab, su, mask, octr = _single_chain(rc, q, p)
            assert r.summary.overall_access == s.overall_access and r.label == lab
            assert (r.setups.setups_exact, r.setups.setups_greedy) == (su.setups_exact, su.setups_greedy)
            assert list(r.setups.mask_hist) == list(su.mask_hist)
    rc.rc_batch_destroy(b)
    for q in items:
        q["bvh"].close()
