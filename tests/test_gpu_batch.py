"""Batched cast: many parts of uneven size in one graph-replayed launch give
exactly the single-part results (bits and counts bit for bit), under every
knob the autotuner may pick and on repeated replays."""
import numpy as np
import pytest

import synth

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
    out = []
    for (V, F), n in zip(_parts(), counts):
        bvh = rc.Bvh(torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda())
        p = rc.rc_params_default(n_dirs=N, seed=len(out))
        P = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
        Nn = torch.zeros_like(P)
        f = torch.zeros(n, dtype=torch.int32, device="cuda")
        rc.rc_sample_points(bvh.h, n, p, P, Nn, f)
        ref_b = torch.zeros((n, (N + 31) // 32), dtype=torch.int32, device="cuda")
        ref_c = torch.zeros(n, dtype=torch.int32, device="cuda")
        rc.rc_hemisphere_cast(bvh.h, P, Nn, p, ref_b, ref_c)
        out.append(dict(bvh=bvh, P=P, N=Nn, ref_b=ref_b, ref_c=ref_c,
                        b=torch.full_like(ref_b, -1), c=torch.full_like(ref_c, -1),
                        ctr=torch.zeros(4, dtype=torch.int64, device="cuda")))
    torch.cuda.synchronize()
    return out


def _check(parts, N):
    torch.cuda.synchronize()
    for q in parts:
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
    _check(parts, N)
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
    _check(parts, N)
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
            for per_sm, fetch, launch, width in ((0, 0, 0, 0), (4, 0, 0, 0), (0, 1, 0, 2), (3, 1, 0, 2),
                                                 (0, 0, 1, 0), (0, 0, 0, 2), (0, 0, 1, 2)):
                q = rc.rc_params_default(n_dirs=N, point_order=order, tile_mode=tile, blocks_per_sm=per_sm,
                                         fetch_mode=fetch, launch_mode=launch, tree_width=width)
                bits = torch.zeros((n, (N + 31) // 32), dtype=torch.int32, device="cuda")
                cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
                rc.rc_hemisphere_cast(bvh.h, P, Nn, q, bits, cnt)
                res.append((bits, cnt))
    torch.cuda.synchronize()
    for bits, cnt in res[1:]:
        assert torch.equal(bits, res[0][0]) and torch.equal(cnt, res[0][1])
    bvh.close()
