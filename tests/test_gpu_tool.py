"""Tool-aware accessibility on the GPU against the oracle (oracle/tool.py):
masks bit for bit outside the oracle's ambiguous axes."""
import numpy as np
import pytest

import oracle
import synth
from oracle import tool

from common import gpu_mesh

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_05467_gb300 as rc
    rc.load()
    return rc


PARTS = {
    "slot": lambda: synth.box_with_pockets((60.0, 40.0, 30.0), (("+z", (20.0, 40.0), (17.0, 23.0), 10.0),),
                                           subdiv=2),
    "multi_pocket": lambda: synth.box_with_pockets((100.0, 60.0, 40.0), (
        ("+z", (35.0, 65.0), (15.0, 45.0), 15.0), ("+x", (10.0, 50.0), (10.0, 30.0), 10.0)), subdiv=1),
    "prismatic_coarse": lambda: synth.prismatic(h=5.0),
}


@pytest.mark.parametrize("name", list(PARTS))
@pytest.mark.parametrize("radius,K", [(0.0, 0), (1.5, 8), (4.0, 8), (2.0, 16), (3.0, 3)])
def test_tool_cast_matches_oracle(rc, name, radius, K):
    V, F = PARTS[name]()
    bvh = rc.Bvh(*gpu_mesh(V, F))
    frame = None
    if name == "multi_pocket" and K == 8:
        frame = [0.8, -0.6, 0, 0.6, 0.8, 0, 0, 0, 1]
    elif name == "prismatic_coarse" and K == 16:
        frame = [1.0, 0.3, 0.0, 0.0, 2.0, 0.25, 0.1, 0.0, 0.5]    # sheared, non-unit columns
    kw = {} if frame is None else {"frame": frame}
    p = rc.rc_params_default(**kw)
    P, Nn, f, _ = oracle.sample_area(V, F, 1500, seed=6)
    Pt, Nt = torch.from_numpy(P).cuda(), torch.from_numpy(Nn).cuda()
    mask = torch.zeros(len(P), dtype=torch.uint8, device="cuda")
    ctr = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc.rc_tool_cast(bvh.h, Pt, Nt, p, radius, K, mask, ctr)
    gm = mask.cpu().numpy()
    om, oam = tool.tool_cast(oracle.Mesh(V, F), P, Nn, radius, K, frame=frame)
    # compare axis by axis outside the oracle's ambiguous axes
    assert np.array_equal(gm & ~oam, om & ~oam)
    c = ctr.cpu().numpy()
    assert c[3] == 0 and c[0] > 0
    if radius == 0.0 and K == 0:
        m2 = torch.zeros_like(mask)
        trav = torch.zeros((len(P), 6), dtype=torch.float32, device="cuda")
        rc.rc_orthogonal_cast(bvh.h, Pt, Nt, p, m2, trav)
        assert torch.equal(mask, m2)
    bvh.close()


def test_tool_cast_arguments(rc):
    V, F = PARTS["slot"]()
    bvh = rc.Bvh(*gpu_mesh(V, F))
    p = rc.rc_params_default()
    P = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    m = torch.zeros(4, dtype=torch.uint8, device="cuda")
    for r, K in ((-1.0, 4), (float("nan"), 4), (1.0, -1), (1.0, 65)):
        with pytest.raises(rc.RcError):
            rc.rc_tool_cast(bvh.h, P, P, p, r, K, m)
    e = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    rc.rc_tool_cast(bvh.h, e, e, p, 1.0, 4, torch.zeros(0, dtype=torch.uint8, device="cuda"))
    bvh.close()
