"""rc_direction_variability_noalloc against rc_direction_variability.

The no-allocation entry point is for callers that cannot let the library
allocate device memory (for example a process whose whole HBM budget is
handed to its own arena).  It keeps its scratch in one static device array
shared by all calls, so this test checks two calls in a row -- with a
different direction count, point set and weighting the second time -- to
see that the array is cleared and the direction table refreshed between
calls.  Outputs must equal the allocating entry point's exactly (the same
tolerance as the other variability parity tests).  The file name makes
pytest collect it last."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _call(rc, name, bits, Nt, w, p):
    n = Nt.shape[0]
    N = p.n_dirs
    acc = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    dom = torch.full((n,), 7, dtype=torch.int8, device="cuda")
    conc = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    dira = torch.full((N,), -1.0, dtype=torch.float64, device="cuda")
    s = rc.Summary()
    fn = getattr(rc.load(), name)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    st = fn(ptr(bits), ptr(Nt), ptr(w), n, ctypes.byref(p), ptr(acc), ptr(dom), ptr(conc), ptr(dira),
            ctypes.byref(s), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, rc.load().rc_last_error()
    torch.cuda.synchronize()
    return acc.cpu().numpy(), dom.cpu().numpy(), conc.cpu().numpy(), dira.cpu().numpy(), s


def test_noalloc_variability_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_05467_gb300 as rc
    rc.load()
    V, F = synth.box_with_pockets((100.0, 60.0, 40.0), (
        ("+z", (35.0, 65.0), (15.0, 45.0), 15.0), ("+x", (10.0, 50.0), (10.0, 30.0), 10.0)), subdiv=2)
    Vt = torch.from_numpy(V).cuda()
    Ft = torch.from_numpy(F).cuda()
    bvh = rc.Bvh(Vt, Ft)
    # first call: area-random points, unit weights, N = 512, conc mode 0;
    # second call: face centroids with area weights, N = 256, conc mode 1
    cases = [(rc.RC_SAMPLE_AREA_RANDOM, 3000, 512, 0), (rc.RC_SAMPLE_FACE_CENTROID, len(F), 256, 1)]
    for mode, n, N, cm in cases:
        p = rc.rc_params_default(n_dirs=N, sample_mode=mode, conc_mode=cm)
        P = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
        Nn = torch.zeros_like(P)
        face = torch.zeros(n, dtype=torch.int32, device="cuda")
        w = torch.zeros(n, dtype=torch.float64, device="cuda")
        rc.rc_sample_points(bvh.h, n, p, P, Nn, face, w)
        bits = torch.zeros((n, (N + 31) // 32), dtype=torch.int32, device="cuda")
        cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
        rc.rc_hemisphere_cast(bvh.h, P, Nn, p, bits, cnt)
        wt = w if mode == rc.RC_SAMPLE_FACE_CENTROID else None
        a = _call(rc, "rc_direction_variability", bits, Nn, wt, p)
        b = _call(rc, "rc_direction_variability_noalloc", bits, Nn, wt, p)
        for x, y in zip(a[:4], b[:4]):
            assert np.array_equal(x, y)
        sa, sb = a[4], b[4]
        for f in ("overall_access", "overall_access_unweighted", "mean_conc", "n_points", "n_counted",
                  "n_zero_visible", "count_sum", "weighted_count_q", "weight_sum_q", "conc_sum_q"):
            assert getattr(sa, f) == getattr(sb, f), f
        assert list(sa.axis_share) == list(sb.axis_share) and list(sa.dom_count) == list(sb.dom_count)
        assert sb.n_counted > 0 and sb.count_sum == int(cnt.sum().item())
    # more directions than the static scratch holds is refused
    p = rc.rc_params_default(n_dirs=16384)
    with pytest.raises(rc.RcError) as ei:
        rc.rc_direction_variability_noalloc(bits, Nn, p)
    assert ei.value.status == 6
    bvh.close()
