"""Serving loop: requests admitted while others run give the oracle's
results (visibility bits outside its ambiguous rays, indicators, label and
setups) and exactly the result of the same request analysed alone
(rc_analyze_part); requests really run side by side; resident parts are
refitted when their triangle list is unchanged, a request that can never fit
the budget is rejected, and a failing request does not disturb the others."""
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


def _alone(rc, V, F, n, p):
    W = (p.n_dirs + 31) // 32
    bits = np.zeros((n, W), np.uint32)
    cnt = np.zeros(n, np.int32)
    r = rc.rc_analyze_part(V, F, n, p, bits=bits, count=cnt)
    return r, bits, cnt


def _same(a, b):
    sa, sb = a.summary, b.summary
    assert sa.overall_access == sb.overall_access and sa.mean_conc == sb.mean_conc
    assert list(sa.axis_share) == list(sb.axis_share) and sa.count_sum == sb.count_sum
    assert a.label == b.label and a.setups_ran == b.setups_ran
    assert a.setups.setups_exact == b.setups.setups_exact and a.setups.setups_greedy == b.setups.setups_greedy
    assert list(a.setups.class_counts) == list(b.setups.class_counts)
    assert list(a.cast_counters)[:1] == list(b.cast_counters)[:1]


def _against_oracle(V, F, n, p, bits, cnt, res):
    """A served request against the oracle run on the same seeded points:
    bits and counts outside its ambiguous rays; indicators and label exactly
    when no ray is ambiguous, else within the ambiguous rays' share; setups
    among the outcomes its ambiguous axis rays allow."""
    N = p.n_dirs
    P, Nn, f, _ = oracle.sample_area(V, F, n, seed=p.seed)
    m = oracle.Mesh(V, F)
    ob, oa, oc = m.hemisphere(P, Nn, N)
    compare_bits(bits, cnt, ob, oa, oc, N)
    n_amb = int(unpack(oa, N).sum())
    M, ac, dom, conc, c2 = oracle.variability(ob, Nn, N)
    s = oracle.summary(c2, dom, conc, N)
    g = res.summary
    if n_amb == 0:
        assert g.overall_access == s["overall_access"] and list(g.axis_share) == s["axis_share"]
        assert g.mean_conc == s["mean_conc"] and res.label == oracle.classify(s)
    else:
        assert abs(g.overall_access - s["overall_access"]) <= max(1e-4, n_amb / (n * N))
    if res.setups_ran:
        om, oam = m.orthogonal(P, Nn)
        outs, _, _ = setup_outcomes(om, oam, oracle.travel(V, P), f, oracle.fixture_faces(V, F), p.tool_length)
        if outs is not None:
            assert gpu_outcome(res.setups) in outs


def _overlap(results):
    """Some two requests whose [t_start, t_end] intervals overlap."""
    for i, a in enumerate(results):
        for b in results[i + 1:]:
            if max(a.t_start, b.t_start) < min(a.t_end, b.t_end):
                return True
    return False


def test_requests_in_a_mix_equal_requests_alone(rc):
    p = rc.rc_params_default(n_dirs=256, always_setups=1, tool_length=40.0)
    jobs = [
        (1, synth.perturbed_part(3, 0.0), 3000),
        (2, synth.prismatic(h=3.0), 5000),
        (3, synth.impeller(h=2.0), 4000),
        (1, synth.perturbed_part(3, 2.5), 3000),    # same triangle list: refit
        (4, synth.cube(20.0, 2), 500),
        (5, synth.deep_hole(), 800),
        (2, synth.prismatic(h=3.0), 2500),          # same part, fewer points
    ]
    srv = rc.rc_server_create(p, slots=3, hbm_budget_bytes=8 << 30)
    ids = [rc.rc_server_submit(srv, key, V, F, n) for key, (V, F), n in jobs]
    res = [rc.rc_server_wait(srv, i, timeout_s=300.0) for i in ids]
    for r, (key, (V, F), n) in zip(res, jobs):
        assert r.status == 0, r.message
        assert r.t_submit <= r.t_admit <= r.t_start <= r.t_end
        alone, bits, cnt = _alone(rc, V, F, n, p)
        _same(r.result, alone)
    assert res[0].rebuilt == 1 and res[3].rebuilt == 0 and res[6].rebuilt == 0
    # the mix really ran side by side: some two requests were on the GPU at once
    assert _overlap(res)
    # the resident maps are those of each key's last request, and the oracle's
    for j in (3, 2, 6, 4, 5):
        key, (V, F), n = jobs[j]
        rb, rcnt = rc.rc_server_read_bits(srv, key, n, p.n_dirs)
        alone, bits, cnt = _alone(rc, V, F, n, p)
        assert np.array_equal(rb, bits) and np.array_equal(rcnt, cnt)
        _against_oracle(V, F, n, p, rb, rcnt, res[j].result)
    st = rc.rc_server_get_stats(srv)
    assert st.completed == len(jobs) and st.failed == 0 and st.resident_parts == 5
    rc.rc_server_destroy(srv)


def test_served_direction_count_not_a_multiple_of_32(rc):
    """The paper's 150 directions: rows of ceil(150/32) = 5 words, read back
    whole; the results against the oracle; a bits buffer that is too small
    is refused instead of overrun."""
    p = rc.rc_params_default(n_dirs=150, always_setups=1, tool_length=40.0, seed=3)
    jobs = [(21, synth.pocket_block(2), 700), (22, synth.prismatic(h=4.0), 1500), (23, synth.deep_hole(), 300)]
    srv = rc.rc_server_create(p, slots=3, hbm_budget_bytes=4 << 30)
    ids = [rc.rc_server_submit(srv, key, V, F, n) for key, (V, F), n in jobs]
    res = [rc.rc_server_wait(srv, i, timeout_s=300.0) for i in ids]
    for r, (key, (V, F), n) in zip(res, jobs):
        assert r.status == 0, r.message
        rb, rcnt = rc.rc_server_read_bits(srv, key, n, 150)
        assert rb.shape == (n, 5) and not (rb[:, 4] >> 22).any()     # bits 150..159 are 0
        alone, bits, cnt = _alone(rc, V, F, n, p)
        assert np.array_equal(rb, bits) and np.array_equal(rcnt, cnt)
        _same(r.result, alone)
        _against_oracle(V, F, n, p, rb, rcnt, r.result)
    import ctypes
    key, (V, F), n = jobs[0]
    small = np.zeros((n, 4), np.uint32)
    st = rc.load().rc_server_read_bits(ctypes.c_void_p(srv), ctypes.c_uint64(key),
                                       small.ctypes.data_as(ctypes.c_void_p), small.size, None, n)
    assert st == 1 and b"h_bits" in rc.load().rc_last_error()
    rc.rc_server_destroy(srv)


def test_budget_rejection_and_failure_isolation(rc):
    p = rc.rc_params_default(n_dirs=64)
    V, F = synth.pocket_block(2)
    srv = rc.rc_server_create(p, slots=2, hbm_budget_bytes=1 << 20)
    big = rc.rc_server_submit(srv, 9, *synth.prismatic(h=3.0), 20000)
    r = rc.rc_server_wait(srv, big, timeout_s=60.0)
    assert r.status == 3                                        # RC_E_OOM: never fits
    rc.rc_server_destroy(srv)

    srv = rc.rc_server_create(p, slots=2, hbm_budget_bytes=1 << 30)
    bad = F.copy()
    bad[5, 1] = len(V) + 7                                      # index out of range
    ids = [rc.rc_server_submit(srv, 1, V, F, 300), rc.rc_server_submit(srv, 2, V, bad, 300),
           rc.rc_server_submit(srv, 3, V, F, 400)]
    res = [rc.rc_server_wait(srv, i, timeout_s=60.0) for i in ids]
    assert res[0].status == 0 and res[2].status == 0
    assert res[1].status == 1 and b"outside" in res[1].message
    alone, _, _ = _alone(rc, V, F, 400, p)
    _same(res[2].result, alone)
    st = rc.rc_server_get_stats(srv)
    assert st.failed == 1 and st.completed == 2
    with pytest.raises(rc.RcError):
        rc.rc_server_wait(srv, 12345, timeout_s=0.1)            # unknown id
    rc.rc_server_destroy(srv)


def test_incremental_resubmission_equals_the_standalone_chain(rc):
    """With cfg.incremental a re-submission with the same triangle list keeps
    the points on their faces and casts only what the edit can change; its
    bits and summary equal a full cast of the edited part at those points."""
    p = rc.rc_params_default(n_dirs=256, always_setups=1, tool_length=40.0, seed=4)
    V0, F = synth.perturbed_part(3, 0.0)
    V1, _ = synth.perturbed_part(3, 2.0, deepen_mm=1.5)
    n = 3000
    srv = rc.rc_server_create(p, slots=2, hbm_budget_bytes=4 << 30, incremental=1)
    a = rc.rc_server_wait(srv, rc.rc_server_submit(srv, 7, V0, F, n), timeout_s=120.0)
    b = rc.rc_server_wait(srv, rc.rc_server_submit(srv, 7, V1, F, n), timeout_s=120.0)
    c = rc.rc_server_wait(srv, rc.rc_server_submit(srv, 7, V1, F, n + 1), timeout_s=120.0)   # other n: full
    assert a.status == b.status == c.status == 0
    assert (a.updated, b.updated, c.updated) == (0, 1, 0) and b.rebuilt == 0
    assert 0 < b.result.cast_counters[0] < n * 256
    rb, rcnt = rc.rc_server_read_bits(srv, 7, n + 1, 256)
    rc.rc_server_destroy(srv)
    # standalone chain on the GPU: sample on the unedited part, keep the
    # points on their faces on the edited one, cast in full
    srv = rc.rc_server_create(p, slots=1, hbm_budget_bytes=4 << 30, incremental=1)
    rc.rc_server_wait(srv, rc.rc_server_submit(srv, 8, V0, F, n), timeout_s=120.0)
    b2 = rc.rc_server_wait(srv, rc.rc_server_submit(srv, 8, V1, F, n), timeout_s=120.0)
    ub, ucnt = rc.rc_server_read_bits(srv, 8, n, 256)
    rc.rc_server_destroy(srv)
    b0 = rc.Bvh(torch.from_numpy(V0).cuda(), torch.from_numpy(F).cuda())
    b1 = rc.Bvh(torch.from_numpy(V1).cuda(), torch.from_numpy(F).cuda())
    P = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    Nn = torch.zeros_like(P)
    f = torch.zeros(n, dtype=torch.int32, device="cuda")
    rc.rc_sample_points(b0.h, n, p, P, Nn, f)
    rc.rc_sample_points_on_faces(b1.h, p, f, P, Nn)
    bits = torch.zeros((n, 8), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    rc.rc_hemisphere_cast(b1.h, P, Nn, p, bits, cnt)
    s = rc.rc_direction_variability(bits, Nn, p)
    torch.cuda.synchronize()
    assert np.array_equal(ub, bits.cpu().numpy().view(np.uint32)) and np.array_equal(ucnt, cnt.cpu().numpy())
    assert b2.result.summary.overall_access == s.overall_access and b2.result.summary.mean_conc == s.mean_conc
    assert b.result.summary.overall_access == s.overall_access
    # the full request that followed (other n) is the ordinary analysis
    alone, bits_a, cnt_a = _alone(rc, V1, F, n + 1, p)
    _same(c.result, alone)
    assert np.array_equal(rb, bits_a)
    b0.close()
    b1.close()


def test_largest_requests_run_one_at_a_time(rc):
    # with small_rays = 500 every request above 500 * 2^(levels-2) rays is in
    # the largest size class: two of them must not overlap, a small one may
    p = rc.rc_params_default(n_dirs=256, tool_length=40.0)
    srv = rc.rc_server_create(p, slots=3, hbm_budget_bytes=8 << 30, small_rays=500)
    V, F = synth.prismatic(h=3.0)
    Vc, Fc = synth.cube(20.0, 2)
    ids = [rc.rc_server_submit(srv, 11, V, F, 4000), rc.rc_server_submit(srv, 12, V, F, 4000),
           rc.rc_server_submit(srv, 13, Vc, Fc, 1)]
    r1, r2, r3 = [rc.rc_server_wait(srv, i, timeout_s=300.0) for i in ids]
    rc.rc_server_destroy(srv)
    for r in (r1, r2, r3):
        assert r.status == 0, r.message
    if r1.priority_level == 0:
        pytest.skip("the device has a single stream priority level")
    assert r1.priority_level == r2.priority_level > r3.priority_level == 0
    assert r2.t_start >= r1.t_end or r1.t_start >= r2.t_end
