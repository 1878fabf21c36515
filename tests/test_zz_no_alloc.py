"""rc_direction_variability_noalloc against rc_direction_variability.

The no-allocation entry point is for callers that cannot let the library
allocate device memory (for example a process whose whole HBM budget is
handed to its own arena).  It keeps its scratch in one static device array
shared by all calls, so this test checks two calls in a row -- with a
different direction count, point set and weighting the second time -- to
see that the array is cleared and the direction table refreshed between
calls.  Outputs must equal the allocating entry point's exactly, except the
per-direction weighted sums, whose FP64 additions run in no fixed order
(relative 1e-12, as in the variability parity tests).  Around each call it
also checks that nothing was allocated: the device's free bytes and the
default memory pool's reserved and used bytes stay the same, and the pool's
high-water mark of used bytes does not rise during the call -- while the
same check does see the allocating entry point's scratch.  The file name
makes pytest collect it last."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# CUmemPool_attribute values of the CUDA driver API
_RESERVED, _USED, _USED_HIGH = 5, 7, 8


class _Pool:
    """The current device's default memory pool, read through the driver
    API (the pool the library's stream-ordered allocations come from)."""

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        z = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, _USED_HIGH, ctypes.byref(z)) == 0


def _outputs(n, N):
    return (torch.full((n,), -1.0, dtype=torch.float32, device="cuda"),
            torch.full((n,), 7, dtype=torch.int8, device="cuda"),
            torch.full((n,), -1.0, dtype=torch.float32, device="cuda"),
            torch.full((N,), -1.0, dtype=torch.float64, device="cuda"))


def _call(rc, name, bits, Nt, w, p, outs, pool=None):
    """One call through the C ABI into preallocated outputs.  With `pool`,
    returns whether the call allocated (free bytes or pool bytes changed,
    or the pool's used high-water mark rose above its level before)."""
    n = Nt.shape[0]
    acc, dom, conc, dira = outs
    s = rc.Summary()
    fn = getattr(rc.load(), name)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    if pool is not None:
        free0 = torch.cuda.mem_get_info()[0]
        res0, used0 = pool.get(_RESERVED), pool.get(_USED)
        pool.reset_high()
    st = fn(ptr(bits), ptr(Nt), ptr(w), n, ctypes.byref(p), ptr(acc), ptr(dom), ptr(conc), ptr(dira),
            ctypes.byref(s), stream)
    assert st == 0, rc.load().rc_last_error()
    torch.cuda.synchronize()
    allocated = None
    if pool is not None:
        allocated = (torch.cuda.mem_get_info()[0] != free0 or pool.get(_RESERVED) != res0
                     or pool.get(_USED) != used0 or pool.get(_USED_HIGH) > used0)
    return (acc.cpu().numpy().copy(), dom.cpu().numpy().copy(), conc.cpu().numpy().copy(),
            dira.cpu().numpy().copy(), s, allocated)


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
    pool = _Pool()
    # first call: area-random points, unit weights, N = 512, conc mode 0;
    # second call: face centroids with area weights, N = 256, conc mode 1
    cases = [(rc.RC_SAMPLE_AREA_RANDOM, 3000, 512, 0), (rc.RC_SAMPLE_FACE_CENTROID, len(F), 256, 1)]
    for c, (mode, n, N, cm) in enumerate(cases):
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
        oa, ob = _outputs(n, N), _outputs(n, N)
        if c == 0:
            # the first call on this device sets the array up (its device
            # address; with lazy module loading the array itself comes into
            # being here), so it is not the one checked for allocations
            _call(rc, "rc_direction_variability_noalloc", bits, Nn, wt, p, ob)
        a = _call(rc, "rc_direction_variability", bits, Nn, wt, p, oa, pool)
        b = _call(rc, "rc_direction_variability_noalloc", bits, Nn, wt, p, ob, pool)
        assert a[5], "the check does not see the allocating entry point's scratch"
        assert not b[5], "rc_direction_variability_noalloc allocated device memory"
        for x, y in zip(a[:3], b[:3]):
            assert np.array_equal(x, y)
        if wt is None:
            assert np.array_equal(a[3], b[3])
        else:
            assert np.allclose(a[3], b[3], rtol=1e-12, atol=0)
        sa, sb = a[4], b[4]
        for f in ("overall_access", "overall_access_unweighted", "mean_conc", "n_points", "n_counted",
                  "n_zero_visible", "count_sum", "weighted_count", "weight_sum", "conc_sum_q"):
            assert getattr(sa, f) == getattr(sb, f), f
        assert list(sa.axis_share) == list(sb.axis_share) and list(sa.dom_count) == list(sb.dom_count)
        assert sb.n_counted > 0 and sb.count_sum == int(cnt.sum().item())
    # more directions than the static scratch holds is refused
    p = rc.rc_params_default(n_dirs=16384)
    with pytest.raises(rc.RcError) as ei:
        rc.rc_direction_variability_noalloc(bits, Nn, p)
    assert ei.value.status == 6
    # and a malformed parameter is refused as by the allocating entry point
    q = rc.rc_params_default(n_dirs=256, conc_mode=2)
    with pytest.raises(rc.RcError) as ei:
        rc.rc_direction_variability_noalloc(bits, Nn, q)
    assert ei.value.status == 1
    bvh.close()
