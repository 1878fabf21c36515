"""Calls that fail after the library has allocated device scratch give that
scratch back: a mesh rejected by the build (an index out of range, a
non-finite vertex), points sampled on out-of-range faces and a changed-face
scan over a bad index all raise, and after many of them the default memory
pool -- where the library's stream-ordered allocations come from -- holds
the same number of used bytes as before.  The failures are made on the host
side of the contract (bad inputs the calls check), nothing faults."""
import ctypes

import numpy as np
import pytest

import synth
from common import gpu_mesh

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

_USED = 7   # CU_MEMPOOL_ATTR_USED_MEM_CURRENT


@pytest.fixture(scope="module")
def rc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_05467_gb300 as rc
    rc.load()
    return rc


def _pool_used():
    cu = ctypes.CDLL("libcuda.so.1")
    dev = ctypes.c_int()
    assert cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    v = ctypes.c_uint64()
    assert cu.cuMemPoolGetAttribute(pool, _USED, ctypes.byref(v)) == 0
    return v.value


def test_rejected_calls_leave_no_device_memory(rc):
    V, F = synth.pocket_block(1)
    Vt, Ft = gpu_mesh(V, F)
    bad_index = Ft.clone()
    bad_index[3, 1] = len(V)
    bad_value = Vt.clone()
    bad_value[5, 2] = float("nan")
    bvh = rc.Bvh(Vt, Ft)
    p = rc.rc_params_default(n_dirs=64)
    n = 16
    face_bad = torch.full((n,), len(F) + 5, dtype=torch.int32, device="cuda")
    P = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    Nn = torch.zeros_like(P)
    changed = torch.zeros(len(F), dtype=torch.uint8, device="cuda")
    calls = [
        lambda: rc.rc_build_bvh(Vt, bad_index),
        lambda: rc.rc_build_bvh(bad_value, Ft),
        lambda: rc.rc_sample_points_on_faces(bvh.h, p, face_bad, P, Nn),
        lambda: rc.rc_changed_faces(Vt, Vt, bad_index, changed),
    ]
    for call in calls:              # once each first: one-time tables and pool growth
        with pytest.raises(rc.RcError):
            call()
    torch.cuda.synchronize()
    used0 = _pool_used()
    for _ in range(10):
        for call in calls:
            with pytest.raises(rc.RcError) as ei:
                call()
            assert ei.value.status == 1        # RC_E_ARG
    torch.cuda.synchronize()
    assert _pool_used() == used0
    bvh.close()
