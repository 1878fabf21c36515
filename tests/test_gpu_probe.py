"""The measurement probes (L2 random reads, FP32 issue) return plausible,
repeatable ceilings and refuse bad arguments."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_05467_gb300 as rc
    rc.load()
    return rc


def test_probes(rc):
    a = rc.rc_probe_l2(64 << 20, 128, 128)
    b = rc.rc_probe_l2(64 << 20, 128, 128)
    assert 500.0 < a < 1e6 and abs(a - b) <= 0.25 * max(a, b)
    assert rc.rc_probe_l2(64 << 20, 16, 128) > 100.0
    f = rc.rc_probe_fp32(2048)
    assert 1.0 < f < 1000.0
    for bad in ((3 << 20, 128, 128), (1 << 10, 128, 128), (64 << 20, 128, 0), (64 << 20, 48, 128)):
        with pytest.raises(rc.RcError):
            rc.rc_probe_l2(*bad)
    with pytest.raises(rc.RcError):
        rc.rc_probe_fp32(0)


def test_stream_status_after_work(rc):
    # a finished stream reports no asynchronous error
    rc.rc_probe_fp32(64)
    rc.rc_stream_status()
    import torch
    s = torch.cuda.Stream()
    rc.rc_stream_status(s)
