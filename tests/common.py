"""Shared helpers for the GPU tests: run the library through the binding and
compare with the oracle.  Imports torch lazily."""
import numpy as np

import oracle


def unpack(bits, N):
    """uint32 [n, N/32] -> bool [n, N] with bit j of row i at column j."""
    b = np.ascontiguousarray(bits, dtype=np.uint32)
    return np.unpackbits(b.view(np.uint8), axis=1, bitorder="little")[:, :N].astype(bool)


def gpu_mesh(V, F):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(V, np.float32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(F, np.int32)).cuda())


def gpu_cast(rc, h, P, Nn, params):
    import torch
    n = len(P)
    W = params.n_dirs // 32
    Pt = torch.from_numpy(np.ascontiguousarray(P, np.float32)).cuda()
    Nt = torch.from_numpy(np.ascontiguousarray(Nn, np.float32)).cuda()
    bits = torch.zeros((n, W), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    ctr = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc.rc_hemisphere_cast(h, Pt, Nt, params, bits, cnt, ctr)
    torch.cuda.synchronize()
    return bits.cpu().numpy().view(np.uint32), cnt.cpu().numpy(), ctr.cpu().numpy()


def compare_bits(gbits, gcnt, obits, oamb, ocnt, N):
    """Bit-exact comparison outside the oracle's ambiguous rays.  Returns
    (number of rays compared, number of ambiguous rays)."""
    g = unpack(gbits, N)
    o = unpack(obits, N)
    a = unpack(oamb, N)
    bad = (g != o) & ~a
    if bad.any():
        i, j = np.argwhere(bad)[0]
        raise AssertionError("visibility differs at point %d direction %d (%d rays differ)" % (i, j, bad.sum()))
    clean = ~a.any(1)
    assert np.array_equal(gcnt[clean], ocnt[clean])
    assert np.array_equal(g.sum(1), gcnt)
    return int((~a).sum()), int(a.sum())
