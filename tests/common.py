"""Shared helpers for the GPU tests: run the library through the binding and
compare with the oracle.  Imports torch lazily."""
import struct

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
    W = (params.n_dirs + 31) // 32
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


def setup_outcomes(om, oam, trav, face, fixture, tool_length, max_amb=10):
    """Every (class counts, mask histogram, exact cover, greedy cover) the
    oracle allows: its own masks ``om`` with each of its ambiguous axis rays
    (``oam`` bits) taken either way.  Returns (set of outcomes, per-point
    classes of the points without ambiguous rays, mask of those points), or
    None for the set when there are more than ``max_amb`` ambiguous rays."""
    om = np.asarray(om, np.uint8)
    oam = np.asarray(oam, np.uint8)
    pts = np.flatnonzero(oam)
    bits = [(i, a) for i in pts for a in range(6) if (oam[i] >> a) & 1]
    clean = oam == 0
    cls0, _ = oracle.face_classes(om, trav, face, fixture, tool_length)
    if len(bits) > max_amb:
        return None, cls0[clean], clean
    outs = set()
    for c in range(1 << len(bits)):
        m = om.copy()
        for b, (i, a) in enumerate(bits):
            if (c >> b) & 1:
                m[i] |= np.uint8(1 << a)
            else:
                m[i] &= np.uint8(~(1 << a) & 0xFF)
        cls, reach = oracle.face_classes(m, trav, face, fixture, tool_length)
        viable = reach[cls == 0]
        hist = tuple(int((viable == k).sum()) for k in range(64))
        counts = tuple(int((cls == k).sum()) for k in range(4))
        outs.add((counts, hist) + oracle.setups_exact(viable) + oracle.setups_greedy(viable))
    return outs, cls0[clean], clean


def gpu_outcome(su):
    """The same tuple from a library ``Setups``."""
    hist = list(su.mask_hist)
    hist[0] = 0
    return (tuple(int(x) for x in su.class_counts), tuple(int(x) for x in hist), su.setups_exact,
            su.chosen_exact, su.setups_greedy, su.chosen_greedy)


def stl_facets(V, F):
    """Triangle corners [T, 3, 3] of a mesh."""
    return np.asarray(V, np.float32)[np.asarray(F, np.int64)]          # [T, 3, 3]


def write_stl_binary(path, V, F, header=b"binary test part"):
    tri = stl_facets(V, F)
    with open(path, "wb") as f:
        f.write(header.ljust(80, b" ")[:80])
        f.write(struct.pack("<I", len(tri)))
        for t in tri:
            f.write(struct.pack("<3f", 0.0, 0.0, 0.0))                  # stored normal: ignored
            f.write(struct.pack("<9f", *t.reshape(9).tolist()))
            f.write(b"\0\0")


def write_stl_ascii(path, V, F, name="part"):
    tri = stl_facets(V, F)
    with open(path, "w") as f:
        f.write("solid %s\n" % name)
        for t in tri:
            f.write("  facet normal 0 0 0\n    outer loop\n")
            for v in t:
                f.write("      vertex %s %s %s\n" % tuple(repr(float(x)) for x in v))
            f.write("    endloop\n  endfacet\n")
        f.write("endsolid %s\n" % name)
