"""Tool-aware accessibility -- TEST INFRASTRUCTURE ONLY (part of the FP64
oracle; only the tests, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` may import it).

The paper's orthogonal cast (Section 3.2) uses thin rays.  This variant
accounts for the tool: a ball-end tool of radius r touching point p has its
centre at c = p + (r + eps) n; along machining axis a its shank is sampled
by the ray from c and K parallel rays from the ring c + r (cos t_k u +
sin t_k v), t_k = 2 pi k / K, with (u, v) the branchless orthonormal basis
of a (Duff et al. 2017, sign taken as +1 for a_z >= 0).  Everything is FP64,
one rounding per operation in the order written, origins rounded to fp32.
Axis a is tool-accessible iff it is eligible (n.a >= -parallel_tol) and no
sampled ray is obstructed (the oracle's own predicate, ``Mesh.cast_rays``).
"""
from __future__ import annotations

import math

import numpy as np

from . import HIT, AMB, PARALLEL_TOL, frame_axes


def ring_table(K):
    """(cos t_k, sin t_k) with t_k = (2 pi k) / K, host libm."""
    return [(math.cos(2.0 * math.pi * k / K), math.sin(2.0 * math.pi * k / K)) for k in range(K)]


def axis_basis(a):
    """Orthonormal (u, v) of fp32 axis a in FP64 (Duff et al. 2017)."""
    ax, ay, az = (float(x) for x in a)
    sg = 1.0 if az >= 0.0 else -1.0
    q = -1.0 / (sg + az)
    bb = (ax * ay) * q
    u = (1.0 + ((sg * ax) * ax) * q, sg * bb, -sg * ax)
    v = (bb, sg + (ay * ay) * q, -ay)
    return u, v


def tool_origins(P, Nn, a, radius, K, eps=1e-4):
    """[n, 1 + K, 3] fp32 origins: the centre ray first, then the ring."""
    P64 = np.asarray(P, np.float32).astype(np.float64)
    N64 = np.asarray(Nn, np.float32).astype(np.float64)
    h = radius + eps
    c = P64 + h * N64
    u, v = axis_basis(a)
    out = np.empty((len(P64), 1 + K, 3), np.float32)
    out[:, 0] = c.astype(np.float32)
    for k, (cs, sn) in enumerate(ring_table(K)):
        rc, rs = radius * cs, radius * sn
        for d in range(3):
            out[:, 1 + k, d] = ((c[:, d] + rc * u[d]) + rs * v[d]).astype(np.float32)
    return out


def tool_cast(mesh, P, Nn, radius, K, frame=None, eps=1e-4, parallel_tol=PARALLEL_TOL):
    """Per point a 6-bit mask of tool-accessible axes and a 6-bit mask of
    axes decided by an ambiguous ray (no clear hit among the sampled rays
    but an ambiguous one)."""
    P = np.asarray(P, np.float32)
    Nn = np.asarray(Nn, np.float32)
    n = len(P)
    axes = frame_axes(frame)
    mask = np.zeros(n, np.uint8)
    amb = np.zeros(n, np.uint8)
    N64 = Nn.astype(np.float64)
    for a in range(6):
        ax = axes[a].astype(np.float64)
        nd = (N64[:, 0] * ax[0] + N64[:, 1] * ax[1]) + N64[:, 2] * ax[2]
        elig = nd >= -parallel_tol
        idx = np.flatnonzero(elig)
        if len(idx) == 0:
            continue
        O = tool_origins(P[idx], Nn[idx], axes[a], radius, K, eps).reshape(-1, 3)
        D = np.broadcast_to(axes[a], O.shape).astype(np.float32)
        st = mesh.cast_rays(O, D).reshape(len(idx), 1 + K)
        hit = (st == HIT).any(1)
        am = ~hit & (st == AMB).any(1)
        mask[idx[~hit & ~am]] |= np.uint8(1 << a)
        amb[idx[am]] |= np.uint8(1 << a)
    return mask, amb
