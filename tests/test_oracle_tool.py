"""Pins for the oracle's tool-aware accessibility (oracle/tool.py): the
thin-tool limit is the orthogonal cast, a slot admits a ball-end tool iff
the tool is narrower than the slot, the ring basis is orthonormal."""
import numpy as np
import pytest

import oracle
import synth
from oracle import tool


def test_zero_radius_without_ring_is_the_orthogonal_cast():
    for V, F in (synth.pocket_block(2), synth.box_with_pockets((100.0, 60.0, 40.0), (
            ("+z", (35.0, 65.0), (15.0, 45.0), 15.0), ("+x", (10.0, 50.0), (10.0, 30.0), 10.0)), subdiv=1)):
        P, Nn, f, _ = oracle.sample_area(V, F, 800, seed=3)
        m = oracle.Mesh(V, F)
        for frame in (None, [0.8, -0.6, 0, 0.6, 0.8, 0, 0, 0, 1]):
            a, aa = m.orthogonal(P, Nn, frame=frame)
            b, ba = tool.tool_cast(m, P, Nn, 0.0, 0, frame=frame)
            assert np.array_equal(a, b) and np.array_equal(aa, ba)


def test_slot_admits_a_tool_narrower_than_the_slot():
    # slot 6 mm wide (y 17..23), 20 mm long, 10 mm deep in the top of a block
    V, F = synth.box_with_pockets((60.0, 40.0, 30.0), (("+z", (20.0, 40.0), (17.0, 23.0), 10.0),), subdiv=2)
    m = oracle.Mesh(V, F)
    P = np.array([[30.0, 20.0, 20.0], [25.0, 19.0, 20.0]], np.float32)     # on the slot floor
    Nn = np.array([[0, 0, 1], [0, 0, 1]], np.float32)
    PZ = 1 << 4
    for r, K, open_ in ((2.5, 8, (True, False)), (3.5, 8, (False, False)), (3.5, 0, (True, True)),
                        (1.5, 4, (True, True))):
        mask, amb = tool.tool_cast(m, P, Nn, r, K)
        assert not (amb & PZ).any()      # (side axes may graze the dyadic end walls' edges)
        # point 0 at the centreline: open iff r < 3; point 1 is 2 mm from a wall: open iff r < 2
        assert tuple(bool(x & PZ) for x in mask) == open_, (r, K)


def test_ring_basis_is_orthonormal():
    rng = np.random.default_rng(4)
    for _ in range(200):
        a = rng.normal(size=3)
        a = (a / np.linalg.norm(a)).astype(np.float32)
        u, v = tool.axis_basis(a)
        M = np.array([u, v, a.astype(np.float64)])
        assert np.allclose(M @ M.T, np.eye(3), atol=1e-7)
    for a in ([0, 0, 1], [0, 0, -1], [1, 0, 0], [0, -1, 0]):
        u, v = tool.axis_basis(np.array(a, np.float32))
        assert np.allclose(np.cross(u, v), a, atol=1e-15)
    table = tool.ring_table(4)
    assert np.allclose(table, [(1, 0), (0, 1), (-1, 0), (0, -1)], atol=1e-15)
