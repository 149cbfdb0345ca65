"""The seeded input generators (paper_2510_09892_gb300/workloads.py) produce the
structures the tests and the bench rely on."""
import math
from collections import Counter

import numpy as np
import pytest

from paper_2510_09892_gb300 import workloads as W


def _fan_areas(nodes, off, fn):
    """per-cell area by the triangle fan from node 0 (Van Oosterom-Strackee)"""
    out = []
    for f in range(len(off) - 1):
        v = nodes[fn[off[f]:off[f + 1]]]
        a = v[0]
        tot = 0.0
        for i in range(1, len(v) - 1):
            b, c = v[i], v[i + 1]
            num = np.dot(a, np.cross(b - a, c - a))
            den = 1 + np.dot(a, b) + np.dot(b, c) + np.dot(c, a)
            tot += 2 * math.atan2(num, den)
        out.append(tot)
    return np.array(out)


@pytest.mark.parametrize("N", [1, 2, 3, 8])
def test_cubed_sphere_cells_form_a_closed_oriented_mesh(N):
    nodes, off, fn = W.cubed_sphere_cells(N)
    assert nodes.shape == (6 * N * N + 2, 3)
    assert len(off) == 6 * N * N + 1 and off[-1] == len(fn) == 24 * N * N
    assert np.allclose(np.linalg.norm(nodes, axis=1), 1.0, atol=4e-16)
    assert len(np.unique(np.round(nodes, 15), axis=0)) == len(nodes)  # each node once
    areas = _fan_areas(nodes, off, fn)
    assert (areas > 0).all()  # counter-clockwise seen from outside
    assert abs(areas.sum() - 4 * math.pi) < 1e-12
    # every arc is used by exactly two cells, once in each direction
    arcs = Counter()
    q = fn.reshape(-1, 4)
    for c in q:
        for i in range(4):
            arcs[(int(c[i]), int(c[(i + 1) % 4]))] += 1
    for (a, b), k in arcs.items():
        assert k == 1 and arcs[(b, a)] == 1


def test_cubed_sphere_poles():
    """Even N: both poles are nodes; odd N: each lies inside one cell."""
    for N, as_node in ((4, True), (5, False)):
        nodes, _, _ = W.cubed_sphere_cells(N)
        has = [bool(np.any(np.all(nodes == np.array([0.0, 0.0, s]), axis=1))) for s in (1.0, -1.0)]
        assert has == [as_node, as_node]


def test_polygon_cells_are_counter_clockwise_and_seeded():
    nodes, off, fn = W.polygon_cells(50, seed=3, radius=(1e-3, 0.4))
    areas = _fan_areas(nodes, off, fn)
    assert (areas > 0).all()
    k = np.diff(off)
    assert k.min() >= 3 and k.max() <= 12
    n2, o2, f2 = W.polygon_cells(50, seed=3, radius=(1e-3, 0.4))
    assert np.array_equal(nodes, n2) and np.array_equal(off, o2) and np.array_equal(fn, f2)


def test_latlon_latitudes():
    z = W.latlon_latitudes(721)
    assert z[0] == -1.0 and z[-1] == 1.0 and np.all(np.diff(z) > 0)
    assert z[360] == pytest.approx(0.0, abs=1e-16)
