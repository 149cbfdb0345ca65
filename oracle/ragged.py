"""Brute-force oracle for the ragged mesh batch: TEST INFRASTRUCTURE ONLY.

Every edge of every mesh is intersected with every latitude of its own mesh's
grid by the exact oracle (``exact.intersect``), with no candidate pruning, and
the hits are listed as records (edge, lat, root, x, y): ``edge`` is the global
edge index, ``lat`` the index into the concatenated latitude array, ``root``
the Eq. 2.2 slot (0 = the alpha* <= 0 root of Algorithm 8, 1 = the other one).
Degenerate pairs (count -1) give no records and are listed separately.
"""
from __future__ import annotations

import numpy as np

from . import exact


def intersect_ragged(A, B, edge_offsets, lat_z, lat_offsets, edges=None):
    """All hits of a mesh batch. ``edges`` optionally restricts to some edge indices.

    Returns (records, flagged, degenerate): records is an int64/float64
    structured list of (edge, lat, root, x, y); flagged the set of (edge, lat)
    pairs whose exact result carries a near-boundary flag; degenerate the set
    of (edge, lat) pairs with count -1.
    """
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    eo = np.asarray(edge_offsets, dtype=np.int64)
    lo_ = np.asarray(lat_offsets, dtype=np.int64)
    lat_z = np.asarray(lat_z, dtype=np.float64)
    mesh_of = np.searchsorted(eo, np.arange(eo[-1]), side="right") - 1
    if edges is None:
        edges = range(int(eo[-1]))
    records, flagged, degenerate = [], set(), set()
    for e in edges:
        m = int(mesh_of[e])
        for k in range(int(lo_[m]), int(lo_[m + 1])):
            r = exact.intersect(A[e], B[e], lat_z[k])
            if r.flags:
                flagged.add((int(e), k))
            if r.count < 0:
                degenerate.add((int(e), k))
                continue
            for slot in range(2):
                x, y, _ = r.pts[slot]
                if x == x:  # not NaN
                    records.append((int(e), k, slot, x, y))
    return records, flagged, degenerate
