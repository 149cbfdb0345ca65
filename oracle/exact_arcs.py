"""Exact-rational oracle for the intersection of two great circle arcs.

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU
legs may use this module.

What it computes (the plain definition)
---------------------------------------
Two arcs a = (a1, a2) and b = (b1, b2), each the shorter great circle arc
between two FP64 points taken as exact reals (Sec. 1.2). Their great circles
have the normals n_a = a1 x a2 and n_b = b1 x b2 and meet in the two
antipodal points +-v / |v|, v = n_a x n_b: three cross products followed by a
normalisation (Sec. 1). A candidate p is a hit iff it lies on both closed
minor arcs, which we decide as for the latitude problem: (a1 x p) . n_a >= 0
and (p x a2) . n_a >= 0, and the same for b. Slot 0 holds +v / |v|, slot 1
-v / |v|; each coordinate of a hit is the exact value v_i / |v| correctly
rounded to nearest, ties to even (Sec. 3).

How
---
After scaling by powers of two, n_a, n_b and v are exact Python integers, so
every on-arc sign is the sign of an integer (the positive factor 1 / |v|
does not change it) and every coordinate is v_i sqrt(S) / S with the integer
S = v . v, rounded by exact.round_quadratic.

Conventions (our readings)
--------------------------
count = -1 : an arc is degenerate (its normal is 0) or both arcs lie on one
             great circle (v = 0).
count = 0  : no hit; also for non-finite inputs.
Unused slots hold NaN.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

from . import exact

FLAG_NEAR_ENDPOINT = 2   # a candidate within angle 2^-40 of an endpoint
FLAG_TINY_NORMAL = 4     # |n_a| or |n_b| below 2^-200 of the endpoints' norms
FLAG_NONFINITE = 8
FLAG_NEAR_PARALLEL = 16  # the great circles meet at an angle below 2^-40

ENDPOINT_LOG2 = 40
PARALLEL_LOG2 = 40
TINY_NORMAL_LOG2 = 200

_NAN = float("nan")


def _scaled(points):
    """Scale a list of FP64 3-vectors to integers by one common power of two."""
    parts = [exact.dyadic(v) for p in points for v in p]
    exps = [e for m, e in parts if m != 0]
    E = min(exps) if exps else 0
    ints = [m << (e - E) if m != 0 else 0 for m, e in parts]
    return [tuple(ints[3 * i:3 * i + 3]) for i in range(len(points))]


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1],
            a[2] * b[0] - a[0] * b[2],
            a[0] * b[1] - a[1] * b[0])


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _meet(na, nb):
    """v = n_a x n_b: the two great circles meet at +-v / |v| (Sec. 1)."""
    return _cross(na, nb)


def _sgn(x):
    return (x > 0) - (x < 0)


@dataclass
class Result:
    count: int
    pts: list = field(default_factory=lambda: [[_NAN] * 3, [_NAN] * 3])
    flags: int = 0


def _angle_below(num2: int, den2: int, log2: int) -> bool:
    """sin(angle) < 2^-log2 given sin^2 = num2 / den2 (both >= 0)."""
    return (num2 << (2 * log2)) < den2


def intersect_arcs(a1, a2, b1, b2) -> Result:
    """Exact hits of the minor arcs a1 -> a2 and b1 -> b2 (Sec. 1, Sec. 1.2)."""
    vals = [float(v) for p in (a1, a2, b1, b2) for v in p]
    if not all(math.isfinite(v) for v in vals):
        return Result(0, flags=FLAG_NONFINITE)
    A1, A2, B1, B2 = _scaled([vals[0:3], vals[3:6], vals[6:9], vals[9:12]])
    na = _cross(A1, A2)
    nb = _cross(B1, B2)
    fl = 0
    for x, y, n in ((A1, A2, na), (B1, B2, nb)):
        if (_dot(n, n) << (2 * TINY_NORMAL_LOG2)) < _dot(x, x) * _dot(y, y):
            fl |= FLAG_TINY_NORMAL
    if na == (0, 0, 0) or nb == (0, 0, 0):
        return Result(-1, flags=fl)
    v = _meet(na, nb)
    if v == (0, 0, 0):
        return Result(-1, flags=fl)
    S = _dot(v, v)
    # |v|^2 = |n_a|^2 |n_b|^2 sin^2(angle between the circles)
    if _angle_below(S, _dot(na, na) * _dot(nb, nb), PARALLEL_LOG2):
        fl |= FLAG_NEAR_PARALLEL
    # on-arc values for +v (those of -v are their negatives)
    ts = [_dot(_cross(A1, v), na), _dot(_cross(v, A2), na),
          _dot(_cross(B1, v), nb), _dot(_cross(v, B2), nb)]
    # near an endpoint: sin(angle(p, x)) = |x x v| / (|x| |v|) small
    for x in (A1, A2, B1, B2):
        c = _cross(x, v)
        if _angle_below(_dot(c, c), _dot(x, x) * S, ENDPOINT_LOG2):
            fl |= FLAG_NEAR_ENDPOINT
    res = Result(0, flags=fl)
    for slot, sigma in enumerate((1, -1)):
        if all(sigma * _sgn(t) >= 0 for t in ts):
            res.pts[slot] = [exact.round_quadratic(0, sigma * vi, S, S) for vi in v]
            res.count += 1
    return res


def _batch_worker(args):
    A1, A2, B1, B2 = args
    out = []
    for i in range(len(A1)):
        r = intersect_arcs(A1[i], A2[i], B1[i], B2[i])
        out.append((r.count, r.pts, r.flags))
    return out


def intersect_arcs_batch(A1, A2, B1, B2, processes: int | None = None):
    """Run intersect_arcs over (n, 3) arrays; returns (count, pts (n,2,3), flags)."""
    import numpy as np
    arrs = [np.asarray(x, dtype=np.float64).reshape(-1, 3) for x in (A1, A2, B1, B2)]
    n = arrs[0].shape[0]
    lists = [a.tolist() for a in arrs]
    count = np.zeros(n, dtype=np.int32)
    pts = np.full((n, 2, 3), np.nan)
    flags = np.zeros(n, dtype=np.int32)
    if processes is None or processes <= 1 or n < 2048:
        rows = _batch_worker(lists)
    else:
        import multiprocessing as mp
        chunk = (n + processes * 4 - 1) // (processes * 4)
        jobs = [tuple(l[i:i + chunk] for l in lists) for i in range(0, n, chunk)]
        with mp.get_context("spawn").Pool(processes) as pool:
            rows = [r for part in pool.map(_batch_worker, jobs) for r in part]
    for i, (c, p, f) in enumerate(rows):
        count[i] = c
        pts[i] = p
        flags[i] = f
    return count, pts, flags
