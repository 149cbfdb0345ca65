"""Pins of the arc x arc oracle (oracle/exact_arcs.py) to things other than itself.

* closed forms: a quarter of the equator against meridian arcs through
  Pythagorean points (p, q, 0) / r, whose intersection p / r, q / r is
  rational and must round exactly as CPython's correctly rounded division;
* brute force: the crossing found by bisection of x(t) . n_b = 0 along the
  normalised chord of arc a at 60 digits (no cross product of normals at
  all), checked for lying on arc b at the same precision;
* symmetries: swapping the arcs or reversing one moves the point to the other
  slot and changes nothing else;
* degenerate and non-finite inputs;
* planted mistakes: a wrong sign or a swapped index in the oracle's v is
  caught by the brute-force pin.
"""
from decimal import Decimal, getcontext

import numpy as np
import pytest

from oracle import exact_arcs as X
from paper_2510_09892_gb300 import workloads as W

getcontext().prec = 60


@pytest.mark.parametrize("p,q,r", [(3, 4, 5), (5, 12, 13), (8, 15, 17), (20, 21, 29),
                                   (119, 120, 169)])
def test_pythagorean_meridians_cross_the_equator_exactly(p, q, r):
    a1, a2 = (1.0, 0.0, 0.0), (0.0, 1.0, 0.0)
    b1, b2 = (float(p), float(q), -7.0), (float(p), float(q), 11.0)
    res = X.intersect_arcs(a1, a2, b1, b2)
    assert res.count == 1 and res.flags == 0
    hit = [s for s in res.pts if s[0] == s[0]]
    assert hit == [[p / r, q / r, 0.0]]


def _dec(v):
    return [Decimal(float(x)) for x in v]


def _cross_d(a, b):
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


def _dot_d(a, b):
    return sum(x * y for x, y in zip(a, b))


def brute_force(a1, a2, b1, b2):
    """Crossing of arc a with the plane of arc b by bisection along a's chord."""
    A1, A2, B1, B2 = (_dec(v) for v in (a1, a2, b1, b2))
    nb = [B1[1] * B2[2] - B1[2] * B2[1], B1[2] * B2[0] - B1[0] * B2[2],
          B1[0] * B2[1] - B1[1] * B2[0]]

    def point(t):
        c = [(1 - t) * x + t * y for x, y in zip(A1, A2)]
        nrm = _dot_d(c, c).sqrt()
        return [x / nrm for x in c]

    def f(t):
        return _dot_d(point(t), nb)

    lo, hi = Decimal(0), Decimal(1)
    flo, fhi = f(lo), f(hi)
    if flo == 0:
        p = point(lo)
    elif fhi == 0:
        p = point(hi)
    elif (flo > 0) == (fhi > 0):
        return None
    else:
        for _ in range(190):
            mid = (lo + hi) / 2
            fm = f(mid)
            if (fm > 0) == (flo > 0):
                lo, flo = mid, fm
            else:
                hi = mid
        p = point((lo + hi) / 2)
    # on arc b: (b1 x p) . n_b >= 0 and (p x b2) . n_b >= 0
    t1 = _dot_d(_cross_d(B1, p), nb)
    t2 = _dot_d(_cross_d(p, B2), nb)
    if t1 < 0 or t2 < 0:
        return None
    # slot 0 holds the point on the side of n_a x n_b
    na = _cross_d(A1, A2)
    slot = 0 if _dot_d(p, _cross_d(na, nb)) > 0 else 1
    return p, slot


def _check_against_brute(A1, A2, B1, B2, intersect=X.intersect_arcs):
    for i in range(len(A1)):
        res = intersect(A1[i], A2[i], B1[i], B2[i])
        if res.flags:
            continue
        bf = brute_force(A1[i], A2[i], B1[i], B2[i])
        if bf is None:
            assert res.count == 0, i
        else:
            p, slot = bf
            assert res.count == 1, i
            hit = res.pts[slot]
            assert hit[0] == hit[0], (i, "hit in the other slot")
            for k in range(3):
                assert abs(Decimal(hit[k]) - p[k]) <= Decimal(2.0 ** -52) * max(
                    abs(p[k]), Decimal(2.0 ** -1000)), (i, k)


def test_brute_force_bisection_agrees():
    A1, A2, B1, B2 = W.arc_pairs(300, seed=91)
    _check_against_brute(A1, A2, B1, B2)


def test_symmetries_swap_and_reverse():
    A1, A2, B1, B2 = W.arc_pairs(400, seed=92)
    for i in range(len(A1)):
        r = X.intersect_arcs(A1[i], A2[i], B1[i], B2[i])
        s = X.intersect_arcs(B1[i], B2[i], A1[i], A2[i])      # v -> -v
        t = X.intersect_arcs(A2[i], A1[i], B1[i], B2[i])      # n_a -> -n_a, v -> -v
        for other in (s, t):
            assert other.count == r.count
            assert np.array_equal(np.array(other.pts[0]), np.array(r.pts[1]), equal_nan=True)
            assert np.array_equal(np.array(other.pts[1]), np.array(r.pts[0]), equal_nan=True)


def test_degenerate_and_nonfinite():
    e = (1.0, 0.0, 0.0)
    assert X.intersect_arcs(e, e, (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)).count == -1     # n_a = 0
    assert X.intersect_arcs(e, (0.0, 1.0, 0.0), (0.0, 2.0, 0.0), (3.0, 0.0, 0.0)).count == -1
    assert X.intersect_arcs((float("nan"), 0, 0), e, e, e).count == 0
    # disjoint arcs on crossing circles
    r = X.intersect_arcs((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (-1.0, -1.0, -1.0), (-1.0, -1.0, 1.0))
    assert r.count == 0


def test_workload_classes_hit_as_built():
    A1, A2, B1, B2, k = W.arc_pairs(3000, seed=93, return_class=True)
    cnt, pts, fl = X.intersect_arcs_batch(A1, A2, B1, B2)
    ok = fl == 0
    assert (cnt[ok & (k != 4)] == 1).mean() > 0.99   # built to cross
    assert (cnt[ok & (k == 4)] == 0).mean() > 0.99   # arc b stops short


@pytest.mark.parametrize("mistake", ["sign", "index"])
def test_planted_mistakes_are_caught(monkeypatch, mistake):
    real = X._meet

    def bad_meet(na, nb):
        v = real(na, nb)
        return (-v[0], -v[1], -v[2]) if mistake == "sign" else (v[1], v[0], v[2])

    monkeypatch.setattr(X, "_meet", bad_meet)
    A1, A2, B1, B2 = W.arc_pairs(60, seed=94)
    with pytest.raises(AssertionError):
        _check_against_brute(A1, A2, B1, B2)
