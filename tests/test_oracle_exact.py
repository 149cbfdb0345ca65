"""Pins of the exact-rational oracle (oracle/exact.py) to things other than itself.

* rounding: CPython's int/int true division is correctly rounded (subnormals
  included), so round_rational must agree with it bit for bit;
  round_quadratic agrees with an 80-digit decimal evaluation;
* closed forms of Eq. 2.2: the equator (z0 = 0), meridian arcs (n_z = 0) and
  arcs mirror-symmetric about the xz-plane, whose P_x = z0 x1 / z1 is
  rational and must round bit-exactly;
* invariants of the exact candidates: |P| = 1, P . n = 0, P_z = z0, and the
  sum of the two roots;
* brute force: the intersections found by bisection of z(t) = z0 along the
  normalised chord (1-t) x1 + t x2 (no use of Eq. 2.2 at all), at 60 digits,
  on small random inputs, must equal the oracle's counts and correctly
  rounded points;
* planted mistakes: a sign flip or an index swap in the candidate formula is
  caught by the brute-force pin.
"""
import math
import random
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

from oracle import exact
from paper_2510_09892_gb300 import workloads as W

getcontext().prec = 80


def _fl(x: Fraction) -> float:
    return x.numerator / x.denominator  # correctly rounded int/int division


# --------------------------------------------------------------- rounding --
def test_round_rational_matches_cpython_division():
    rng = random.Random(1)
    for _ in range(4000):
        num = rng.randrange(-(1 << rng.randrange(1, 300)), 1 << rng.randrange(1, 300))
        den = rng.randrange(1, 1 << rng.randrange(1, 300))
        if rng.random() < 0.2:  # push into the subnormal range
            den <<= 1070
        assert exact.round_rational(num, den) == num / den


def test_round_rational_ties_to_even():
    # 1 + 2^-53 is a tie between 1 and 1 + 2^-52: even mantissa (1) wins
    assert exact.round_rational((1 << 53) + 1, 1 << 53) == 1.0
    assert exact.round_rational((1 << 53) + 3, 1 << 53) == 1.0 + 2.0 ** -51
    # smallest subnormal tie: 2^-1075 rounds to 0, 3 * 2^-1075 to 2 * 2^-1074
    assert exact.round_rational(1, 1 << 1075) == 0.0
    assert exact.round_rational(3, 1 << 1075) == 2 * 5e-324


def _dec_sqrt_quot(alpha, beta, Q, c):
    return (Decimal(alpha) + Decimal(beta) * Decimal(Q).sqrt()) / Decimal(c)


def test_round_quadratic_matches_decimal():
    rng = random.Random(2)
    for _ in range(2000):
        Q = rng.randrange(1, 1 << rng.randrange(2, 200))
        alpha = rng.randrange(-(1 << 150), 1 << 150)
        beta = rng.randrange(-(1 << 60), 1 << 60)
        c = rng.randrange(1, 1 << 120)
        d = _dec_sqrt_quot(alpha, beta, Q, c)
        want = _fl(Fraction(d))
        assert exact.round_quadratic(alpha, beta, Q, c) == want


def test_round_quadratic_perfect_square_is_exact():
    # (1 + 3*sqrt(4)) / 7 = 1 exactly
    assert exact.round_quadratic(1, 3, 4, 7) == 1.0
    assert exact.round_quadratic(-5, 1, 9, 4) == -0.5


def test_sign_quadratic_against_decimal():
    rng = random.Random(3)
    for _ in range(3000):
        Q = rng.randrange(0, 1 << 80)
        b = rng.randrange(-(1 << 40), 1 << 40)
        r = math.isqrt(Q)
        a = -b * r + rng.randrange(-3, 4)  # close to cancellation
        d = Decimal(a) + Decimal(b) * Decimal(Q).sqrt()
        want = (d > 0) - (d < 0)
        assert exact.sign_quadratic(a, b, Q) == want
    assert exact.sign_quadratic(-6, 3, 4) == 0  # -6 + 3*2


# ------------------------------------------------------------ closed forms --
def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def test_equator_closed_form():
    """z0 = 0: P = -/+ (n_y, -n_x, 0) / |n_xy| (Eq. 2.2 with s^2 = |n_xy|^2)."""
    rng = np.random.default_rng(4)
    checked = 0
    for _ in range(300):
        x1 = _unit(rng.standard_normal(3))
        x2 = _unit(rng.standard_normal(3))
        r = exact.intersect(x1, x2, 0.0)
        X1 = [Fraction(v) for v in x1]
        X2 = [Fraction(v) for v in x2]
        nx = X1[1] * X2[2] - X1[2] * X2[1]
        ny = X1[2] * X2[0] - X1[0] * X2[2]
        nxy = (Decimal(nx.numerator) / Decimal(nx.denominator)) ** 2 + \
              (Decimal(ny.numerator) / Decimal(ny.denominator)) ** 2
        norm = nxy.sqrt()
        cand = [(-Decimal(ny.numerator) / Decimal(ny.denominator) / norm,
                 Decimal(nx.numerator) / Decimal(nx.denominator) / norm),
                (Decimal(ny.numerator) / Decimal(ny.denominator) / norm,
                 -Decimal(nx.numerator) / Decimal(nx.denominator) / norm)]
        for slot in range(2):
            if not math.isnan(r.pts[slot][0]):
                assert r.pts[slot][0] == _fl(Fraction(cand[slot][0]))
                assert r.pts[slot][1] == _fl(Fraction(cand[slot][1]))
                assert r.pts[slot][2] == 0.0
                checked += 1
    assert checked > 50


def test_meridian_closed_form():
    """Arcs in the plane x = y (n_z = 0 exactly): both coordinates equal
    -/+ sign(n_y) sqrt((1 - z0^2) / 2) ... written out from Eq. 2.2 with n_y = -n_x."""
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(200):
        a1, a2 = rng.uniform(-1, 1, 2)
        z1, z2 = rng.uniform(-1, 1, 2)
        x1 = np.array([a1, a1, z1])
        x2 = np.array([a2, a2, z2])
        lo, hi = sorted([z1 / math.sqrt(2 * a1 * a1 + z1 * z1), z2 / math.sqrt(2 * a2 * a2 + z2 * z2)])
        z0 = float(rng.uniform(lo, hi))
        r = exact.intersect(x1, x2, z0)
        nx = Fraction(a1) * Fraction(z2) - Fraction(z1) * Fraction(a2)
        if nx == 0:
            continue
        # n = (nx, -nx, 0): P(sigma) = -sigma s (n_y, -n_x) / S2 = sigma s nx (1, 1) / (2 nx^2)
        val = (Decimal(1) - Decimal(z0) ** 2).sqrt() / Decimal(2).sqrt()
        sgn = 1 if nx > 0 else -1
        for slot, sigma in ((0, 1), (1, -1)):
            if not math.isnan(r.pts[slot][0]):
                want = _fl(Fraction(sigma * sgn * val))
                assert r.pts[slot][0] == want and r.pts[slot][1] == want
                checked += 1
    assert checked > 100


def test_mirror_symmetric_closed_form():
    """x2 = (x1, -y1, z1): n = (2 y1 z1, 0, -2 x1 y1), so P_x = z0 x1 / z1 exactly
    (a rational: the rounding must be bit-exact) and P_y = +-sqrt(1 - z0^2 - P_x^2)."""
    rng = np.random.default_rng(6)
    checked = 0
    for _ in range(300):
        x1 = _unit(rng.standard_normal(3))
        x2 = np.array([x1[0], -x1[1], x1[2]])
        # the arc's z-range runs from z1 up/down to its apex z1 / sqrt(x1^2 + z1^2)
        zt = x1[2] / math.sqrt(x1[0] ** 2 + x1[2] ** 2)
        z0 = float(x1[2] + rng.uniform(0, 1) * (zt - x1[2]))
        r = exact.intersect(x1, x2, z0)
        px = Fraction(z0) * Fraction(x1[0]) / Fraction(x1[2])
        assert r.count in (1, 2)
        for slot in range(2):
            if not math.isnan(r.pts[slot][0]):
                assert r.pts[slot][0] == _fl(px)
                d = Decimal(1) - Decimal(z0) ** 2 - (Decimal(px.numerator) / Decimal(px.denominator)) ** 2
                assert abs(r.pts[slot][1]) == _fl(Fraction(d.sqrt()))
                checked += 1
    assert checked >= 300
    # tangency: z0 at the apex of a symmetric arc with rational apex height
    x1 = np.array([0.75, 0.5, 1.0])
    x2 = np.array([0.75, -0.5, 1.0])
    zt = 1.0 / math.sqrt(0.75 ** 2 + 1.0)  # = 0.8 exactly
    assert zt == 0.8
    r = exact.intersect(x1, x2, 0.8)
    ex = exact.setup(x1, x2, 0.8)
    assert ex.Qi != 0 or r.count == 1  # 0.8 is not exactly 4/5 in binary: Q is tiny


# -------------------------------------------------------------- invariants --
def test_exact_invariants():
    rng = np.random.default_rng(7)
    from paper_2510_09892_gb300 import workloads as W
    A, B, z = W.uniform_arcs(200, seed=11)
    for i in range(200):
        ex = exact.setup(A[i], B[i], z[i])
        # P . n = 0 and P_z = z0 in exact integer form (c P = U + sigma sqrt(Q) V)
        assert sum(u * n for u, n in zip(ex.U, ex.N)) == 0
        assert sum(v * n for v, n in zip(ex.V, ex.N)) == 0
        assert ex.U[2] * (1 << ex.F) == ex.Z * ex.c
        assert ex.V[2] == 0
        # |c P|^2 = c^2: |U|^2 + Q |V|^2 = c^2 and U . V = 0 (the cross terms cancel)
        assert sum(u * v for u, v in zip(ex.U, ex.V)) == 0
        assert sum(u * u for u in ex.U) + ex.Qi * sum(v * v for v in ex.V) == ex.c * ex.c
        r = exact.intersect(A[i], B[i], z[i])
        for slot in range(2):
            p = np.array(r.pts[slot])
            if math.isnan(p[0]):
                continue
            assert abs(np.dot(p, p) - 1.0) < 8e-16
            assert abs(np.dot(p, np.cross(A[i], B[i]))) < 8e-16
        if r.count == 2:
            # P+ + P- = -2 z0 n_z (n_x, n_y) / S2
            nx, ny, nz = (Fraction(v) for v in np.cross(A[i], B[i]))
            s = np.array(r.pts[0]) + np.array(r.pts[1])
            nn = ex.N
            S2 = Fraction(ex.S2i)
            want_x = -2 * Fraction(z[i]) * nn[2] * nn[0] / S2
            want_y = -2 * Fraction(z[i]) * nn[2] * nn[1] / S2
            assert abs(s[0] - float(want_x)) < 4e-16 and abs(s[1] - float(want_y)) < 4e-16


# ------------------------------------------------------------- brute force --
def _bisect_hits(x1, x2, z0, prec=60):
    """Hits of the minor arc with z = z0 by bisection on the normalised chord."""
    getcontext().prec = prec
    X1 = [Decimal(v) for v in x1]
    X2 = [Decimal(v) for v in x2]
    Z0 = Decimal(z0)

    def point(t):
        c = [(1 - t) * a + t * b for a, b in zip(X1, X2)]
        nrm = (c[0] * c[0] + c[1] * c[1] + c[2] * c[2]).sqrt()
        return [v / nrm for v in c]

    def z(t):
        return point(t)[2]

    # the one interior extremum of z (if any) by golden-section search on |z - z_end|
    lo, hi = Decimal(0), Decimal(1)
    za, zb = z(lo), z(hi)
    # decide whether z has an interior max or min from the midpoint
    zm = z(Decimal("0.5"))
    pieces = [(Decimal(0), Decimal(1))]
    for sgn in (1, -1):
        a, b = Decimal(0), Decimal(1)
        for _ in range(240):
            m1 = a + (b - a) / 3
            m2 = b - (b - a) / 3
            if sgn * z(m1) < sgn * z(m2):
                a = m1
            else:
                b = m2
        t = (a + b) / 2
        if Decimal(0) < t < Decimal(1) and sgn * z(t) > max(sgn * za, sgn * zb) + Decimal(10) ** -40:
            pieces = [(Decimal(0), t), (t, Decimal(1))]
    hits = []
    for a, b in pieces:
        fa, fb = z(a) - Z0, z(b) - Z0
        if fa == 0:
            hits.append(a)
            continue
        if fb == 0:
            hits.append(b)
            continue
        if (fa > 0) == (fb > 0):
            continue
        for _ in range(220):
            m = (a + b) / 2
            fm = z(m) - Z0
            if (fm > 0) == (fa > 0):
                a, fa = m, fm
            else:
                b = m
        hits.append((a + b) / 2)
    out = []
    for t in hits:
        p = point(t)
        if not any(all(abs(p[k] - q[k]) < Decimal(10) ** -30 for k in range(3)) for q in out):
            out.append(p)
    getcontext().prec = 80
    return out


def _match_points(r, pts):
    found = [r.pts[s] for s in range(2) if not math.isnan(r.pts[s][0])]
    assert len(found) == len(pts)
    for p in pts:
        want = [_fl(Fraction(v)) for v in p[:2]]
        assert any(f[0] == want[0] and f[1] == want[1] for f in found), (found, want)


def test_brute_force_bisection_small():
    from paper_2510_09892_gb300 import workloads as W
    A, B, z = W.uniform_arcs(120, seed=12)
    for i in range(120):
        r = exact.intersect(A[i], B[i], z[i])
        if r.flags:
            continue
        pts = _bisect_hits(A[i], B[i], z[i])
        assert r.count == len(pts)
        _match_points(r, pts)


def test_brute_force_no_hit_and_two_hits():
    rng = np.random.default_rng(13)
    seen = {0: 0, 1: 0, 2: 0}
    for _ in range(150):
        x1 = _unit(rng.standard_normal(3))
        x2 = _unit(rng.standard_normal(3))
        z0 = float(rng.uniform(-1, 1))
        r = exact.intersect(x1, x2, z0)
        if r.flags:
            continue
        pts = _bisect_hits(x1, x2, z0)
        assert r.count == len(pts)
        _match_points(r, pts)
        seen[r.count] += 1
    assert seen[0] > 10 and seen[1] > 10


# -------------------------------------------------------- degenerate cases --
def test_degenerate_conventions():
    e = np.array([1.0, 0.0, 0.0])
    assert exact.intersect(e, e, 0.1).count == -1            # n = 0
    assert exact.intersect(e, -e, 0.0).count == -1           # antipodal: n = 0
    eq1, eq2 = np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0])
    assert exact.intersect(eq1, eq2, 0.0).count == -1        # coincident circles
    assert exact.intersect(eq1, eq2, 0.5).count == 0         # parallel planes
    r = exact.intersect(eq1, np.array([0.0, 0.0, 1.0]), float("nan"))
    assert r.count == 0 and r.flags & exact.FLAG_NONFINITE
    # unnormalised inputs give the same result as their normalised versions (Sec. 1.2)
    x1, x2 = np.array([1.0, 2.0, 3.0]), np.array([-2.0, 1.0, 0.5])
    a = exact.intersect(x1, x2, 0.5)
    b = exact.intersect(4 * x1, 0.5 * x2, 0.5)  # power-of-two scaling keeps inputs exact
    assert a.count == b.count and a.pts == b.pts or all(
        (math.isnan(p) and math.isnan(q)) or p == q for u, v in zip(a.pts, b.pts) for p, q in zip(u, v))


# -------------------------------------------------------- planted mistakes --
def _planted_candidate(mistake):
    orig = exact.candidate_point

    def bad(ex, sigma):
        if mistake == "sign":
            return orig(ex, -sigma)
        if mistake == "swap":
            px, py, pz = orig(ex, sigma)
            return (py, px, pz)
        raise ValueError(mistake)
    return bad


@pytest.mark.parametrize("mistake", ["sign", "swap"])
def test_planted_mistakes_are_caught(monkeypatch, mistake):
    from paper_2510_09892_gb300 import workloads as W
    monkeypatch.setattr(exact, "candidate_point", _planted_candidate(mistake))
    A, B, z = W.uniform_arcs(12, seed=12)
    caught = 0
    for i in range(12):
        r = exact.intersect(A[i], B[i], z[i])
        pts = _bisect_hits(A[i], B[i], z[i])
        try:
            _match_points(r, pts)
        except AssertionError:
            caught += 1
    assert caught >= 10


# ------------------------------------------------- second implementation --
# The same intersections derived differently, in exact rationals: a point of
# the great circle is P = alpha x1 + beta x2 (the plane of the arc), so
# alpha z1 + beta z2 = z0 and |P|^2 = 1, a quadratic in one unknown. The arc
# holds P iff alpha >= 0 and beta >= 0 ((x1 x P).n = beta |n|^2 and
# (P x x2).n = alpha |n|^2). Coordinates have the form (X + Y sqrt D) / Z and
# are rounded by refining an integer square root until both ends of the
# bracket round to the same double (float() of a Fraction rounds correctly).
def _sign_surd(u, v, D):
    """Sign of u + v sqrt(D) for rationals u, v and D >= 0."""
    su = (u > 0) - (u < 0)
    sv = (v > 0) - (v < 0) if D != 0 else 0
    if su == sv or sv == 0:
        return su
    if su == 0:
        return sv
    d = u * u - v * v * D
    return su if d > 0 else (sv if d < 0 else 0)


def _round_surd(X, Y, D, Z):
    """(X + Y sqrt D) / Z rounded to the nearest double (Z != 0)."""
    import math
    if Y == 0 or D == 0:
        return float(X / Z)
    k = 80
    while True:
        scale = 1 << k
        n = D * scale * scale
        r = math.isqrt(n.numerator // n.denominator)
        lo, hi = Fraction(r, scale), Fraction(r + 2, scale)  # sqrt D in [lo, hi]
        a = (X + Y * lo) / Z
        b = (X + Y * hi) / Z
        if float(a) == float(b):
            return float(a)
        k *= 2


def _plane_basis_hits(x1, x2, z0):
    a = [Fraction(v) for v in x1]
    b = [Fraction(v) for v in x2]
    z = Fraction(z0)
    if b[2] == 0:  # solve for the other coefficient instead
        pts = _plane_basis_hits(x2, x1, z0)
        return pts
    p0, p1 = z / b[2], -a[2] / b[2]  # beta = p0 + p1 alpha
    w = [a[i] + p1 * b[i] for i in range(3)]  # P = p0 b + alpha w
    ww = sum(c * c for c in w)
    wb = sum(w[i] * b[i] for i in range(3))
    bb = sum(c * c for c in b)
    qa, qb, qc = ww, 2 * p0 * wb, p0 * p0 * bb - 1
    D = qb * qb - 4 * qa * qc
    if D < 0:
        return []
    out = []
    for s in ((1,) if D == 0 else (1, -1)):
        # alpha = (-qb + s sqrt D) / (2 qa), beta = p0 + p1 alpha
        if _sign_surd(-qb, Fraction(s), D) < 0:
            continue
        if _sign_surd(2 * qa * p0 - p1 * qb, s * p1, D) < 0:
            continue
        pt = tuple(_round_surd(2 * qa * p0 * b[i] - qb * w[i], s * w[i], D, 2 * qa) for i in range(2))
        out.append(pt)
    return out


def test_second_implementation_plane_basis():
    """1000 seeded arcs (uniform and the stress mix): hit sets, bit for bit."""
    A, B, z = W.uniform_arcs(600, seed=77)
    A2, B2, z2 = W.stress_arcs(400, seed=78)
    A, B, z = np.concatenate([A, A2]), np.concatenate([B, B2]), np.concatenate([z, z2])
    checked = 0
    for i in range(len(z)):
        x1, x2, z0 = tuple(A[i]), tuple(B[i]), float(z[i])
        if x1[2] == 0 and x2[2] == 0:
            continue
        r = exact.intersect(x1, x2, z0)
        if r.count < 0:
            continue
        want = sorted(tuple(p[:2]) for p in r.pts if not np.isnan(p[0]))
        got = sorted(_plane_basis_hits(x1, x2, z0))
        assert len(got) == r.count and got == want, (i, got, want)
        checked += 1
    assert checked >= 990
